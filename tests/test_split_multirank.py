"""One tree's evaluation split across processes, on CPU: two gloo ranks run
the host logic of paper_2010_11254_gb300.distributed.  Each rank takes its
contiguous share of the groups (group_share, the library's rule for
sfg_set_group_share), evaluates the rows of that share -- with the FP64
oracle standing in for the GPU, which this container does not have -- and
one all-reduce assembles the outputs.  Checked: the shares cover every group
exactly once; the assembled field equals the unsplit one bit for bit (the
other rank's rows are zeros); the assembled adjoint equals the unsplit one
to FP64 rounding; the reduce-scatter form leaves each rank its block of the
summed gradients."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _setup():
    import gen
    import oracle
    c = gen.clumpy_cloud(6000, n_clumps=8, n_sink=6, seed=17)
    act = gen.active_subset(c.n, 0.4, seed=18)
    ca, cp = gen.cotangents(act.size, seed=19)
    o = oracle.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=16)
    o.walk(act, 16, 0.5)
    return c, act, ca, cp, o


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2010_11254_gb300 import distributed as D
    c, act, ca, cp, o = _setup()
    groups = o.groups()
    targets = o.keys()[1][o.group_targets()]  # sorted ranks -> particle indices
    g0, g1 = D.group_share(len(groups), rank, world)
    rows = targets[groups[g0, 1]:groups[g1 - 1, 1] + groups[g1 - 1, 2]] if g1 > g0 else targets[:0]
    rows = np.sort(rows)
    at = np.searchsorted(act, rows)
    acc = np.zeros((act.size, 3))
    phi = np.zeros(act.size)
    d_pos = np.zeros((c.n, 3))
    d_mass = np.zeros(c.n)
    if rows.size:
        acc[at], phi[at] = o.accel_group(rows)
        d_pos, d_mass = o.vjp(rows, ca[at], cp[at])
    t = [torch.from_numpy(np.ascontiguousarray(x)) for x in (acc, phi, d_pos, d_mass)]
    blk = D.scatter_rows(t[2].clone())
    D.combine(*t)
    out[rank] = dict(g=(g0, g1), acc=t[0].numpy(), phi=t[1].numpy(), d_pos=t[2].numpy(), d_mass=t[3].numpy(),
                     blk=blk.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_group_share_rule_covers_every_group_once():
    from paper_2010_11254_gb300 import distributed as D
    for ng in (0, 1, 5, 17, 1000):
        for world in (1, 2, 3, 8):
            seen = np.zeros(ng, int)
            for r in range(world):
                g0, g1 = D.group_share(ng, r, world)
                seen[g0:g1] += 1
            assert (seen == 1).all()


def test_two_rank_split_matches_unsplit():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    c, act, ca, cp, o = _setup()
    ng = len(o.groups())
    # every group exactly once
    assert res[0]["g"][0] == 0 and res[0]["g"][1] == res[1]["g"][0] and res[1]["g"][1] == ng
    a_ref, p_ref = o.accel_group(act)
    d_ref, m_ref = o.vjp(act, ca, cp)
    for rank in range(world):
        r = res[rank]
        np.testing.assert_array_equal(r["acc"], a_ref)
        np.testing.assert_array_equal(r["phi"], p_ref)
        np.testing.assert_allclose(r["d_pos"], d_ref, rtol=0, atol=1e-12 * np.abs(d_ref).max())
        np.testing.assert_allclose(r["d_mass"], m_ref, rtol=0, atol=1e-12 * np.abs(m_ref).max())
        per = -(-c.n // world)
        np.testing.assert_allclose(r["blk"], d_ref[rank * per:(rank + 1) * per], rtol=0,
                                   atol=1e-12 * np.abs(d_ref).max())
