"""Ensemble of independent clouds in one forest (sfg_build_batch): every cloud
must match its own oracle tree -- keys, topology, moments and the field with
identical lists -- and no gravity may act between clouds."""
import numpy as np
import pytest

import gen
from _helpers import oracle_tree, rel_err

pytestmark = pytest.mark.gpu


def _ensemble():
    clouds = [gen.uniform_cloud(3000, seed=101, n_sink=5),
              gen.clumpy_cloud(9000, n_clumps=16, n_sink=7, seed=102),
              gen.uniform_cloud(1, seed=103),
              gen.uniform_cloud(2, seed=104, n_sink=1),
              gen.uniform_cloud(700, seed=105, h0=0.2),
              gen.clumpy_cloud(20000, n_clumps=40, n_sink=0, seed=106)]
    # far apart in space: a leak of gravity between clouds would show up
    shifts = [np.array([10.0 * k, -3.0 * k, 0.5 * k]) for k in range(len(clouds))]
    pos = np.concatenate([c.pos + s for c, s in zip(clouds, shifts)])
    mass = np.concatenate([c.mass for c in clouds])
    soft = np.concatenate([c.soft for c in clouds])
    sink = np.concatenate([c.is_sink for c in clouds])
    off = np.cumsum([0] + [c.n for c in clouds])
    parts = [gen.Cloud(c.pos + s, c.mass, c.soft, c.is_sink, 0, "part") for c, s in zip(clouds, shifts)]
    return parts, pos, mass, soft, sink, off


def _tree(torch, sfg, pos, mass, soft, sink, off, **kw):
    d = [torch.from_numpy(x).cuda() for x in (pos, mass, soft, sink)]
    return sfg.Tree(*d, offsets=list(off), **kw)


def test_batch_structure_per_cloud_is_bit_exact():
    import torch
    import paper_2010_11254_gb300 as sfg
    parts, pos, mass, soft, sink, off = _ensemble()
    t = _tree(torch, sfg, pos, mass, soft, sink, off, leaf_size=8)
    st = t.stats()
    assert st["n_clouds"] == len(parts)
    keys = t.export(sfg.FIELD_KEYS)
    order = t.export(sfg.FIELD_ORDER).astype(np.int64)
    gi = t.export(sfg.FIELD_NODE_INT).astype(np.int64)
    gf = t.export(sfg.FIELD_NODE_F64)
    frames = t.export(sfg.FIELD_FRAMES)
    for c, part in enumerate(parts):
        o = oracle_tree(part, 8)
        ok, oo = o.keys()
        np.testing.assert_array_equal(keys[off[c]:off[c + 1]], ok)
        np.testing.assert_array_equal(order[off[c]:off[c + 1]] - off[c], oo)
        np.testing.assert_array_equal(frames[c, :3], o.x0)
        assert frames[c, 3] == o.L0
        mine = np.nonzero(gi[:, 15] == c)[0]
        sel = mine[np.lexsort((gi[mine, 1], gi[mine, 0]))]
        oi = o.nodes_int()
        assert len(sel) == len(oi)
        np.testing.assert_array_equal(gi[sel, 0], oi[:, 0])
        np.testing.assert_array_equal(gi[sel, 1] - off[c], oi[:, 1])
        np.testing.assert_array_equal(gi[sel, 2], oi[:, 2])
        np.testing.assert_array_equal(gi[sel, 5], oi[:, 5])
        np.testing.assert_array_equal(gi[sel, 6:15], oi[:, 9:18])
        np.testing.assert_array_equal(gf[sel], o.nodes_f64()[:, :11])
    t.close()


@pytest.mark.parametrize("frac", [1.0, 0.3])
def test_batch_field_and_adjoint_per_cloud(frac):
    import torch
    import paper_2010_11254_gb300 as sfg
    parts, pos, mass, soft, sink, off = _ensemble()
    n = pos.shape[0]
    act = gen.active_subset(n, frac, seed=7)
    t = _tree(torch, sfg, pos, mass, soft, sink, off, theta=0.5)
    a_t = torch.from_numpy(act).cuda()
    acc, phi = t.accel(a_t)
    ca, cp = gen.cotangents(act.size, seed=8)
    d_pos, d_mass = t.accel_vjp(a_t, torch.from_numpy(ca).cuda(), torch.from_numpy(cp).cuda())
    assert t.status() == sfg.SFG_OK
    t.close()
    acc, phi, d_pos, d_mass = (x.cpu().numpy() for x in (acc, phi, d_pos, d_mass))
    for c, part in enumerate(parts):
        rows = np.nonzero((act >= off[c]) & (act < off[c + 1]))[0]
        if rows.size == 0 or part.n < 2:
            continue
        local = act[rows] - off[c]
        o = oracle_tree(part, 16)
        o.walk(local, 32, 0.5)
        ao, po = o.accel_group(local)
        assert np.median(rel_err(acc[rows], ao)) <= 1e-5
        assert rel_err(phi[rows], po).max() <= 1e-6
        op, om = o.vjp(local, ca[rows], cp[rows])
        sl = slice(off[c], off[c + 1])
        scale = np.abs(op).max()
        assert np.abs(d_pos[sl] - op).max() <= 1e-4 * scale
        assert np.abs(d_mass[sl] - om).max() <= 1e-4 * np.abs(om).max()


def test_batch_equals_separate_builds():
    import torch
    import paper_2010_11254_gb300 as sfg
    parts, pos, mass, soft, sink, off = _ensemble()
    t = _tree(torch, sfg, pos, mass, soft, sink, off)
    acc, phi = t.accel(None)
    acc, phi = acc.cpu().numpy(), phi.cpu().numpy()
    t.close()
    for c, part in enumerate(parts):
        d = [torch.from_numpy(x).cuda() for x in (part.pos, part.mass, part.soft, part.is_sink)]
        ts = sfg.Tree(*d)
        a1, p1 = ts.accel(None)
        ts.close()
        np.testing.assert_allclose(acc[off[c]:off[c + 1]], a1.cpu().numpy(), rtol=1e-6,
                                   atol=1e-6 * max(np.abs(acc[off[c]:off[c + 1]]).max(), 1e-300))
        np.testing.assert_allclose(phi[off[c]:off[c + 1]], p1.cpu().numpy(), rtol=1e-6)


def test_batch_rejects_bad_offsets():
    import torch
    import paper_2010_11254_gb300 as sfg
    parts, pos, mass, soft, sink, off = _ensemble()
    for bad in ([1] + list(off[1:]), [0, 5, 5] + list(off[3:]), list(off[:-1]) + [off[-1] + 3]):
        with pytest.raises(sfg.SfgError):
            _tree(torch, sfg, pos, mass, soft, sink, bad)


def test_cuda_graph_replay_equals_eager():
    """The field and adjoint of a batched tree captured in one CUDA graph give
    the eager results.  While a stream is captured the calls walk per
    evaluation (stored lists are sized with a synchronization), so the eager
    reference uses that mode too and must agree to the bit for the forward."""
    import torch
    import paper_2010_11254_gb300 as sfg
    parts, pos, mass, soft, sink, off = _ensemble()
    t = _tree(torch, sfg, pos, mass, soft, sink, off, theta=0.6, store_lists=False)
    t.set_timing(True)
    n = pos.shape[0]
    ca, cp = (torch.from_numpy(x).cuda() for x in gen.cotangents(n, seed=3))
    a0, p0 = t.accel(None)
    d0, m0 = t.accel_vjp(None, ca, cp)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        a1, p1 = t.accel(None)
        d1, m1 = t.accel_vjp(None, ca, cp)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert t.status() == sfg.SFG_OK
    torch.testing.assert_close(a1, a0, rtol=1e-6, atol=1e-6 * a0.abs().max().item())
    torch.testing.assert_close(p1, p0, rtol=1e-9, atol=0)
    torch.testing.assert_close(d1, d0, rtol=1e-6, atol=1e-6 * d0.abs().max().item())
    f, v = t.cloud_times()
    assert f.shape == (len(parts),) and np.all(f > 0) and np.all(v > 0)
    t.close()


def test_capture_before_any_eager_call_is_rejected():
    """A tree allocates its workspace on its first call; a first call made
    while the stream is being captured into a CUDA graph is refused with
    SFG_EINVAL (the memory would belong to the graph), and eager calls work
    afterwards."""
    import torch
    import paper_2010_11254_gb300 as sfg
    c = gen.uniform_cloud(3000, seed=12)
    pos, mass, soft, sink = (torch.from_numpy(x).cuda() for x in (c.pos, c.mass, c.soft, c.is_sink))
    t = sfg.Tree(pos, mass, soft, sink, theta=0.6, store_lists=False)
    g = torch.cuda.CUDAGraph()
    with pytest.raises(sfg.SfgError) as e:
        with torch.cuda.graph(g):
            t.accel(None)
    assert e.value.code == sfg.SFG_EINVAL
    torch.cuda.synchronize()
    a, p = t.accel(None)
    t.check()
    assert torch.isfinite(a).all()
    t.close()


def test_batch_many_clouds_small_leaves():
    """64 clouds (sizes 1 .. 5000, log-uniform) at leaf size 8 and group size
    16: per-cloud structure bit-exact and the field of every cloud equal to
    its own separate build, through the node-capacity retry if needed."""
    import torch
    import paper_2010_11254_gb300 as sfg
    rng = np.random.default_rng(64)
    sizes = np.exp(rng.uniform(0.0, np.log(5000.0), 64)).astype(int)
    clouds = [gen.uniform_cloud(int(k), seed=500 + i, h0=0.05 * (4096.0 / k) ** (1 / 3), n_sink=int(k) % 5)
              for i, k in enumerate(sizes)]
    pos = np.concatenate([c.pos for c in clouds])
    mass = np.concatenate([c.mass for c in clouds])
    soft = np.concatenate([c.soft for c in clouds])
    sink = np.concatenate([c.is_sink for c in clouds])
    off = np.cumsum([0] + [c.n for c in clouds])
    t = _tree(torch, sfg, pos, mass, soft, sink, off, leaf_size=8, group_size=16)
    keys = t.export(sfg.FIELD_KEYS)
    gi = t.export(sfg.FIELD_NODE_INT).astype(np.int64)
    gf = t.export(sfg.FIELD_NODE_F64)
    acc, phi = (x.cpu().numpy() for x in t.accel(None))
    assert t.status() == sfg.SFG_OK
    t.close()
    for c, part in enumerate(clouds):
        if c % 4:
            continue
        o = oracle_tree(part, 8)
        np.testing.assert_array_equal(keys[off[c]:off[c + 1]], o.keys()[0])
        mine = np.nonzero(gi[:, 15] == c)[0]
        sel = mine[np.lexsort((gi[mine, 1], gi[mine, 0]))]
        assert len(sel) == o.n_nodes
        np.testing.assert_array_equal(gf[sel], o.nodes_f64()[:, :11])
        d = [torch.from_numpy(x).cuda() for x in (part.pos, part.mass, part.soft, part.is_sink)]
        ts = sfg.Tree(*d, leaf_size=8, group_size=16)
        a1, p1 = (x.cpu().numpy() for x in ts.accel(None))
        ts.close()
        np.testing.assert_allclose(acc[off[c]:off[c + 1]], a1, rtol=1e-6,
                                   atol=1e-6 * max(np.abs(a1).max(), 1e-300))
        np.testing.assert_allclose(phi[off[c]:off[c + 1]], p1, rtol=1e-6)
