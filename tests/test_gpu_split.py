"""One tree's evaluation split into group shares (sfg_set_group_share), the
shares run one after another in one process on one GPU: every group is
evaluated by exactly one share (the interaction counts of the shares add up
to the unsplit call's), rows outside a share come out as zeros, and the sum
of the shares' outputs -- what one all-reduce over processes forms -- equals
the unsplit field and adjoint."""
import numpy as np
import pytest

import gen
from _helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
def test_group_shares_sum_to_the_unsplit_result(world):
    import torch
    import paper_2010_11254_gb300 as sfg
    c = gen.clumpy_cloud(30000, n_clumps=16, n_sink=8, seed=51)
    act = torch.from_numpy(gen.active_subset(c.n, 0.3, seed=52)).cuda()
    ca, cp = (torch.from_numpy(x).cuda() for x in gen.cotangents(act.numel(), seed=53))
    pos, mass, soft, sink = to_dev(c, torch)
    t = sfg.Tree(pos, mass, soft, sink, theta=0.5, leaf_size=16, group_size=16)
    a0, p0 = t.accel(act)
    st0 = t.stats()
    d0, m0 = t.accel_vjp(act, ca, cp)
    t.check()
    sa, sp = torch.zeros_like(a0), torch.zeros_like(p0)
    sd, sm = torch.zeros_like(d0), torch.zeros_like(m0)
    n_p2p = n_p2m = 0
    covered = torch.zeros(act.numel(), dtype=torch.int64, device="cuda")
    for r in range(world):
        t.set_group_share(r, world)
        a, p = t.accel(act)
        st = t.stats()
        n_p2p += st["n_p2p"]
        n_p2m += st["n_p2m"]
        d, m = t.accel_vjp(act, ca, cp)
        t.check()
        covered += (a.abs().sum(dim=1) > 0).long()
        sa += a
        sp += p
        sd += d
        sm += m
    t.set_group_share(0, 1)
    assert (n_p2p, n_p2m) == (st0["n_p2p"], st0["n_p2m"])
    assert int(covered.max()) == 1 and int(covered.min()) == 1  # every row from exactly one share
    torch.testing.assert_close(sa, a0, rtol=1e-6, atol=1e-6 * a0.abs().max().item())
    torch.testing.assert_close(sp, p0, rtol=1e-6, atol=0)
    torch.testing.assert_close(sd, d0, rtol=0, atol=1e-5 * d0.abs().max().item())
    torch.testing.assert_close(sm, m0, rtol=0, atol=1e-5 * m0.abs().max().item())
    with pytest.raises(sfg.SfgError):
        t.set_group_share(world, world)
    t.close()
