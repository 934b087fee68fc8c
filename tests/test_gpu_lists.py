"""Stored interaction lists (store_lists): the list walk writes the same lists
the per-evaluation walk uses, so both evaluation modes agree to FP32
summation order with identical interaction counts; the adjoint reuses the
forward's lists only for the same active set (content, not pointer)."""
import numpy as np
import pytest

import gen
from _helpers import oracle_tree, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _tree(c, **kw):
    import torch
    import paper_2010_11254_gb300 as sfg
    return sfg.Tree(*to_dev(c, torch), **kw)


@pytest.mark.parametrize("leaf_size,group_size", [(16, 32), (8, 16), (4, 3)])
def test_stored_lists_match_walk_evaluation(leaf_size, group_size):
    import torch
    c = gen.clumpy_cloud(1 << 15, n_clumps=64, n_sink=32, seed=21)
    rows = gen.active_subset(c.n, 0.2, seed=3)
    ca, cp = gen.cotangents(rows.size, seed=4)
    r = torch.from_numpy(rows).cuda()
    ca_t, cp_t = torch.from_numpy(ca).cuda(), torch.from_numpy(cp).cuda()
    out = {}
    for sl in (True, False):
        t = _tree(c, theta=0.5, leaf_size=leaf_size, group_size=group_size, store_lists=sl)
        a, p = t.accel(r)
        st = t.stats()
        dp, dm = t.accel_vjp(r, ca_t, cp_t)
        t.check()
        t.close()
        out[sl] = [x.cpu().numpy() for x in (a, p, dp, dm)] + [st]
    a1, p1, dp1, dm1, s1 = out[True]
    a0, p0, dp0, dm0, s0 = out[False]
    for k in ("n_groups", "n_targets", "n_p2p", "n_p2m"):
        assert s1[k] == s0[k], k
    assert np.median(rel_err(a1, a0)) <= 1e-6 and rel_err(a1, a0).max() <= 1e-4
    assert rel_err(p1, p0).max() <= 1e-6
    np.testing.assert_allclose(dp1, dp0, rtol=0, atol=1e-5 * np.abs(dp0).max())
    np.testing.assert_allclose(dm1, dm0, rtol=0, atol=1e-5 * np.abs(dm0).max())
    # and both against the oracle with its own lists
    o = oracle_tree(c, leaf_size)
    o.walk(rows, group_size, 0.5)
    ao, po = o.accel_group(rows)
    assert np.median(rel_err(a1, ao)) <= 1e-5
    assert rel_err(p1, po).max() <= 1e-6


def test_adjoint_list_reuse_follows_the_active_contents():
    """accel(A) then accel_vjp(B) must use B's lists, also when B is the same
    device array as A with its contents changed in place."""
    import torch
    c = gen.uniform_cloud(20000, seed=31, n_sink=16)
    a_rows = gen.active_subset(c.n, 0.3, seed=1)
    b_rows = gen.active_subset(c.n, 0.3, seed=2)
    assert a_rows.size == b_rows.size and not np.array_equal(a_rows, b_rows)
    ca, cp = gen.cotangents(b_rows.size, seed=5)
    ca_t, cp_t = torch.from_numpy(ca).cuda(), torch.from_numpy(cp).cuda()
    fresh = _tree(c, theta=0.6)
    ref = [x.cpu().numpy() for x in fresh.accel_vjp(torch.from_numpy(b_rows).cuda(), ca_t, cp_t)]
    fresh.close()
    t = _tree(c, theta=0.6)
    buf = torch.from_numpy(a_rows).cuda()
    t.accel(buf)
    buf.copy_(torch.from_numpy(b_rows))
    got = [x.cpu().numpy() for x in t.accel_vjp(buf, ca_t, cp_t)]
    # same active set again (reuse): identical lists, same result
    t.accel(buf)
    again = [x.cpu().numpy() for x in t.accel_vjp(buf, ca_t, cp_t)]
    t.check()
    t.close()
    for g, r_, a_ in zip(got, ref, again):
        np.testing.assert_allclose(g, r_, rtol=0, atol=1e-6 * np.abs(r_).max())
        np.testing.assert_allclose(a_, r_, rtol=0, atol=1e-6 * np.abs(r_).max())


def test_all_active_none_and_explicit_rows_agree():
    import torch
    c = gen.uniform_cloud(6000, seed=9, n_sink=4)
    t = _tree(c, theta=0.5)
    a0, p0 = (x.cpu().numpy() for x in t.accel(None))
    a1, p1 = (x.cpu().numpy() for x in t.accel(torch.arange(c.n, device="cuda")))
    t.close()
    np.testing.assert_allclose(a1, a0, rtol=1e-6, atol=1e-6 * np.abs(a0).max())
    np.testing.assert_allclose(p1, p0, rtol=1e-9)
