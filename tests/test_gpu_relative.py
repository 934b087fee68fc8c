"""GPU walk with the relative (acceleration-based) opening criterion of
Sec. 2.2 against the oracle: groups and P2M node sets bit-exact, P2P particle
sets equal (the FP64 test is the same IEEE products on both sides), fields
within the FP32 tolerance of the other parity tests (median 1e-5, p99 2e-4,
potential 1e-6), and switching the criterion off restores the theta lists."""
import numpy as np
import pytest

import gen
from _helpers import oracle_tree, rel_err, to_dev
from test_gpu_accel import particles_of

pytestmark = pytest.mark.gpu


def _lists_equal(t, act, o):
    groups, p2m, p2p = t.debug_lists(act)
    og = o.groups()
    nodes = o.nodes_int()
    np.testing.assert_array_equal(groups[:, 0], og[:, 1])
    np.testing.assert_array_equal(groups[:, 1], og[:, 2])
    np.testing.assert_array_equal(groups[:, 2], og[:, 4])
    om = np.cumsum(np.r_[0, groups[:, 2]])
    op = np.cumsum(np.r_[0, groups[:, 3]])
    for g in range(len(og)):
        lm, lp = o.group_lists(g, og)
        np.testing.assert_array_equal(np.sort(p2m[om[g]:om[g + 1]]), np.sort(lm))
        assert particles_of(nodes, p2p[op[g]:op[g + 1]]) == particles_of(nodes, lp)
    return int(groups[:, 2].sum())


@pytest.mark.parametrize("alpha", [1e-2, 1e-3])
@pytest.mark.parametrize("kind", ["uniform", "clumpy"])
def test_relative_lists_and_fields(kind, alpha):
    import oracle
    import torch
    import paper_2010_11254_gb300 as sfg
    if kind == "uniform":
        c = gen.uniform_cloud(4096, n_sink=8)
        act = np.arange(c.n)
        theta = 0.7
    else:
        c = gen.clumpy_cloud(20000, n_clumps=16, n_sink=16, seed=14)
        act = gen.active_subset(c.n, 0.25, seed=3)
        theta = 0.5
    ad, _ = oracle.direct(c.pos, c.mass, c.soft, c.is_sink, targets=np.arange(c.n))
    gprev = np.linalg.norm(ad, axis=1)
    pos, mass, soft, sink = to_dev(c, torch)
    t = sfg.Tree(pos, mass, soft, sink, theta=theta, leaf_size=16, group_size=32)
    a_t = torch.from_numpy(act).cuda()
    t.set_relative(torch.from_numpy(gprev).cuda(), alpha)
    acc, phi = t.accel(a_t)
    assert t.status() == sfg.SFG_OK
    o = oracle_tree(c, 16)
    o.set_relative(gprev, alpha)
    o.walk(act, 32, theta)
    n_rel = _lists_equal(t, a_t, o)
    ao, po = o.accel_group(act)
    e = rel_err(acc.cpu().numpy(), ao)
    assert np.median(e) <= 1e-5 and np.percentile(e, 99) <= 2e-4
    assert rel_err(phi.cpu().numpy(), po).max() <= 1e-6
    # off again: the theta-rule lists, with fewer accepted-node entries
    t.set_relative(None)
    t.accel(a_t)
    o.set_relative(None)
    o.walk(act, 32, theta)
    n_theta = _lists_equal(t, a_t, o)
    assert n_rel != n_theta
    t.close()


def test_relative_adjoint_matches_oracle():
    import oracle
    import torch
    import paper_2010_11254_gb300 as sfg
    c = gen.uniform_cloud(3000, seed=19, n_sink=6)
    act = gen.active_subset(c.n, 0.5, seed=5)
    ad, _ = oracle.direct(c.pos, c.mass, c.soft, c.is_sink, targets=np.arange(c.n))
    gprev = np.linalg.norm(ad, axis=1)
    ca, cp = gen.cotangents(act.size, seed=8)
    pos, mass, soft, sink = to_dev(c, torch)
    t = sfg.Tree(pos, mass, soft, sink, theta=0.6, leaf_size=8, group_size=16)
    t.set_relative(torch.from_numpy(gprev).cuda(), 3e-3)
    a_t = torch.from_numpy(act).cuda()
    d_pos, d_mass = t.accel_vjp(a_t, torch.from_numpy(ca).cuda(), torch.from_numpy(cp).cuda())
    assert t.status() == sfg.SFG_OK
    t.close()
    o = oracle_tree(c, 8)
    o.set_relative(gprev, 3e-3)
    o.walk(act, 16, 0.6)
    od_pos, od_mass = o.vjp(act, ca, cp)
    scale = np.abs(od_pos).max()
    np.testing.assert_allclose(d_pos.cpu().numpy(), od_pos, rtol=0, atol=1e-4 * scale)
    np.testing.assert_allclose(d_mass.cpu().numpy(), od_mass, rtol=0, atol=1e-4 * np.abs(od_mass).max())


@pytest.mark.parametrize("G", [1e-45, 1e40])
def test_relative_lists_extreme_magnitudes(G):
    """The walk screens the relative test in FP32 and decides in FP64 where
    the FP32 sides are not normal numbers or lie close together; with G and
    |g_prev| scaled far from 1 (all of one side, or part of it, outside the
    FP32 screen's range) the lists stay those of the oracle's FP64 test."""
    import oracle
    import torch
    import paper_2010_11254_gb300 as sfg
    c = gen.clumpy_cloud(12000, n_clumps=12, n_sink=8, seed=31)
    act = gen.active_subset(c.n, 0.3, seed=2)
    ad, _ = oracle.direct(c.pos, c.mass, c.soft, c.is_sink, targets=np.arange(c.n))
    gprev = G * np.linalg.norm(ad, axis=1)
    pos, mass, soft, sink = to_dev(c, torch)
    t = sfg.Tree(pos, mass, soft, sink, theta=0.8, leaf_size=16, group_size=32, G=G)
    a_t = torch.from_numpy(act).cuda()
    t.set_relative(torch.from_numpy(gprev).cuda(), 2e-3)
    o = oracle_tree(c, 16)
    o.set_relative(gprev, 2e-3, G=G)
    o.walk(act, 32, 0.8)
    n_rel = _lists_equal(t, a_t, o)
    assert t.status() == sfg.SFG_OK
    o.set_relative(None)
    o.walk(act, 32, 0.8)
    assert n_rel != int(o.groups()[:, 4].sum())  # the relative clause opened nodes
    t.close()
