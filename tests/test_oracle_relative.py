"""Pins of the oracle's relative (acceleration-based) opening criterion
(Sec. 2.2: the rule taken from GADGET-2, a node's quadrupole-order error
scale G M L^2 / r^4 must stay below alpha |g| of the previous step, applied
together with the geometric theta rule):

- alpha -> infinity leaves the theta-rule lists unchanged;
- alpha = 0 opens every node of positive mass: the tree is the direct sum;
- every group acceptance satisfies the per-target criterion in FP64 for every
  member of the group (the integer-gap group form is conservative);
- smaller alpha opens more (interaction counts never fall) and, with g_prev
  the exact field, bounds the worst relative force error by alpha."""
import numpy as np
import pytest

import gen


@pytest.fixture(scope="module")
def cloud(oracle_lib):
    c = gen.clumpy_cloud(12000, n_clumps=12, n_sink=8, seed=13)
    act = gen.active_subset(c.n, 0.3, seed=2)
    ad, _ = oracle_lib.direct(c.pos, c.mass, c.soft, c.is_sink, targets=np.arange(c.n))
    return c, act, ad


def _lists(t, ng):
    g = t.groups()
    return [tuple(np.sort(t.group_lists(k, g)[0])) for k in range(ng)]


def test_huge_alpha_keeps_theta_lists(oracle_lib, cloud):
    c, act, ad = cloud
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=16)
    ng = t.walk(act, 32, 0.6)
    ref = _lists(t, ng)
    t.set_relative(np.linalg.norm(ad, axis=1), 1e30)
    assert t.walk(act, 32, 0.6) == ng
    assert _lists(t, ng) == ref


def test_zero_alpha_is_direct_sum(oracle_lib, cloud):
    c, act, ad = cloud
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=16)
    t.set_relative(np.linalg.norm(ad, axis=1), 0.0)
    t.walk(act, 32, 0.6)
    a, _ = t.accel_group(act)
    np.testing.assert_allclose(a, ad[act], rtol=1e-11, atol=1e-11 * np.abs(ad).max())


def test_group_acceptances_hold_per_target(oracle_lib, cloud):
    c, act, ad = cloud
    g = np.linalg.norm(ad, axis=1)
    alpha = 2e-3
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=16)
    t.set_relative(g, alpha)
    ng = t.walk(act, 32, 0.6)
    gr = t.groups()
    nodes = t.nodes_int()
    mf = t.nodes_f64()
    key, order = t.keys()
    tg = t.group_targets()
    checked = 0
    for k in range(0, ng, 7):
        p2m, _ = t.group_lists(k, gr)
        ranks = tg[gr[k, 1]:gr[k, 1] + gr[k, 2]]
        idx = order[ranks]
        x = c.pos[idx]
        for ni in p2m:
            M = mf[ni, 0]
            L = t.L0 * 2.0 ** -int(nodes[ni, 0])
            r2 = ((mf[ni, 1:4] - x) ** 2).sum(1)
            assert np.all(M * L * L <= alpha * g[idx] * r2 * r2)
            checked += 1
    assert checked > 100


def test_alpha_tightens_lists_and_bounds_error(oracle_lib, cloud):
    c, act, ad = cloud
    g = np.linalg.norm(ad, axis=1)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=16)
    prev_work, prev_err = 0, np.inf
    for alpha in (1e-1, 1e-2, 1e-3, 1e-4):
        t.set_relative(g, alpha)
        t.walk(act, 32, 0.7)
        gr = t.groups()
        work = int((gr[:, 2] * (gr[:, 4] + gr[:, 6])).sum())
        a, _ = t.accel_group(act)
        err = (np.linalg.norm(a - ad[act], axis=1) / g[act]).max()
        assert work >= prev_work
        assert err <= prev_err
        if alpha <= 1e-2:
            assert err <= alpha
        prev_work, prev_err = work, err
