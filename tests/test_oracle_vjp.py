"""Pins of the oracle's analytic VJP (lists frozen) against FP64 central finite
differences of the frozen-list field (Sec. 2.2: g, T = -grad grad Phi with the
same softened kernel).  The loss is L = sum_rows cot_a . a + cot_phi * phi."""
import numpy as np
import pytest

import gen


def _loss(t, pos, mass, rows, ca, cp, quad=True):
    a, p = t.eval_frozen(pos, mass, rows, quadrupole=quad)
    return float((a * ca).sum() + (p * cp).sum())


@pytest.mark.parametrize("quad", [True, False])
def test_vjp_matches_central_differences(oracle_lib, quad):
    c = gen.uniform_cloud(1500, seed=31, n_sink=16, h0=0.08)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    rows = gen.active_subset(c.n, 0.5, seed=2)
    t.walk(rows, 16, 0.6)
    ca, cp = gen.cotangents(rows.size, seed=3)
    d_pos, d_mass = t.vjp(rows, ca, cp, quadrupole=quad)
    rng = np.random.default_rng(0)
    h = 1e-6
    pick = rng.choice(c.n, 24, replace=False)
    scale = np.abs(d_pos).max()
    for k in pick:
        for ax in range(3):
            pp = c.pos.copy()
            pp[k, ax] += h
            lp = _loss(t, pp, c.mass, rows, ca, cp, quad)
            pp[k, ax] -= 2 * h
            lm = _loss(t, pp, c.mass, rows, ca, cp, quad)
            fd = (lp - lm) / (2 * h)
            assert fd == pytest.approx(d_pos[k, ax], rel=1e-6, abs=1e-6 * scale)
        mm = c.mass.copy()
        hm = 1e-6 * c.mass[k]
        mm[k] += hm
        lp = _loss(t, c.pos, mm, rows, ca, cp, quad)
        mm[k] -= 2 * hm
        lm = _loss(t, c.pos, mm, rows, ca, cp, quad)
        fd = (lp - lm) / (2 * hm)
        assert fd == pytest.approx(d_mass[k], rel=1e-6, abs=1e-6 * np.abs(d_mass).max())


def test_duplicate_rows_sum(oracle_lib):
    c = gen.uniform_cloud(800, seed=41)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    rows = np.array([5, 17, 5, 300])
    t.walk(rows, 8, 0.5)
    ca, cp = gen.cotangents(4, seed=1)
    d1, m1 = t.vjp(rows, ca, cp)
    rows2 = np.array([5, 17, 300])
    ca2 = np.stack([ca[0] + ca[2], ca[1], ca[3]])
    cp2 = np.array([cp[0] + cp[2], cp[1], cp[3]])
    d2, m2 = t.vjp(rows2, ca2, cp2)
    np.testing.assert_allclose(d1, d2, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m1, m2, rtol=1e-12, atol=1e-14)


def test_vjp_momentum_identity(oracle_lib):
    """A rigid translation of every particle leaves the frozen-list field
    unchanged, so the position gradient sums to zero over particles."""
    c = gen.uniform_cloud(600, seed=43, n_sink=4)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    rows = np.arange(c.n)
    t.walk(rows, 8, 0.7)
    ca = np.tile(np.array([[0.3, -1.0, 0.5]]), (c.n, 1))
    cp = np.zeros(c.n) + 0.7
    d_pos, _ = t.vjp(rows, ca, cp)
    assert np.abs(d_pos.sum(0)).max() <= 1e-10 * np.abs(d_pos).sum()
