"""Pins of the oracle's jerk j = da/dt (Sec. 2.2: summed in the same pass as g,
pairs with the same softened kernel and symmetrisation, nodes by their
monopole contributions):

- the direct-sum jerk is the central time difference of the direct field
  with every particle moved along its velocity;
- with the quadrupole off, the group-form jerk is the time difference of the
  frozen-list monopole field (node centres of mass move with the node's
  mass-weighted velocity);
- a uniform velocity added to every particle changes nothing (Galilean);
- two point masses on a circle: j_1 = G m_2 (v_2 - v_1) / r^3 exactly;
- at theta = 0 the tree equals the direct sum."""
import math

import numpy as np
import pytest

import gen


def _vel(n, seed):
    return np.random.default_rng(seed).normal(size=(n, 3)) * 0.3


def test_direct_jerk_is_time_derivative(oracle_lib):
    o = oracle_lib
    c = gen.uniform_cloud(400, seed=61, n_sink=5, h0=0.15)
    v = _vel(c.n, 1)
    tg = np.arange(0, c.n, 7)
    J = o.direct_jerk(c.pos, v, c.mass, c.soft, c.is_sink, targets=tg)
    dt = 1e-6
    ap, _ = o.direct(c.pos + dt * v, c.mass, c.soft, c.is_sink, targets=tg)
    am, _ = o.direct(c.pos - dt * v, c.mass, c.soft, c.is_sink, targets=tg)
    fd = (ap - am) / (2 * dt)
    np.testing.assert_allclose(J, fd, rtol=0, atol=1e-6 * np.abs(J).max())


def test_group_jerk_is_time_derivative_of_monopole_field(oracle_lib):
    c = gen.uniform_cloud(1500, seed=62, n_sink=10, h0=0.08)
    v = _vel(c.n, 2)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    rows = gen.active_subset(c.n, 0.4, seed=3)
    t.walk(rows, 16, 0.6)
    J = t.jerk_group(v, rows)
    dt = 1e-6
    ap, _ = t.eval_frozen(c.pos + dt * v, c.mass, rows, quadrupole=False)
    am, _ = t.eval_frozen(c.pos - dt * v, c.mass, rows, quadrupole=False)
    fd = (ap - am) / (2 * dt)
    np.testing.assert_allclose(J, fd, rtol=0, atol=2e-6 * np.abs(J).max())


def test_galilean_invariance(oracle_lib):
    c = gen.uniform_cloud(1200, seed=63, n_sink=4)
    v = _vel(c.n, 3)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    rows = np.arange(c.n)
    t.walk(rows, 16, 0.7)
    J0 = t.jerk_group(v, rows)
    J1 = t.jerk_group(v + np.array([2.0, -1.0, 0.5]), rows)
    np.testing.assert_allclose(J1, J0, rtol=0, atol=1e-9 * np.abs(J0).max())


def test_circular_two_body(oracle_lib):
    G, m1, m2, r = 1.0, 1.0, 0.3, 2.0
    M = m1 + m2
    om = math.sqrt(G * M / r ** 3)
    x = np.array([[-m2 / M * r, 0, 0], [m1 / M * r, 0, 0]])
    v = np.array([[0, -m2 / M * r * om, 0], [0, m1 / M * r * om, 0]])
    J = oracle_lib.direct_jerk(x, v, np.array([m1, m2]), np.full(2, 1e-3), np.ones(2, np.uint8))
    np.testing.assert_allclose(J[0], G * m2 * (v[1] - v[0]) / r ** 3, rtol=1e-13)
    np.testing.assert_allclose(J[1], G * m1 * (v[0] - v[1]) / r ** 3, rtol=1e-13)
    a, _ = oracle_lib.direct(x, np.array([m1, m2]), np.full(2, 1e-3), np.ones(2, np.uint8))
    assert np.linalg.norm(J[0]) == pytest.approx(om * np.linalg.norm(a[0]), rel=1e-13)


def test_theta_zero_tree_equals_direct(oracle_lib):
    c = gen.uniform_cloud(700, seed=64, n_sink=6)
    v = _vel(c.n, 4)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    rows = np.arange(0, c.n, 3)
    t.walk(rows, 8, 0.0)
    J = t.jerk_group(v, rows)
    Jd = oracle_lib.direct_jerk(c.pos, v, c.mass, c.soft, c.is_sink, targets=rows)
    np.testing.assert_allclose(J, Jd, rtol=1e-11, atol=1e-11 * np.abs(Jd).max())
