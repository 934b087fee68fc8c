"""Pins of the oracle's tidal tensor T = -grad grad Phi (Sec. 2.2: summed in
the same tree pass and with the same opening criterion as g; Sec. 2.2.1: the
same softened kernel and symmetrisation) and of the tidal timestep of Sec. 2.3.

- T is the derivative of the frozen-list field with respect to the target's
  own position (FP64 central differences);
- the trace of one softened pair is -4 pi G times the M4 kernel density
  (Poisson's equation), and it vanishes beyond the support (vacuum);
- at theta = 0 (every node opened) the tree equals the direct sum;
- a point mass gives |T|^2 / 6 = (G M / r^3)^2, so the timestep is
  sqrt(eta) times the dynamical time sqrt(r^3 / G M) (the Sec. 2.3 remark);
- inside a uniform sphere T = -(4 pi / 3) G rho I = -(G M / R^3) I, less the
  target's own excluded kernel."""
import math

import numpy as np
import pytest

import gen

_IA = [0, 1, 2, 0, 0, 1]
_IB = [0, 1, 2, 1, 2, 2]


def _full(T6):
    T = np.zeros((3, 3))
    for c in range(6):
        T[_IA[c], _IB[c]] = T[_IB[c], _IA[c]] = T6[c]
    return T


@pytest.mark.parametrize("quad", [True, False])
def test_tidal_is_derivative_of_frozen_field(oracle_lib, quad):
    c = gen.uniform_cloud(1500, seed=51, n_sink=16, h0=0.08)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    rows = gen.active_subset(c.n, 0.5, seed=5)
    t.walk(rows, 16, 0.6)
    pick = rows[np.random.default_rng(1).choice(rows.size, 20, replace=False)]
    T = t.tidal_group(pick, quadrupole=quad)
    h = 1e-6
    for k, i in enumerate(pick):
        fd = np.zeros((3, 3))
        for b in range(3):
            pp = c.pos.copy()
            pp[i, b] += h
            ap, _ = t.eval_frozen(pp, c.mass, [i], quadrupole=quad)
            pp[i, b] -= 2 * h
            am, _ = t.eval_frozen(pp, c.mass, [i], quadrupole=quad)
            fd[:, b] = (ap[0] - am[0]) / (2 * h)
        Tf = _full(T[k])
        scale = np.abs(Tf).max()
        np.testing.assert_allclose(Tf, fd, rtol=0, atol=2e-6 * scale)


def _m4_density(u):
    if u < 0.5:
        return 8 / math.pi * (1 - 6 * u * u + 6 * u ** 3)
    if u < 1.0:
        return 8 / math.pi * 2 * (1 - u) ** 3
    return 0.0


@pytest.mark.parametrize("sink", [0, 1])
def test_pair_trace_is_kernel_density(oracle_lib, sink):
    """tr T = -laplacian Phi = -4 pi G rho for one softened source (unit mass)."""
    o = oracle_lib
    hi, hj = 0.7, 0.4
    rng = np.random.default_rng(3)
    for r in np.linspace(0.03, 1.1, 40):
        d = rng.normal(size=3)
        d *= r / np.linalg.norm(d)
        pos = np.array([[0.0, 0.0, 0.0], d])
        T = o.direct_tidal(pos, np.array([1.0, 1.0]), np.array([hi, hj]), np.array([sink, 0]), targets=[0])[0]
        tr = T[0] + T[1] + T[2]
        if sink:
            h = max(hi, hj)
            rho = _m4_density(r / h) / h ** 3
        else:
            rho = 0.5 * (_m4_density(r / hi) / hi ** 3 + _m4_density(r / hj) / hj ** 3)
        assert tr == pytest.approx(-4 * math.pi * rho, abs=1e-10 * max(1.0, 1 / r ** 3))


def test_theta_zero_tree_equals_direct(oracle_lib):
    c = gen.uniform_cloud(700, seed=53, n_sink=6)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    rows = np.arange(0, c.n, 3)
    t.walk(rows, 8, 0.0)
    T = t.tidal_group(rows)
    Td = oracle_lib.direct_tidal(c.pos, c.mass, c.soft, c.is_sink, targets=rows)
    np.testing.assert_allclose(T, Td, rtol=1e-11, atol=1e-11 * np.abs(Td).max())


def test_point_mass_timestep_is_dynamical_time(oracle_lib):
    o = oracle_lib
    M, eta = 3.0, 0.01
    for r in (0.5, 1.0, 4.0):
        pos = np.array([[0.0, 0.0, 0.0], [r / math.sqrt(3)] * 3])
        T = o.direct_tidal(pos, np.array([1.0, M]), np.array([1e-3, 1e-3]), targets=[0])
        f2 = (_full(T[0]) ** 2).sum()
        assert f2 / 6 == pytest.approx((M / r ** 3) ** 2, rel=1e-12)
        # eigenvalues (2, -1, -1) G M / r^3: a radial stretch, transverse squeeze
        ev = np.sort(np.linalg.eigvalsh(_full(T[0])))
        np.testing.assert_allclose(ev, np.array([-1, -1, 2]) * M / r ** 3, rtol=1e-12)
        dt = o.tidal_dt(T, eta)[0]
        assert dt == pytest.approx(math.sqrt(eta) * math.sqrt(r ** 3 / M), rel=1e-12)
    assert np.isinf(o.tidal_dt(np.zeros((1, 6)), eta)[0])


def test_uniform_sphere_interior(oracle_lib):
    """T = -(4 pi / 3) G rho I inside a uniform sphere.  A cubic lattice (no
    Poisson noise) of spacing a fills the unit sphere; with a softening of 4a
    the kernel sum over the lattice reproduces rho, except that the target's
    own kernel (self term excluded) is missing: by cubic symmetry every
    diagonal element is -(4 pi / 3) G (rho - m W(0)), W(0) = 8 / (pi h^3)."""
    a = 0.06
    g = np.arange(-1.0 + a / 2, 1.0, a)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pos = pos[np.linalg.norm(pos, axis=1) < 1.0]
    n = pos.shape[0]
    m = 1.0 / n
    soft = np.full(n, 4 * a)
    inner = np.flatnonzero(np.linalg.norm(pos, axis=1) < 0.4)
    T = oracle_lib.direct_tidal(pos, np.full(n, m), soft, targets=inner)
    expect = -4 * math.pi / 3 * (m / a ** 3 - 8 * m / (math.pi * (4 * a) ** 3))
    np.testing.assert_allclose(T[:, :3], expect, rtol=0.003)
    np.testing.assert_allclose(T[:, 3:], 0.0, atol=0.003 * abs(expect))
