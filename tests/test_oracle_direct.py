"""Pins of the oracle's FP64 direct sum against closed forms and invariants:
two-body antisymmetry and total momentum (Sec. 2.2.1: all pair interactions
are antisymmetric), the uniform-sphere and Plummer potentials, and Newton's
law for well-separated particles."""
import math

import numpy as np
import pytest

import gen
from gen.clouds import _plummer_radii, _unit_vectors, _rng


def test_two_body_antisymmetry(oracle_lib):
    o = oracle_lib
    pos = np.array([[0.0, 0.0, 0.0], [0.07, -0.02, 0.03]])
    mass = np.array([0.3, 1.7])
    for soft, sink in [([0.1, 0.02], [0, 0]), ([0.1, 0.02], [1, 0]), ([0.01, 0.2], [0, 1]), ([0.05, 0.05], [1, 1])]:
        a, _ = o.direct(pos, mass, np.array(soft), np.array(sink, np.uint8))
        np.testing.assert_allclose(mass[0] * a[0], -mass[1] * a[1], rtol=1e-14, atol=0)


def test_newton_beyond_support(oracle_lib):
    o = oracle_lib
    pos = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    a, phi = o.direct(pos, np.array([1.0, 3.0]), np.array([0.5, 1.0]), G=2.0)
    assert a[0, 0] == pytest.approx(2.0 * 3.0 / 4.0, rel=1e-15)
    assert phi[0] == pytest.approx(-2.0 * 3.0 / 2.0, rel=1e-15)


def test_total_momentum_vanishes(oracle_lib):
    o = oracle_lib
    c = gen.uniform_cloud(1500, seed=7, n_sink=20)
    a, _ = o.direct(c.pos, c.mass, c.soft, c.is_sink)
    tot = (c.mass[:, None] * a).sum(0)
    scale = (c.mass[:, None] * np.abs(a)).sum(0)
    assert np.all(np.abs(tot) <= 1e-13 * scale)


def test_uniform_sphere_potential(oracle_lib):
    """Phi = -G M (3 R^2 - r^2) / (2 R^3), a = -G M r / R^3 inside a uniform sphere.

    A cubic lattice clipped to the unit sphere (quiet start) keeps the
    discreteness noise far below the random-cloud Poisson noise."""
    o = oracle_lib
    s = 0.04
    g = np.arange(-1.0, 1.0 + s / 2, s)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + s / 4
    pos = pos[np.linalg.norm(pos, axis=1) < 1.0]
    n = pos.shape[0]
    mass = np.full(n, 1.0 / n)
    soft = np.full(n, 2.5 * s)
    r = np.linalg.norm(pos, axis=1)
    tg = np.nonzero((r > 0.3) & (r < 0.7))[0][::40]
    a, phi = o.direct(pos, mass, soft, None, tg)
    rr = r[tg]
    phi_exact = -(3 - rr ** 2) / 2
    a_exact = -pos[tg]
    assert np.median(np.abs(phi / phi_exact - 1)) < 3e-3
    err = np.linalg.norm(a - a_exact, axis=1) / np.linalg.norm(a_exact, axis=1)
    assert np.median(err) < 2e-2
    # the random cloud of the 4096-cell workload agrees within its Poisson noise
    c = gen.uniform_cloud(100_000, seed=11, h0=0.02)
    r = np.linalg.norm(c.pos, axis=1)
    tg = np.nonzero((r > 0.3) & (r < 0.7))[0][:200]
    _, phi = o.direct(c.pos, c.mass, c.soft, None, tg)
    assert np.median(np.abs(phi / (-(3 - r[tg] ** 2) / 2) - 1)) < 3e-3


def test_plummer_potential(oracle_lib):
    """Phi = -G M / sqrt(r^2 + b^2) for a Plummer sphere of scale b."""
    o = oracle_lib
    n = 100_000
    rng = _rng(5)
    b = 0.1
    rad = _plummer_radii(rng, n, b, rmax_over_a=1e6)
    pos = _unit_vectors(rng, n) * rad[:, None]
    mass = np.full(n, 1.0 / n)
    soft = np.full(n, 1e-3)
    tg = np.nonzero((rad > 0.5 * b) & (rad < 3 * b))[0][:300]
    _, phi = o.direct(pos, mass, soft, None, tg)
    exact = -1.0 / np.sqrt(rad[tg] ** 2 + b * b)
    assert np.median(np.abs(phi / exact - 1)) < 5e-3
