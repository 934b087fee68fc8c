"""Pins of the oracle's modified Hermite step for sink particles (Sec. 2.3,
the predictor and corrector equations, two field + jerk evaluations per
step) and of its direct two-body timestep:
- the e = 0.9 binary of Sec. 2.3 keeps the relative energy error below the
  paper's 1e-6 per orbit at eta = 0.01, and converges at 4th order or
  better (error ratio >= 16 for 4 eta);
- on a circular orbit one step matches the exact Kepler rotation with a
  local error falling at least as dt^4.5 (the scheme is 4th order, so the
  local error is O(dt^5));
- a lone particle moves on a straight line, exactly;
- a uniform velocity added to every particle (Galilean boost) moves the
  result by that velocity times dt.
"""
import math

import numpy as np

G = 1.0
M2 = np.array([0.6, 0.4])
H = np.full(2, 1e-6)


def _binary(e=0.9, a=1.0):
    M = M2.sum()
    ra = a * (1 + e)
    va = math.sqrt(G * M * (1 - e) / (a * (1 + e)))
    x = np.array([[-M2[1] / M * ra, 0, 0], [M2[0] / M * ra, 0, 0]])
    v = np.array([[0, -M2[1] / M * va, 0], [0, M2[0] / M * va, 0]])
    return x, v, 2 * math.pi * math.sqrt(a ** 3 / (G * M))


def _energy(x, v):
    r = np.linalg.norm(x[1] - x[0])
    return 0.5 * (M2 * (v * v).sum(1)).sum() - G * M2[0] * M2[1] / r


def _error_per_orbit(oracle, eta, orbits=3):
    x, v, period = _binary()
    e0 = _energy(x, v)
    t = 0.0
    while t < orbits * period:
        dt = oracle.two_body_dt(x, v, M2, H, eta, G=G)
        x, v = oracle.hermite_step(x, v, M2, H, dt, G=G)
        t += dt
    return abs(_energy(x, v) - e0) / abs(e0) / orbits


def test_binary_energy_error_and_order(oracle_lib):
    e01 = _error_per_orbit(oracle_lib, 0.01)
    assert e01 < 1e-6
    e04 = _error_per_orbit(oracle_lib, 0.04)
    assert e04 / e01 >= 16.0


def _circular(r=1.0):
    M = M2.sum()
    om = math.sqrt(G * M / r ** 3)
    d = np.array([-M2[1] / M * r, M2[0] / M * r])  # positions along x of the two bodies

    def state(t):
        c, s = math.cos(om * t), math.sin(om * t)
        x = np.array([[d[0] * c, d[0] * s, 0.0], [d[1] * c, d[1] * s, 0.0]])
        v = np.array([[-d[0] * om * s, d[0] * om * c, 0.0], [-d[1] * om * s, d[1] * om * c, 0.0]])
        return x, v

    return state, 2 * math.pi / om


def test_circular_orbit_local_error_order(oracle_lib):
    state, period = _circular()
    x0, v0 = state(0.0)
    errs = []
    for dt in (period / 50, period / 100, period / 200):
        x1, v1 = oracle_lib.hermite_step(x0, v0, M2, H, dt, G=G)
        xe, ve = state(dt)
        errs.append(np.abs(x1 - xe).max() + np.abs(v1 - ve).max() * dt)
    for a, b in zip(errs, errs[1:]):
        assert a / b >= 2 ** 4.5, errs


def test_lone_particle_moves_straight(oracle_lib):
    x = np.array([[0.25, -0.5, 1.0]])
    v = np.array([[0.5, 0.25, -0.125]])
    x1, v1 = oracle_lib.hermite_step(x, v, [1.0], [1e-3], 0.5, G=G)
    np.testing.assert_array_equal(v1, v)
    np.testing.assert_array_equal(x1, x + 0.5 * v)


def test_galilean_boost(oracle_lib):
    rng = np.random.default_rng(7)
    n = 16
    x = rng.standard_normal((n, 3))
    v = rng.standard_normal((n, 3)) * 0.1
    m = rng.random(n) + 0.5
    h = np.full(n, 0.05)
    u = np.array([0.3, -0.2, 0.1])
    dt = 1e-3
    x1, v1 = oracle_lib.hermite_step(x, v, m, h, dt, G=G)
    x2, v2 = oracle_lib.hermite_step(x, v + u, m, h, dt, G=G)
    np.testing.assert_allclose(v2, v1 + u, rtol=0, atol=1e-13)
    np.testing.assert_allclose(x2, x1 + u * dt, rtol=0, atol=1e-13)


def test_two_body_dt_circular(oracle_lib):
    """Circular orbit, negligible softening: t_c = r / v = 1 / omega = t_dyn."""
    r, M = 2.0, 1.0
    om = math.sqrt(G * M / r ** 3)
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0], [0.0, om * r, 0.0]])
    dt = oracle_lib.two_body_dt(x, v, [0.5, 0.5], [1e-9, 1e-9], 0.01, G=G)
    assert abs(dt - math.sqrt(0.01) / (2 * om)) <= 1e-12 * dt
