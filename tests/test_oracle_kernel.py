"""Pins of the oracle's softened pair law (Sec. 2.2.1, Sec. 2.3.1) against
closed forms: the textbook M4 density via Poisson's equation, the Plummer
equivalent softening, Newtonian gravity beyond the support, continuity, and
the pair rules (averaged gas-gas kernels, max softening with a sink)."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kernel_special_values.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, u, v = line.split()
        out[name] = (float(u), float(v))
    return out


def test_golden_special_values(oracle_lib):
    o = oracle_lib
    g = _golden()
    # Plummer-equivalent softening epsilon = h/2.8 (Sec. 2.3.1): phi(0) = -2.8 G m / h.
    assert o.kernel_W(g["W_at_zero"][0]) == pytest.approx(g["W_at_zero"][1], abs=1e-15)
    assert o.kernel_W(g["W_at_one"][0]) == pytest.approx(g["W_at_one"][1], abs=1e-15)
    assert o.kernel_g(g["g_at_one"][0]) == pytest.approx(g["g_at_one"][1], abs=1e-15)
    # Poisson: (1/(4 pi u^2)) d(u^3 g)/du at u -> 0 equals the M4 central density 8/pi.
    u = 1e-4
    fd = ((u + 1e-7) ** 3 * o.kernel_g(u + 1e-7) - (u - 1e-7) ** 3 * o.kernel_g(u - 1e-7)) / 2e-7
    assert fd / (4 * math.pi * u * u) == pytest.approx(g["density_norm_u0"][1], rel=1e-6)


@pytest.mark.parametrize("u0", [0.5, 1.0])
def test_continuity_at_branch_points(oracle_lib, u0):
    o = oracle_lib
    e = 1e-12
    assert o.kernel_W(u0 - e) == pytest.approx(o.kernel_W(u0 + e), abs=1e-10)
    assert o.kernel_g(u0 - e) == pytest.approx(o.kernel_g(u0 + e), abs=1e-9)
    assert o.kernel_dg_over_u(u0 - e) == pytest.approx(o.kernel_dg_over_u(u0 + e), abs=1e-8)


def test_poisson_reproduces_m4_density(oracle_lib):
    """-laplacian(phi)/(4 pi G) of the softened point mass is the normalised M4 spline."""
    o = oracle_lib
    h = 1.0

    def m4(u):
        if u < 0.5:
            return 8 / math.pi * (1 - 6 * u * u + 6 * u ** 3)
        if u < 1.0:
            return 8 / math.pi * 2 * (1 - u) ** 3
        return 0.0

    for u in np.linspace(0.02, 1.4, 71):
        if abs(u - 0.5) < 1e-3 or abs(u - 1.0) < 1e-3:
            continue
        s = 1e-6
        f = lambda x: x ** 3 * o.kernel_g(x)
        lap = (f(u + s) - f(u - s)) / (2 * s) / (u * u * h ** 3)
        assert lap / (4 * math.pi) == pytest.approx(m4(u), abs=2e-7), u
    # total mass 1 inside the support
    uu = np.linspace(0, 1, 20001)
    rho = np.array([m4(x) for x in uu])
    mass = np.trapezoid(4 * math.pi * uu * uu * rho, uu)
    assert mass == pytest.approx(1.0, abs=1e-6)


def test_force_is_minus_gradient_of_potential(oracle_lib):
    """a = -grad phi: W'(u) = u g(u) (finite differences), and g'(u)/u."""
    o = oracle_lib
    for u in np.linspace(0.01, 1.5, 60):
        s = 1e-6
        dW = (o.kernel_W(u + s) - o.kernel_W(u - s)) / (2 * s)
        assert dW == pytest.approx(u * o.kernel_g(u), rel=1e-7, abs=1e-8)
        dg = (o.kernel_g(u + s) - o.kernel_g(u - s)) / (2 * s)
        assert dg / u == pytest.approx(o.kernel_dg_over_u(u), rel=1e-6, abs=1e-6)


def test_newtonian_beyond_support(oracle_lib):
    o = oracle_lib
    for r, h in [(1.0, 0.5), (2.0, 2.0), (3.7, 0.1)]:
        K, P, Kr = o.pair(r, h, h)
        assert K == 1.0 / r ** 3
        assert P == -1.0 / r
        assert Kr == pytest.approx(-3.0 / r ** 5, rel=1e-15)


def test_pair_rules(oracle_lib):
    """Gas-gas: mean of the two kernels; any sink: one kernel of max(h_i, h_j)."""
    o = oracle_lib
    # r = 0.3 with h_i = 1 (u = 0.3, softened) and h_j = 0.2 (Newtonian)
    K, P, _ = o.pair(0.3, 1.0, 0.2)
    u = 0.3
    K_soft = 32 / 3 - 192 / 5 * u * u + 32 * u ** 3
    W_soft = 16 / 3 * u * u - 48 / 5 * u ** 4 + 32 / 5 * u ** 5 - 14 / 5
    assert K == pytest.approx(0.5 * (K_soft + 1 / 0.3 ** 3), rel=1e-14)
    assert P == pytest.approx(0.5 * (W_soft - 1 / 0.3), rel=1e-14)
    # with a sink on either side: single kernel of support max(h) = 1
    for si, sj in [(1, 0), (0, 1), (1, 1)]:
        K2, P2, _ = o.pair(0.3, 1.0, 0.2, si, sj)
        assert K2 == pytest.approx(K_soft, rel=1e-14)
        assert P2 == pytest.approx(W_soft, rel=1e-14)
    # zero separation inside the support: finite potential, Phi(0) = -2.8/h
    K0, P0, _ = o.pair(0.0, 0.5, 0.5)
    assert P0 == pytest.approx(-2.8 / 0.5, rel=1e-15)
    assert math.isfinite(K0)
