"""Pins of the oracle's sink two-body timestep (Sec. 2.3, Delta t_2-body, with
the minima taken in the tree pass and the masses within an accepted node
combined):

- two sinks give the closed form sqrt(eta) / (1/t_c + 1/t_dyn) with
  t_c = sqrt(r^2 + eps^2) / v and t_dyn = sqrt((r^2 + eps^2)^{3/2} / (G M));
- at theta = 0 (every node opened) the tree equals the direct minima;
- a compact, distant cluster accepted as one node enters with its total
  mass at its centre of mass and its mass-weighted velocity;
- the timestep scales as sqrt(eta)."""
import math

import numpy as np
import pytest


def test_two_sinks_closed_form(oracle_lib):
    G, eta, h = 1.0, 0.01, 0.05
    x = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 1.2]])
    v = np.array([[0.1, 0.0, 0.0], [-0.2, 0.5, 0.1]])
    m = np.array([0.7, 0.2])
    dt = oracle_lib.direct_tstep(x, v, m, np.full(2, h), eta, G=G)
    s2 = ((x[1] - x[0]) ** 2).sum() + (h / 2.8) ** 2
    tc = math.sqrt(s2) / np.linalg.norm(v[1] - v[0])
    td = math.sqrt(s2 ** 1.5 / (G * m.sum()))
    expect = math.sqrt(eta) / (1 / tc + 1 / td)
    np.testing.assert_allclose(dt, expect, rtol=1e-14)


def _sinks(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n, 3)), rng.normal(size=(n, 3)) * 0.2, rng.lognormal(np.log(1e-3), 1.0, n),
            np.full(n, 1e-3), np.ones(n, np.uint8))


def test_theta_zero_equals_direct(oracle_lib):
    x, v, m, h, sk = _sinks(300, 1)
    t = oracle_lib.Tree(x, m, h, sk, leaf_size=4)
    rows = np.arange(300)
    t.walk(rows, 8, 0.0)
    np.testing.assert_allclose(t.tstep_group(v, 0.01, rows), oracle_lib.direct_tstep(x, v, m, h, 0.01, rows),
                               rtol=1e-13)


def test_distant_cluster_combines_as_one_node(oracle_lib):
    """One sink far from a compact cluster: with the cluster accepted as one
    node, the sink's limits use the cluster's total mass, centre of mass and
    mass-weighted velocity."""
    rng = np.random.default_rng(4)
    k = 40
    xc = rng.normal(size=(k, 3)) * 1e-3 + np.array([10.0, 0.0, 0.0])
    vc = rng.normal(size=(k, 3)) * 0.1 + np.array([0.0, 1.0, 0.0])
    mc = rng.random(k) + 0.5
    x = np.vstack([[0.0, 0.0, 0.0], xc])
    v = np.vstack([[0.0, 0.0, 0.0], vc])
    m = np.r_[0.3, mc]
    h = np.full(k + 1, 1e-4)
    t = oracle_lib.Tree(x, m, h, np.ones(k + 1, np.uint8), leaf_size=4)
    t.walk(np.array([0]), 1, 0.5)
    p2m, p2p = t.group_lists(0)
    assert len(p2m) >= 1
    dt = t.tstep_group(v, 0.01, np.array([0]))[0]
    M = mc.sum()
    com = (mc[:, None] * xc).sum(0) / M
    vcom = (mc[:, None] * vc).sum(0) / M
    s2 = (com ** 2).sum() + (1e-4 / 2.8) ** 2
    whole = math.sqrt(0.01) / (np.linalg.norm(vcom) / math.sqrt(s2) + math.sqrt((0.3 + M) / s2 ** 1.5))
    nodes = t.nodes_int()
    # the whole cluster is one accepted node; the only P2P particle is the target itself
    assert len(p2m) == 1 and nodes[p2m[0], 2] == k
    assert sum(int(nodes[j, 2]) for j in p2p) == 1
    assert dt == pytest.approx(whole, rel=1e-12)
    # smaller than the direct, member-by-member minima
    direct = oracle_lib.direct_tstep(x, v, m, h, 0.01, np.array([0]))[0]
    assert dt < direct


def test_sqrt_eta_scaling(oracle_lib):
    x, v, m, h, sk = _sinks(100, 2)
    t = oracle_lib.Tree(x, m, h, sk, leaf_size=4)
    rows = np.arange(100)
    t.walk(rows, 8, 0.5)
    a = t.tstep_group(v, 0.01, rows)
    b = t.tstep_group(v, 0.04, rows)
    np.testing.assert_allclose(b, 2 * a, rtol=1e-14)
