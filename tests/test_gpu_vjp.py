"""GPU adjoint (VJP with frozen lists) against the oracle's analytic FP64 VJP
and against FP64 central finite differences of the oracle's frozen-list field
(Sec. 2.2: the tidal tensor of the same softened kernel).  Tolerance: 1e-4
relative to the largest gradient component, and 1e-4 median per-row."""
import numpy as np
import pytest

import gen
from _helpers import edge_clouds, oracle_tree, to_dev

pytestmark = pytest.mark.gpu

VJP_TOL = 1e-4


def _gpu_vjp(c, rows, ca, cp, theta, leaf_size=16, group_size=32, quad=True, G=1.0, list_depth=0):
    import torch
    import paper_2010_11254_gb300 as sfg
    pos, mass, soft, sink = to_dev(c, torch)
    t = sfg.Tree(pos, mass, soft, sink, theta=theta, leaf_size=leaf_size, group_size=group_size, quadrupole=quad,
                 G=G, list_depth=list_depth)
    r = torch.from_numpy(np.asarray(rows, np.int64)).cuda()
    d_pos, d_mass = t.accel_vjp(r, torch.from_numpy(ca).cuda(), None if cp is None else torch.from_numpy(cp).cuda())
    assert t.status() == sfg.SFG_OK
    t.close()
    return d_pos.cpu().numpy(), d_mass.cpu().numpy()


def _close(g, o, tol=VJP_TOL):
    scale = np.abs(o).max()
    assert np.abs(g - o).max() <= tol * scale, np.abs(g - o).max() / scale
    if o.ndim == 2:
        rows = np.linalg.norm(o, axis=1)
        big = rows > 1e-3 * rows.max()
        e = np.linalg.norm(g - o, axis=1)[big] / rows[big]
    else:
        big = np.abs(o) > 1e-3 * np.abs(o).max()
        e = np.abs(g - o)[big] / np.abs(o)[big]
    assert np.median(e) <= tol, np.median(e)


@pytest.mark.parametrize("quad", [True, False])
def test_vjp_matches_oracle(quad):
    c = gen.uniform_cloud(20000, seed=31, n_sink=16)
    rows = gen.active_subset(c.n, 0.5, seed=2)
    ca, cp = gen.cotangents(rows.size, seed=3)
    g_pos, g_mass = _gpu_vjp(c, rows, ca, cp, 0.6, quad=quad)
    o = oracle_tree(c, 16)
    o.walk(rows, 32, 0.6)
    o_pos, o_mass = o.vjp(rows, ca, cp, quadrupole=quad)
    _close(g_pos, o_pos)
    _close(g_mass, o_mass)


@pytest.mark.parametrize("list_depth", [1, 2, 4])
def test_vjp_list_depths(list_depth):
    c = gen.clumpy_cloud(1 << 14, n_clumps=16, n_sink=12, seed=26)
    rows = gen.active_subset(c.n, 0.3, seed=27)
    ca, cp = gen.cotangents(rows.size, seed=28)
    g_pos, g_mass = _gpu_vjp(c, rows, ca, cp, 0.5, group_size=13, list_depth=list_depth)
    o = oracle_tree(c, 16)
    o.walk(rows, 13, 0.5)
    o_pos, o_mass = o.vjp(rows, ca, cp)
    _close(g_pos, o_pos)
    _close(g_mass, o_mass)


def test_vjp_clumpy_sparse_and_sizes():
    c = gen.clumpy_cloud(1 << 15, n_clumps=64, n_sink=32, seed=5)
    rows = gen.active_subset(c.n, 0.1, seed=6)
    ca, cp = gen.cotangents(rows.size, seed=7)
    for leaf, grp in [(16, 32), (4, 8)]:
        g_pos, g_mass = _gpu_vjp(c, rows, ca, cp, 0.5, leaf_size=leaf, group_size=grp)
        o = oracle_tree(c, leaf)
        o.walk(rows, grp, 0.5)
        o_pos, o_mass = o.vjp(rows, ca, cp)
        _close(g_pos, o_pos)
        _close(g_mass, o_mass)


def test_vjp_against_central_differences():
    """FP64 central differences (step 1e-6) of the frozen-list oracle field on
    64 sampled particles (the config-3 check, at a size the oracle finishes in
    seconds)."""
    c = gen.uniform_cloud(8000, seed=41, n_sink=8)
    rows = np.arange(c.n)
    ca, cp = gen.cotangents(c.n, seed=4)
    g_pos, g_mass = _gpu_vjp(c, rows, ca, cp, 0.5)
    o = oracle_tree(c, 16)
    o.walk(rows, 32, 0.5)
    rng = np.random.default_rng(3)
    pick = rng.choice(c.n, 64, replace=False)
    h = 1e-6
    scale = np.abs(g_pos).max()

    def loss(p, m):
        a, ph = o.eval_frozen(p, m, rows)
        return float((a * ca).sum() + (ph * cp).sum())

    for k in pick:
        ax = int(rng.integers(0, 3))
        pp = c.pos.copy()
        pp[k, ax] += h
        lp = loss(pp, c.mass)
        pp[k, ax] -= 2 * h
        lm = loss(pp, c.mass)
        assert abs((lp - lm) / (2 * h) - g_pos[k, ax]) <= VJP_TOL * scale
    mscale = np.abs(g_mass).max()
    for k in pick[:16]:
        mm = c.mass.copy()
        hm = 1e-6 * c.mass[k]
        mm[k] += hm
        lp = loss(c.pos, mm)
        mm[k] -= 2 * hm
        lm = loss(c.pos, mm)
        assert abs((lp - lm) / (2 * hm) - g_mass[k]) <= VJP_TOL * mscale


def test_vjp_duplicate_rows_and_no_phi_cotangent():
    c = gen.uniform_cloud(3000, seed=8)
    rows = np.array([5, 17, 5, 300, 17, 17])
    ca, cp = gen.cotangents(rows.size, seed=1)
    d1, m1 = _gpu_vjp(c, rows, ca, None, 0.5)
    u = np.array([5, 17, 300])
    ca2 = np.stack([ca[0] + ca[2], ca[1] + ca[4] + ca[5], ca[3]])
    d2, m2 = _gpu_vjp(c, u, ca2, None, 0.5)
    np.testing.assert_allclose(d1, d2, rtol=1e-6, atol=1e-6 * np.abs(d2).max())
    np.testing.assert_allclose(m1, m2, rtol=1e-6, atol=1e-6 * np.abs(m2).max())
    o = oracle_tree(c, 16)
    o.walk(rows, 32, 0.5)
    o_pos, o_mass = o.vjp(rows, ca, np.zeros(rows.size))
    _close(d1, o_pos)


def test_vjp_massless_particles():
    c = edge_clouds()["massless"]
    rows = np.arange(c.n)
    ca, cp = gen.cotangents(c.n, seed=9)
    g_pos, g_mass = _gpu_vjp(c, rows, ca, cp, 0.5, leaf_size=8)
    o = oracle_tree(c, 8)
    o.walk(rows, 32, 0.5)
    o_pos, o_mass = o.vjp(rows, ca, cp)
    _close(g_pos, o_pos)
    _close(g_mass, o_mass)


def test_autograd_function_matches_direct_calls():
    import torch
    import paper_2010_11254_gb300 as sfg
    c = gen.uniform_cloud(4000, seed=10, n_sink=4)
    pos, mass, soft, sink = to_dev(c, torch)
    pos.requires_grad_(True)
    mass.requires_grad_(True)
    act = torch.arange(0, c.n, 2, device="cuda")
    acc, phi = sfg.gravity(pos, mass, soft, sink, act, theta=0.6)
    ca, cp = gen.cotangents(act.numel(), seed=2)
    ca_t, cp_t = torch.from_numpy(ca).cuda(), torch.from_numpy(cp).cuda()
    loss = (acc * ca_t).sum() + (phi * cp_t).sum()
    gp, gm = torch.autograd.grad(loss, (pos, mass))
    d_pos, d_mass = _gpu_vjp(c, act.cpu().numpy(), ca, cp, 0.6)
    np.testing.assert_allclose(gp.cpu().numpy(), d_pos, rtol=0, atol=1e-6 * np.abs(d_pos).max())
    np.testing.assert_allclose(gm.cpu().numpy(), d_mass, rtol=0, atol=1e-6 * np.abs(d_mass).max())


def test_vjp_adjoint_workload_full_size():
    """The adjoint workload at its stated size: the uniform recipe with 2^20
    cells and 128 sinks, every particle active, N(0,1) cotangents, theta 0.5.
    (1) The GPU VJP of all rows against the oracle's analytic FP64 VJP;
    (2) the GPU VJP of 4096 sampled rows against FP64 central differences
    (step 1e-6) of the oracle's frozen-list field of the same rows, at 64
    sampled particle coordinates and 16 masses."""
    c = gen.adjoint_cloud(1 << 20, n_sink=128, seed=gen.CONFIG_SEED[3])
    rows = np.arange(c.n)
    ca, cp = gen.cotangents(c.n, seed=gen.CONFIG_SEED[3] + 7)
    g_pos, g_mass = _gpu_vjp(c, rows, ca, cp, 0.5)
    o = oracle_tree(c, 16)
    o.walk(rows, 32, 0.5)
    o_pos, o_mass = o.vjp(rows, ca, cp)
    _close(g_pos, o_pos)
    _close(g_mass, o_mass)
    # finite differences on a row sample (the frozen-list loss of 4096 rows)
    rng = np.random.default_rng(11)
    sub = np.sort(rng.choice(c.n, 4096, replace=False))
    s_pos, s_mass = _gpu_vjp(c, sub, ca[sub], cp[sub], 0.5)
    o.walk(sub, 32, 0.5)
    h = 1e-6
    scale = np.abs(s_pos).max()

    def loss(p, m):
        a, ph = o.eval_frozen(p, m, sub)
        return float((a * ca[sub]).sum() + (ph * cp[sub]).sum())

    # half the probes on the sampled rows themselves, half anywhere
    pick = np.concatenate([rng.choice(sub, 32, replace=False), rng.choice(c.n, 32, replace=False)])
    for k in pick:
        ax = int(rng.integers(0, 3))
        pp = c.pos.copy()
        pp[k, ax] += h
        lp = loss(pp, c.mass)
        pp[k, ax] -= 2 * h
        lm = loss(pp, c.mass)
        assert abs((lp - lm) / (2 * h) - s_pos[k, ax]) <= VJP_TOL * scale
    mscale = np.abs(s_mass).max()
    for k in pick[::4]:
        mm = c.mass.copy()
        hm = 1e-6 * c.mass[k]
        mm[k] += hm
        lp = loss(c.pos, mm)
        mm[k] -= 2 * hm
        lm = loss(c.pos, mm)
        assert abs((lp - lm) / (2 * hm) - s_mass[k]) <= VJP_TOL * mscale
