"""Pins of the oracle oct-tree (Sec. 2.2): frame/keys/order/topology
invariants, moments against flat sums, the opening rule's guarantees, the
theta = 0 limit (always open) equal to the direct sum, error decreasing with
theta, quadrupole order, and translation invariance (Galilean-invariance idea
of Sec. 2.5 reused for positions)."""
import math

import numpy as np
import pytest

import gen

LMAX = 21


def _decode(key):
    key = key.astype(np.uint64)
    q = np.zeros((key.size, 3), np.int64)
    for b in range(LMAX):
        q[:, 0] |= ((key >> np.uint64(3 * b + 2)) & np.uint64(1)).astype(np.int64) << b
        q[:, 1] |= ((key >> np.uint64(3 * b + 1)) & np.uint64(1)).astype(np.int64) << b
        q[:, 2] |= ((key >> np.uint64(3 * b)) & np.uint64(1)).astype(np.int64) << b
    return q


@pytest.fixture(scope="module")
def small(oracle_lib):
    c = gen.uniform_cloud(3000, seed=3, n_sink=12)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    return c, t


def test_frame_and_keys(small):
    c, t = small
    ext = (c.pos.max(0) - c.pos.min(0)).max()
    assert t.L0 >= ext and t.L0 < 2 * ext
    assert math.frexp(t.L0)[0] == 0.5  # power of two
    np.testing.assert_array_equal(t.x0, c.pos.min(0))
    key, order = t.keys()
    assert np.all(np.diff(key.astype(np.float64)) >= 0)
    same = key[1:] == key[:-1]
    assert np.all(order[1:][same] > order[:-1][same])
    assert sorted(order.tolist()) == list(range(c.n))
    q = _decode(key)
    s = (c.pos[order] - t.x0) * (2.0 ** LMAX / t.L0)
    assert np.all(q <= s + 1e-9) and np.all((s < q + 1 + 1e-9) | (q == 2 ** LMAX - 1))


def test_topology_invariants(small):
    c, t = small
    key, order = t.keys()
    nd = t.nodes_int()
    lev, first, count, parent, cf, nch = (nd[:, k] for k in range(6))
    assert lev[0] == 0 and first[0] == 0 and count[0] == c.n and parent[0] == -1
    order_ok = np.lexsort((first, lev))
    np.testing.assert_array_equal(order_ok, np.arange(len(nd)))
    for i in range(len(nd)):
        leaf = nch[i] == 0
        assert leaf == (count[i] <= t.leaf_size or lev[i] == LMAX)
        sh = np.uint64(3 * (LMAX - lev[i]))
        pre = key[first[i]:first[i] + count[i]] >> sh
        assert np.all(pre == pre[0])
        if not leaf:
            ch = np.arange(cf[i], cf[i] + nch[i])
            assert np.all(parent[ch] == i) and np.all(lev[ch] == lev[i] + 1)
            assert first[ch[0]] == first[i]
            np.testing.assert_array_equal(first[ch[1:]], first[ch[:-1]] + count[ch[:-1]])
            assert first[ch[-1]] + count[ch[-1]] == first[i] + count[i]


def test_moments_against_flat_sums(small):
    c, t = small
    key, order = t.keys()
    nd = t.nodes_int()
    mf = t.nodes_f64()
    x = c.pos[order]
    m = c.mass[order]
    h = c.soft[order]
    q = _decode(key)
    for i in range(len(nd)):
        sl = slice(nd[i, 1], nd[i, 1] + nd[i, 2])
        M = m[sl].sum()
        com = (m[sl, None] * x[sl]).sum(0) / M
        s = x[sl] - com
        s2 = (s * s).sum(1)
        Q = np.einsum("k,ka,kb->ab", m[sl], 3 * s, s) - np.eye(3) * (m[sl] * s2).sum()
        assert mf[i, 0] == pytest.approx(M, rel=1e-13)
        np.testing.assert_allclose(mf[i, 1:4], com, rtol=0, atol=1e-13)
        Qo = mf[i, 4:10]
        Qf = np.array([Q[0, 0], Q[1, 1], Q[2, 2], Q[0, 1], Q[0, 2], Q[1, 2]])
        # Q is summed about the cell centre c and moved to the centre of mass
        # (parallel-axis theorem): the shift cancels down from the second
        # moment about c, so rounding is bounded by a few ulps of
        # sum m |x - c|^2 <= M (sqrt(3)/2 L)^2, L the cell side.
        L = t.L0 * 2.0 ** -int(nd[i, 0])
        tol = 1e-11 * (m[sl] * s2).sum() + 1e-14 * M * L * L
        np.testing.assert_allclose(Qo, Qf, rtol=0, atol=max(tol, 1e-300))
        assert abs(Qo[0] + Qo[1] + Qo[2]) <= max(tol, 1e-300)
        assert mf[i, 10] == h[sl].max()
        np.testing.assert_array_equal(nd[i, 9:12], q[sl].min(0))
        np.testing.assert_array_equal(nd[i, 12:15], q[sl].max(0))
        np.testing.assert_array_equal(mf[i, 11:14], x[sl].min(0))
        np.testing.assert_array_equal(mf[i, 14:17], x[sl].max(0))


def group_level(U, G):
    """Largest L with G 8^L <= U (0 below 8 G): the depth at which a uniform
    cloud's nodes hold about G targets."""
    L, v = 0, 8 * G
    while v <= U and L < 21:
        L, v = L + 1, v * 8
    return L


def test_group_level_values():
    assert [group_level(U, 16) for U in (1, 127, 128, 1023, 1024, 209741, 2000102)] == [0, 0, 1, 1, 2, 4, 5]


def test_groups_stay_inside_one_cell_of_the_group_level(oracle_lib):
    """A clumpy cloud with a sparse background: every group's targets lie in
    one node of the group level, or in one leaf above it (a group never packs
    sparse octants of the top levels together)."""
    c = gen.clumpy_cloud(60000, n_clumps=16, n_sink=8, seed=12)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=16)
    act = gen.active_subset(c.n, 0.1, seed=2)
    G = 16
    ng = t.walk(act, G, 0.5)
    g = t.groups()
    tg = t.group_targets()
    nd = t.nodes_int()
    key = t.keys()[0]
    gl = group_level(len(tg), G)
    assert gl >= 2
    cell = key >> np.uint64(3 * (21 - gl))
    # the leaf holding each sorted rank
    leaf_of = np.full(c.n, -1, np.int64)
    for i in np.nonzero(nd[:, 5] == 0)[0]:
        leaf_of[nd[i, 1]:nd[i, 1] + nd[i, 2]] = i
    shallow = 0
    for k in range(ng):
        tf, tc = g[k, 1], g[k, 2]
        r = tg[tf:tf + tc]
        if np.all(cell[r] == cell[r[0]]):
            continue
        assert np.all(leaf_of[r] == leaf_of[r[0]]) and nd[leaf_of[r[0]], 0] < gl
        shallow += 1
    assert shallow < ng


def test_groups_partition_targets(oracle_lib):
    c = gen.uniform_cloud(5000, seed=9, n_sink=8)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=16)
    act = gen.active_subset(c.n, 0.3, seed=1)
    G = 32
    ng = t.walk(act, G, 0.5)
    g = t.groups()
    tg = t.group_targets()
    key, order = t.keys()
    rank = np.empty(c.n, np.int64)
    rank[order] = np.arange(c.n)
    assert sorted(tg.tolist()) == sorted(rank[act].tolist())
    nd = t.nodes_int()
    isact = np.zeros(c.n, bool)
    isact[rank[act]] = True
    assert np.all(np.diff(g[:, 1]) > 0)  # Morton order of first targets
    np.testing.assert_array_equal(np.cumsum(g[:, 2])[:-1], g[1:, 1])
    gl = group_level(len(tg), G)
    for k in range(ng):
        node, tf, tc = g[k, :3]
        assert 1 <= tc <= G
        inside = tg[tf:tf + tc]
        # the run lies inside the node that packed it, and that node holds > G
        # targets unless it is the root or lies above the group level
        assert np.all((inside >= nd[node, 1]) & (inside < nd[node, 1] + nd[node, 2]))
        if node != 0 and nd[node, 0] >= gl:
            assert isact[nd[node, 1]:nd[node, 1] + nd[node, 2]].sum() > G
    # groups are no smaller than the packing rule allows: two consecutive runs
    # packed under the same node never fit together into one group unless a
    # child holding more than G targets separates them
    fill = g[:, 2].mean() / G
    assert fill > 0.5


def test_lists_cover_every_source_once_and_are_conservative(oracle_lib):
    """Accepted nodes and opened leaves partition all particles; every accepted
    node is beyond both softening radii of every member pair and subtends
    L/r <= theta at every target of the group (the paper's rule, Sec. 2.2)."""
    c = gen.uniform_cloud(2500, seed=21, n_sink=10)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=8)
    theta = 0.6
    act = np.arange(c.n)
    t.walk(act, 16, theta)
    g = t.groups()
    tg = t.group_targets()
    nd = t.nodes_int()
    mf = t.nodes_f64()
    key, order = t.keys()
    x = c.pos[order]
    h = c.soft[order]
    for k in range(0, len(g), 7):
        p2m, p2p = t.group_lists(k, g)
        cover = np.zeros(c.n, np.int64)
        for ni in np.concatenate([p2m, p2p]):
            cover[nd[ni, 1]:nd[ni, 1] + nd[ni, 2]] += 1
        assert np.all(cover == 1)
        targets = tg[g[k, 1]:g[k, 1] + g[k, 2]]
        for ni in p2m:
            L = t.L0 * 2.0 ** -nd[ni, 0]
            mem = slice(nd[ni, 1], nd[ni, 1] + nd[ni, 2])
            for i in targets:
                assert L <= theta * np.linalg.norm(mf[ni, 1:4] - x[i]) * (1 + 1e-12)
                d = np.linalg.norm(x[mem] - x[i], axis=1)
                assert np.all(d >= np.maximum(h[i], h[mem]) * (1 - 1e-12))


def test_theta_zero_equals_direct_sum(oracle_lib):
    c = gen.uniform_cloud(1200, seed=4, n_sink=6)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=4)
    act = np.arange(c.n)
    ad, pd = oracle_lib.direct(c.pos, c.mass, c.soft, c.is_sink)
    t.walk(act, 8, 0.0)
    assert t.groups()[:, 4].sum() == 0  # nothing accepted
    a, p = t.accel_group(act)
    np.testing.assert_allclose(a, ad, rtol=1e-12, atol=1e-12 * np.abs(ad).max())
    np.testing.assert_allclose(p, pd, rtol=1e-12)
    a2, p2, _ = t.accel_pp(act, 0.0)
    np.testing.assert_allclose(a2, ad, rtol=1e-12, atol=1e-12 * np.abs(ad).max())


def test_error_decreases_with_theta(oracle_lib):
    c = gen.uniform_cloud(4096, seed=1)
    t = oracle_lib.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=16)
    act = np.arange(c.n)
    ad, _ = oracle_lib.direct(c.pos, c.mass, c.soft, c.is_sink)
    prev = None
    for theta in [1.0, 0.7, 0.5, 0.3]:
        t.walk(act, 32, theta)
        a, _ = t.accel_group(act)
        e = np.median(np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1))
        ap, _, _ = t.accel_pp(act, theta)
        ep = np.median(np.linalg.norm(ap - ad, axis=1) / np.linalg.norm(ad, axis=1))
        if prev is not None:
            assert e < prev[0] and ep < prev[1]
        prev = (e, ep)
    assert prev[0] < 2e-4


def test_quadrupole_order(oracle_lib):
    """Two equal masses at +-b z: the monopole error falls as (b/r)^2, the
    monopole+quadrupole error as (b/r)^4 (exact two-point field)."""
    o = oracle_lib
    b = 0.01
    errs = {True: [], False: []}
    dists = [0.2, 0.4, 0.8]
    for D in dists:
        dirn = np.array([0.3, -0.5, 0.81])
        dirn /= np.linalg.norm(dirn)
        pos = np.array([[0, 0, b], [0, 0, -b], list(D * dirn)])
        mass = np.array([0.5, 0.5, 1e-9])
        soft = np.full(3, 1e-4)
        t = o.Tree(pos, mass, soft, None, leaf_size=2)
        t.walk([2], 1, 0.9)
        ad, _ = o.direct(pos, mass, soft, None, [2])
        for quad in (True, False):
            a, _ = t.accel_group([2], quadrupole=quad)
            errs[quad].append(np.linalg.norm(a - ad) / np.linalg.norm(ad))
        assert t.groups()[0, 4] >= 1  # the pair's node was accepted
    rq = np.array(errs[True])
    rm = np.array(errs[False])
    np.testing.assert_allclose(rm[:-1] / rm[1:], 4.0, rtol=0.05)
    np.testing.assert_allclose(rq[:-1] / rq[1:], 16.0, rtol=0.1)


def test_translation_invariance_dyadic(oracle_lib):
    """Dyadic inputs shifted by a multiple of the cell size: identical keys,
    topology, lists and (bit-identical) fields."""
    n = 4096
    c = gen.uniform_cloud(n, seed=13)
    pos = np.round(c.pos * 2.0 ** 20) / 2.0 ** 20
    mass = np.full(n, 2.0 ** -12)
    t0 = oracle_lib.Tree(pos, mass, c.soft, None, leaf_size=16)
    shift = np.array([3.0, -5.0, 7.0]) * t0.L0 / 2.0 ** 21 * 1024
    t1 = oracle_lib.Tree(pos + shift, mass, c.soft, None, leaf_size=16)
    np.testing.assert_array_equal(t0.keys()[0], t1.keys()[0])
    np.testing.assert_array_equal(t0.nodes_int(), t1.nodes_int())
    act = np.arange(n)
    t0.walk(act, 32, 0.5)
    t1.walk(act, 32, 0.5)
    g0, g1 = t0.groups(), t1.groups()
    np.testing.assert_array_equal(g0, g1)
    for k in range(0, len(g0), 5):
        for l0, l1 in zip(t0.group_lists(k, g0), t1.group_lists(k, g1)):
            np.testing.assert_array_equal(l0, l1)
    # centres of mass are quotients, so the fields agree to rounding only
    a0, p0 = t0.accel_group(act)
    a1, p1 = t1.accel_group(act)
    np.testing.assert_allclose(a0, a1, rtol=1e-12, atol=1e-12 * np.abs(a0).max())
    np.testing.assert_allclose(p0, p1, rtol=1e-12)
