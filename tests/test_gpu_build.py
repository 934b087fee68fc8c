"""GPU build (frame, keys, sort, octree, FP64 moments) against the oracle:
bit-exact keys, order, topology, integer boxes, centre-of-mass cells and FP64
moments (same integer-quantised geometry, same fixed operation order)."""
import numpy as np
import pytest

import gen
from _helpers import edge_clouds, oracle_tree, to_dev

pytestmark = pytest.mark.gpu


def _compare_build(c, leaf_size):
    import torch
    import paper_2010_11254_gb300 as sfg
    pos, mass, soft, sink = to_dev(c, torch)
    t = sfg.Tree(pos, mass, soft, sink, leaf_size=leaf_size)
    o = oracle_tree(c, leaf_size)
    st = t.stats()
    assert st["n_nodes"] == o.n_nodes
    assert st["L0"] == o.L0
    np.testing.assert_array_equal(np.array(st["x0"]), o.x0)
    key, order = o.keys()
    np.testing.assert_array_equal(t.export(sfg.FIELD_KEYS), key)
    np.testing.assert_array_equal(t.export(sfg.FIELD_ORDER).astype(np.int64), order)
    gi = t.export(sfg.FIELD_NODE_INT).astype(np.int64)
    oi = o.nodes_int()
    np.testing.assert_array_equal(gi[:, :6], oi[:, :6])          # level first count parent child_first nchild
    np.testing.assert_array_equal(gi[:, 6:15], oi[:, 9:18])      # lo, hi, cq
    np.testing.assert_array_equal(t.export(sfg.FIELD_NODE_HQ).astype(np.int64), oi[:, 18])
    gf = t.export(sfg.FIELD_NODE_F64)
    of = o.nodes_f64()
    np.testing.assert_array_equal(gf, of[:, :11])                # M com Q hmax, bit for bit
    _check_f32_records(t, c, order, gi, gf)
    assert t.status() == sfg.SFG_OK
    t.close()


def _cell_centres(level, lo, x0, L0):
    """Centres of the cells (level, lower corner in grid units): the exact
    corner-plus-half-side in grid units times the half-cell size, plus x0."""
    sh = 21 - level
    corner = (lo >> sh[:, None]) << sh[:, None]
    return x0[None, :] + (2 * corner + (np.int64(1) << sh)[:, None]).astype(np.float64) * np.ldexp(L0, -22)


def _check_f32_records(t, c, order, gi, gf):
    """The evaluation's FP32 records are the round-to-nearest-even FP32 values
    of the FP64 quantities (numpy's float64 -> float32 cast), bit for bit:
    particle offsets from their leaf's cell centre and masses; node centre-
    of-mass offsets from the cell centre, masses and quadrupoles."""
    import paper_2010_11254_gb300 as sfg
    st = t.stats()
    x0, L0 = np.array(st["x0"]), st["L0"]
    cen = _cell_centres(gi[:, 0], gi[:, 6:9], x0, L0)
    ef = t.export(sfg.FIELD_NODE_F32)
    want = np.concatenate([gf[:, 1:4] - cen, gf[:, 0:1], gf[:, [4, 5, 7, 8, 9]]], 1).astype(np.float32)
    np.testing.assert_array_equal(ef.view(np.uint32), want.view(np.uint32))
    leaf = np.flatnonzero(gi[:, 5] == 0)
    first, count = gi[leaf, 1], gi[leaf, 2]
    owner = np.repeat(np.arange(leaf.size), count)
    rank = np.concatenate([np.arange(f, f + k) for f, k in zip(first, count)]) if leaf.size else np.zeros(0, int)
    pw = t.export(sfg.FIELD_PARTICLE_F32)
    assert np.array_equal(np.sort(rank), np.arange(c.n))
    d = c.pos[order[rank]] - cen[leaf[owner]]
    np.testing.assert_array_equal(pw[rank, :3].view(np.uint32), d.astype(np.float32).view(np.uint32))
    np.testing.assert_array_equal(pw[rank, 3].view(np.uint32), c.mass[order[rank]].astype(np.float32).view(np.uint32))


@pytest.mark.parametrize("leaf_size", [1, 8, 16, 64])
def test_build_uniform_4096(leaf_size):
    _compare_build(gen.uniform_cloud(4096), leaf_size)


def test_build_clumpy_with_sinks():
    _compare_build(gen.clumpy_cloud(1 << 15, n_clumps=64, n_sink=32, seed=12), 16)


def test_build_sizes_spanning_tiles():
    # sizes around the radix-sort and scan tiles (2048) and the leaf chunks, with a ragged tail
    for n in [2047, 2049, 4095, 4097, 12289, 70001]:
        _compare_build(gen.uniform_cloud(n, seed=n, n_sink=n % 7), 16)


@pytest.mark.parametrize("leaf_size", [16, 100])
def test_build_large_staged_leaves(leaf_size):
    """From 2^22 particles on, the leaf moments read chunks of sorted ranks
    staged in shared memory; a leaf that starts near a chunk's end and runs
    past the staged margin (leaf size 100 > the 64-rank margin) reads the
    rest from global memory.  Same bit-exact moments and records."""
    n = (1 << 22) + 4099
    _compare_build(gen.uniform_cloud(n, seed=leaf_size, n_sink=9), leaf_size)


def test_build_node_capacity_retry():
    """Close pairs (a few cells apart) make chains of one-child nodes: at leaf
    size 1 the tree needs several times the first node-capacity estimate, so
    the octree is rebuilt with a doubled capacity until it fits."""
    rng = np.random.default_rng(77)
    m = 3000
    a = rng.uniform(-1.0, 1.0, (m, 3))
    d = rng.standard_normal((m, 3))
    b = a + 3e-6 * d / np.linalg.norm(d, axis=1, keepdims=True)
    pos = np.ascontiguousarray(np.concatenate([a, b]))
    c = gen.Cloud(pos, np.full(2 * m, 1.0 / (2 * m)), np.full(2 * m, 1e-3), np.zeros(2 * m, np.uint8), 77, "pairs")
    assert oracle_tree(c, 1).n_nodes > 2 * (6 * (c.n // 3) + 4096 + 64)
    _compare_build(c, 1)


@pytest.mark.parametrize("name", ["n1", "n2", "identical", "duplicates", "decades", "sinks_only", "massless"])
def test_build_edge_cases(name):
    _compare_build(edge_clouds()[name], 8)


def test_build_rejects_bad_inputs():
    import torch
    import paper_2010_11254_gb300 as sfg
    c = gen.uniform_cloud(100, seed=1)
    pos, mass, soft, sink = to_dev(c, torch)
    for bad in ["nan_pos", "neg_mass", "zero_soft", "inf_soft"]:
        p, m, s = pos.clone(), mass.clone(), soft.clone()
        if bad == "nan_pos":
            p[5, 1] = float("nan")
        elif bad == "neg_mass":
            m[3] = -1.0
        elif bad == "zero_soft":
            s[9] = 0.0
        else:
            s[0] = float("inf")
        with pytest.raises(sfg.SfgError) as e:
            sfg.Tree(p, m, s, sink)
        assert e.value.code == sfg.SFG_EINVAL
