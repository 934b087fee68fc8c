"""Shared helpers for the GPU parity tests: run the CUDA path through the C
ABI binding and the oracle on the same seeded cloud."""
import numpy as np

import gen


def to_dev(c, torch):
    dev = torch.device("cuda:0")
    return (torch.from_numpy(c.pos).to(dev), torch.from_numpy(c.mass).to(dev), torch.from_numpy(c.soft).to(dev),
            torch.from_numpy(c.is_sink).to(dev))


def rel_err(a, b):
    """Per-row |a - b| / |b| (vectors) or |a - b| / |b| (scalars)."""
    a = np.asarray(a)
    b = np.asarray(b)
    if a.ndim == 2:
        return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def oracle_tree(c, leaf_size):
    import oracle
    return oracle.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=leaf_size)


def edge_clouds():
    """Degenerate and adversarial inputs."""
    out = {}
    rng = np.random.default_rng(77)
    # single particle, two particles
    out["n1"] = gen.Cloud(np.zeros((1, 3)), np.ones(1), np.full(1, 0.1), np.zeros(1, np.uint8), 0, "n1")
    out["n2"] = gen.Cloud(np.array([[0.0, 0, 0], [1.0, 0.5, -0.25]]), np.array([1.0, 2.0]), np.array([0.3, 0.1]),
                          np.zeros(2, np.uint8), 0, "n2")
    # all particles at one point (one level-21 leaf holding everything)
    n = 300
    out["identical"] = gen.Cloud(np.full((n, 3), 0.37), np.full(n, 1.0 / n), np.full(n, 0.05),
                                 np.zeros(n, np.uint8), 0, "identical")
    # duplicates mixed with a random cloud, one sink on top of a gas cell
    c = gen.uniform_cloud(2000, seed=5, n_sink=1)
    pos = c.pos.copy()
    pos[100:140] = pos[7]
    pos[-1] = pos[3]
    out["duplicates"] = gen.Cloud(pos, c.mass, c.soft, c.is_sink, 5, "duplicates")
    # extents over many decades: a tight clump of 1e-9 size inside a unit cloud
    c = gen.uniform_cloud(3000, seed=6, h0=0.02)
    pos = c.pos.copy()
    pos[:500] = 0.2 + 1e-9 * rng.standard_normal((500, 3))
    soft = c.soft.copy()
    soft[:500] = 1e-10 * (1 + rng.random(500))
    out["decades"] = gen.Cloud(pos, c.mass, soft, c.is_sink, 6, "decades")
    # sinks only
    m = 40
    out["sinks_only"] = gen.Cloud(rng.standard_normal((m, 3)), rng.random(m) + 0.1, np.full(m, 1e-3),
                                  np.ones(m, np.uint8), 0, "sinks_only")
    # massless particles mixed in
    c = gen.uniform_cloud(1500, seed=8)
    mass = c.mass.copy()
    mass[::3] = 0.0
    out["massless"] = gen.Cloud(c.pos, mass, c.soft, c.is_sink, 8, "massless")
    return out
