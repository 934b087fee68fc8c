"""Seeded cloud generators (input recipe for every test and benchmark).

Workloads (the paper's GMC initial conditions are not available, so these
synthetic clouds stand in for them; shapes follow Sec. 2.2 and Table 1 of the
STARFORGE methods paper: gas cells of equal mass with adaptive softening equal
to a neighbour-count kernel radius, N_NGB = 32, plus sink particles with a
fixed softening):

* ``uniform_cloud``  - N equal-mass cells uniform in the unit sphere, total
  mass 1, h_i = 0.05 exp(0.3 z_i), z_i ~ N(0, 1)  (the 4096-cell plain case).
* ``clumpy_cloud``   - N cells: 70 % of the mass in Plummer clumps with scale
  radii log-uniform in [1e-3, 3e-2] and clump masses proportional to radius^2,
  30 % uniform in the unit sphere; h = distance to the 32nd nearest neighbour
  (self excluded); plus sinks at copies of randomly chosen cell positions,
  masses LogNormal(ln 1e-4, 1.2), softening 1e-3.
* ``adjoint_cloud``  - the uniform recipe plus sinks uniform in the sphere.
* ``ensemble``       - many uniform clouds of log-uniform size with 0..64 sinks.
* ``paper_scale_cloud`` - the clumpy recipe at 2e7 cells, 2048 clumps, 1024 sinks.

Every generator takes an explicit seed and uses numpy's PCG64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Seed convention: 2010_11254 + workload number.
CONFIG_SEED = {1: 2010_11254 + 1, 2: 2010_11254 + 2, 3: 2010_11254 + 3,
               4: 2010_11254 + 4, 5: 2010_11254 + 5}


@dataclasses.dataclass
class Cloud:
    pos: np.ndarray      # [n, 3] float64
    mass: np.ndarray     # [n] float64
    soft: np.ndarray     # [n] float64, kernel radius of compact support
    is_sink: np.ndarray  # [n] uint8 (1 = sink particle)
    seed: int
    recipe: str

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_sink(self) -> int:
        return int(self.is_sink.sum())


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    nrm = np.sqrt((v * v).sum(axis=1, keepdims=True))
    nrm[nrm == 0] = 1.0
    return v / nrm


def _uniform_sphere(rng: np.random.Generator, n: int, radius: float = 1.0) -> np.ndarray:
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return _unit_vectors(rng, n) * r[:, None]


def _plummer_radii(rng: np.random.Generator, n: int, a: float, rmax_over_a: float = 20.0) -> np.ndarray:
    """Plummer-sphere radii by inverse CDF, r = a (U^(-2/3) - 1)^(-1/2), rejecting r > 20 a."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        u = rng.random(2 * (n - filled) + 8)
        u = u[u > 0]
        r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        r = r[np.isfinite(r) & (r <= rmax_over_a * a)]
        take = min(r.size, n - filled)
        out[filled:filled + take] = r[:take]
        filled += take
    return out


def _largest_remainder(weights: np.ndarray, total: int) -> np.ndarray:
    w = weights / weights.sum() * total
    base = np.floor(w).astype(np.int64)
    rem = total - int(base.sum())
    if rem > 0:
        order = np.argsort(-(w - base), kind="stable")
        base[order[:rem]] += 1
    return base


def knn_softening(pos: np.ndarray, k: int = 32, workers: int = -1) -> np.ndarray:
    """Distance to the k-th nearest neighbour, self excluded (FP64)."""
    from scipy.spatial import cKDTree
    n = pos.shape[0]
    kk = min(k + 1, n)
    tree = cKDTree(pos)
    d, _ = tree.query(pos, k=kk, workers=workers)
    d = np.asarray(d).reshape(n, -1)
    h = d[:, -1].copy()
    # Duplicate positions can give zero distance; keep every radius positive.
    pos_min = h[h > 0].min() if np.any(h > 0) else 1.0
    h[h <= 0] = pos_min
    return h


def _sinks(rng: np.random.Generator, n_sink: int, positions: np.ndarray, soft: float = 1e-3):
    m = rng.lognormal(mean=math.log(1e-4), sigma=1.2, size=n_sink)
    h = np.full(n_sink, soft)
    return positions, m, h


def uniform_cloud(n: int, seed: int = CONFIG_SEED[1], h0: float = 0.05, n_sink: int = 0,
                  sink_soft: float = 1e-3) -> Cloud:
    rng = _rng(seed)
    pos = _uniform_sphere(rng, n)
    z = rng.standard_normal(n)
    soft = h0 * np.exp(0.3 * z)
    mass = np.full(n, 1.0 / n)
    is_sink = np.zeros(n, np.uint8)
    if n_sink:
        spos, sm, sh = _sinks(rng, n_sink, _uniform_sphere(rng, n_sink), sink_soft)
        pos = np.concatenate([pos, spos])
        mass = np.concatenate([mass, sm])
        soft = np.concatenate([soft, sh])
        is_sink = np.concatenate([is_sink, np.ones(n_sink, np.uint8)])
    return Cloud(np.ascontiguousarray(pos), mass, soft, is_sink, seed,
                 f"uniform(n={n}, n_sink={n_sink})")


def clumpy_cloud(n_gas: int, n_clumps: int = 512, n_sink: int = 256, seed: int = CONFIG_SEED[2],
                 clump_frac: float = 0.7, k_ngb: int = 32, workers: int = -1) -> Cloud:
    rng = _rng(seed)
    a = np.exp(rng.uniform(math.log(1e-3), math.log(3e-2), n_clumps))
    n_in_clumps = int(round(clump_frac * n_gas))
    per_clump = _largest_remainder(a * a, n_in_clumps)
    centres = _uniform_sphere(rng, n_clumps)
    parts = []
    for k in range(n_clumps):
        nk = int(per_clump[k])
        if nk == 0:
            continue
        r = _plummer_radii(rng, nk, float(a[k]))
        parts.append(centres[k] + _unit_vectors(rng, nk) * r[:, None])
    parts.append(_uniform_sphere(rng, n_gas - n_in_clumps))
    pos = np.concatenate(parts)
    soft = knn_softening(pos, k_ngb, workers)
    mass = np.full(n_gas, 1.0 / n_gas)
    is_sink = np.zeros(n_gas, np.uint8)
    if n_sink:
        at = rng.integers(0, n_gas, n_sink)
        spos, sm, sh = _sinks(rng, n_sink, pos[at].copy())
        pos = np.concatenate([pos, spos])
        mass = np.concatenate([mass, sm])
        soft = np.concatenate([soft, sh])
        is_sink = np.concatenate([is_sink, np.ones(n_sink, np.uint8)])
    return Cloud(np.ascontiguousarray(pos), mass, soft, is_sink, seed,
                 f"clumpy(n_gas={n_gas}, clumps={n_clumps}, n_sink={n_sink})")


def adjoint_cloud(n_gas: int = 1 << 20, n_sink: int = 128, seed: int = CONFIG_SEED[3]) -> Cloud:
    return uniform_cloud(n_gas, seed=seed, n_sink=n_sink)


def paper_scale_cloud(n_gas: int = 20_000_000, n_sink: int = 1024, seed: int = CONFIG_SEED[5],
                      workers: int = -1) -> Cloud:
    return clumpy_cloud(n_gas, n_clumps=2048, n_sink=n_sink, seed=seed, workers=workers)


def ensemble(n_clouds: int = 256, n_min: int = 1000, n_max: int = 200_000, max_sink: int = 64,
             seed: int = CONFIG_SEED[4]) -> list[Cloud]:
    rng = _rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_clouds)).astype(np.int64)
    sinks = rng.integers(0, max_sink + 1, n_clouds)
    sub = rng.integers(0, 2**62, n_clouds)
    out = []
    for k in range(n_clouds):
        # Mixed softening: the per-cloud base softening follows the cell spacing.
        h0 = 0.05 * (4096.0 / float(sizes[k])) ** (1.0 / 3.0)
        out.append(uniform_cloud(int(sizes[k]), seed=int(sub[k]), h0=h0, n_sink=int(sinks[k])))
    return out


def active_subset(n: int, frac: float, seed: int) -> np.ndarray:
    """Uniform subset without replacement over all particles, sorted (int64)."""
    if frac >= 1.0:
        return np.arange(n, dtype=np.int64)
    rng = _rng(seed)
    k = max(1, int(round(frac * n)))
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def cotangents(n_rows: int, seed: int):
    rng = _rng(seed)
    return (np.ascontiguousarray(rng.standard_normal((n_rows, 3))),
            np.ascontiguousarray(rng.standard_normal(n_rows)))
