"""Autotuner for the launch-shape parameters of a workload.

The tree's leaf size (N_leaf) and group size (targets sharing one walk) trade
walk length against list length; the best pair depends on the particle
distribution, the active fraction and the GPU.  ``tune`` builds the tree with
each candidate pair on the caller's own data, times one forward + adjoint
(CUDA events, after one warm-up), and returns the fastest pair.  Results are
cached in a JSON file keyed by GPU name and a coarse workload class, so a
repeated workload pays the search once.  The interaction-list buffers are
fixed by design (tiles of 32 sources, 64-entry lists per warp), so there is
no list depth to tune.
"""
from __future__ import annotations

import json
import math
import os

import torch

DEFAULT_CANDIDATES = ((8, 16), (8, 32), (16, 16), (16, 32), (32, 16), (32, 32))


def _cache_path() -> str:
    return os.environ.get("SFG_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sfg", "autotune.json"))


def workload_key(n: int, n_clouds: int, n_active: int, theta: float) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    frac = max(n_active, 1) / max(n, 1)
    return (f"{name}|n=2^{round(math.log2(max(n, 1)))}|clouds=2^{round(math.log2(max(n_clouds, 1)))}"
            f"|active=2^{round(math.log2(frac))}|theta={theta:g}")


def _load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def tune(pos, mass, soft, is_sink=None, *, offsets=None, active=None, cot_a=None, cot_phi=None, theta=0.5,
         candidates=DEFAULT_CANDIDATES, use_cache: bool = True, cache_path: str | None = None) -> dict:
    """Fastest (leaf_size, group_size) for this workload: {"leaf_size", "group_size", "ms", "key", "trials"}."""
    from . import Tree
    n = pos.shape[0]
    n_active = n if active is None else active.numel()
    n_clouds = 1 if offsets is None else len(offsets) - 1
    key = workload_key(n, n_clouds, n_active, theta)
    path = cache_path or _cache_path()
    cache = _load_cache(path) if use_cache else {}
    if key in cache:
        return dict(cache[key], key=key, cached=True)
    if cot_a is None:
        cot_a = torch.ones((n_active, 3), dtype=torch.float64, device=pos.device)
    trials = []
    stream = torch.cuda.current_stream(pos.device)
    for leaf, group in candidates:
        best = float("inf")
        for rep in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t = Tree(pos, mass, soft, is_sink, theta=theta, leaf_size=leaf, group_size=group, offsets=offsets)
            t.accel(active)
            t.accel_vjp(active, cot_a, cot_phi)
            e1.record(stream)
            e1.synchronize()
            t.close()
            if rep:  # the first pass warms up allocations and caches
                best = min(best, e0.elapsed_time(e1))
        trials.append({"leaf_size": leaf, "group_size": group, "ms": best})
    win = min(trials, key=lambda r: r["ms"])
    out = {"leaf_size": win["leaf_size"], "group_size": win["group_size"], "ms": win["ms"], "trials": trials}
    if use_cache:
        cache[key] = out
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, path)
        except OSError:
            pass
    return dict(out, key=key, cached=False)
