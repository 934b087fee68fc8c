"""Autotuner for the launch-shape parameters of a workload.

The tree's leaf size (N_leaf) and group size (targets sharing one walk) trade
walk length against list length, and the list-buffer depth (the sources
each active lane stages per chunk of the evaluation: 1, 2 or 4) trades the
per-chunk costs against shared memory per warp; the best choice depends on
the particle distribution, the active fraction and the GPU.  ``tune`` builds
the tree with each candidate on the caller's own data, times one forward +
adjoint (CUDA events, after one warm-up), and returns the fastest: first over
(leaf size, group size) at depth 1, then over the other depths at the best
pair.  Results are cached in a JSON file keyed by GPU name and a coarse
workload class, so a repeated workload pays the search once.
"""
from __future__ import annotations

import json
import math
import os

import torch

DEFAULT_CANDIDATES = ((8, 16), (8, 32), (16, 16), (16, 32), (32, 16), (32, 32))
DEPTHS = (1, 2, 4)
KEY_VERSION = "v4"  # cache entries carry the list depth


def _cache_path() -> str:
    return os.environ.get("SFG_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sfg", "autotune.json"))


def workload_key(n: int, n_clouds: int, n_active: int, theta: float) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    frac = max(n_active, 1) / max(n, 1)
    return (f"{name}|n=2^{round(math.log2(max(n, 1)))}|clouds=2^{round(math.log2(max(n_clouds, 1)))}"
            f"|active=2^{round(math.log2(frac))}|theta={theta:g}|{KEY_VERSION}")


def _load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def tune(pos, mass, soft, is_sink=None, *, offsets=None, active=None, cot_a=None, cot_phi=None, theta=0.5,
         candidates=DEFAULT_CANDIDATES, depths=DEPTHS, use_cache: bool = True, cache_path: str | None = None) -> dict:
    """Fastest (leaf_size, group_size, list_depth) for this workload:
    {"leaf_size", "group_size", "list_depth", "ms", "key", "trials"}."""
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

    def trial(leaf, group, depth):
        best = float("inf")
        for rep in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t = Tree(pos, mass, soft, is_sink, theta=theta, leaf_size=leaf, group_size=group, list_depth=depth,
                     offsets=offsets)
            t.accel(active)
            t.accel_vjp(active, cot_a, cot_phi)
            e1.record(stream)
            e1.synchronize()
            t.close()
            if rep:  # the first pass warms up allocations and caches
                best = min(best, e0.elapsed_time(e1))
        trials.append({"leaf_size": leaf, "group_size": group, "list_depth": depth, "ms": best})
        return trials[-1]

    first = 1 if 1 in depths else depths[0]
    for leaf, group in candidates:
        trial(leaf, group, first)
    win = min(trials, key=lambda r: r["ms"])
    for depth in depths:
        if depth != first:
            trial(win["leaf_size"], win["group_size"], depth)
    win = min(trials, key=lambda r: r["ms"])
    out = {"leaf_size": win["leaf_size"], "group_size": win["group_size"], "list_depth": win["list_depth"],
           "ms": win["ms"], "trials": trials}
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
