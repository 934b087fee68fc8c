"""Host logic of the launch-shape autotuner: workload classes and the JSON
cache (a cached workload is answered without building a tree)."""
import json

import numpy as np
import torch

from paper_2010_11254_gb300 import autotune


def test_workload_key_classes():
    k1 = autotune.workload_key(1 << 20, 1, 1 << 17, 0.5)
    assert k1.split("|")[1:] == ["n=2^20", "clouds=2^0", "active=2^-3", "theta=0.5", autotune.KEY_VERSION]
    # sizes within a factor sqrt(2) share a class; theta and cloud count do not merge
    assert autotune.workload_key(1_100_000, 1, 110_000, 0.5).split("|")[1] == "n=2^20"
    assert autotune.workload_key(1 << 20, 256, 1 << 20, 0.5) != autotune.workload_key(1 << 20, 1, 1 << 20, 0.5)
    assert autotune.workload_key(1 << 20, 1, 1 << 20, 0.7) != autotune.workload_key(1 << 20, 1, 1 << 20, 0.5)


def test_cache_hit_skips_search(tmp_path):
    n = 5000
    pos = torch.zeros((n, 3), dtype=torch.float64)
    key = autotune.workload_key(n, 3, n, 0.5)
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({key: {"leaf_size": 8, "group_size": 16, "list_depth": 4, "ms": 1.0, "trials": []}}))
    r = autotune.tune(pos, None, None, offsets=[0, 1000, 2000, n], theta=0.5, cache_path=str(path))
    assert r["cached"] and (r["leaf_size"], r["group_size"], r["list_depth"]) == (8, 16, 4) and r["key"] == key


def test_unreadable_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert autotune._load_cache(str(path)) == {}
    assert np.isfinite(len(autotune.DEFAULT_CANDIDATES))
