"""The CPU oracle baseline of bench.py (its cpu_baseline and the reference
arm's step): the estimate of a whole step is extrapolated from a sampled
pass per walked group and per evaluated row, so a pass over every row must
reproduce the measured pass, and sampled passes must land near it."""
import numpy as np

import bench
import gen


def _cloud():
    c = gen.clumpy_cloud(40000, n_clumps=16, n_sink=8, seed=31)
    act = gen.active_subset(c.n, 0.2, seed=3)
    ca, cp = gen.cotangents(act.size, seed=4)
    return c, act, ca, cp


def test_full_sample_covers_every_row_and_group():
    c, act, ca, cp = _cloud()
    r = bench.cpu_baseline({"theta": 0.5}, c, act, ca, cp, sample=act.size)
    assert r["rows"] == act.size and r["kind"] == "oracle" and r["cores"] >= 1
    assert f"of {act.size} active rows" in r["sample"]
    # every group is walked when every row is needed
    walked, total = [int(x) for x in r["sample"].split("then ")[1].split(" group walks")[0].split(" of ")]
    assert walked == total
    assert r["value"] > 0 and np.isclose(r["value"], act.size / r["est_step_s"], rtol=1e-3)


def test_sampled_estimates_agree_with_the_full_pass():
    c, act, ca, cp = _cloud()
    full = bench.cpu_baseline({"theta": 0.5}, c, act, ca, cp, sample=act.size, seed=1)
    part = bench.cpu_baseline({"theta": 0.5}, c, act, ca, cp, sample=act.size // 4, seed=2)
    # smaller passes run the OpenMP loops less efficiently: conservative, but
    # within a small factor of the full pass
    assert 0.2 * full["value"] < part["value"] < 2.0 * full["value"]


def test_growing_sample_stops_at_every_row():
    c, act, ca, cp = _cloud()
    r = bench.cpu_baseline({"theta": 0.5}, c, act, ca, cp, sample=None, target_s=1e3)
    assert r["rows"] == act.size
