#!/usr/bin/env python
"""Benchmark of the self-gravity hot path (STARFORGE methods paper, Sec. 2.2).

One step = the whole path over one synthetic cloud: sfg_build (frame, keys,
sort, octree, FP64 moments) + sfg_accel (groups, walk, FP32 evaluation) at the
active particles + sfg_accel_vjp (adjoint with frozen lists) for random
cotangents.  Metric: active-particle gravity evaluations per second
(= active particles / step time), with the walk kernel's FP32 throughput
against the GB300 FP32 ALU peak.

Default workload (paper-20M): the paper-scale clumpy GMC-like cloud --
2e7 equal-mass cells, 70 % of the mass in 2048 Plummer clumps and 30 %
uniform in the unit sphere, 32nd-neighbour softening, 1024 sinks
(log-normal masses, softening 1e-3), theta = 0.5, quadrupoles, a random 10 %
active subset.  clumpy-2M is the same recipe at 2^21 cells, 512 clumps and
256 sinks.  Inputs are resident in HBM when the timed region starts; L2 (129
MB) is flushed before every timed step by writing a 512 MB buffer.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload paper-20M|clumpy-2M|ensemble-256] [--active-frac F]
    python bench.py --opening-curve     # accuracy vs cost of the opening rules

Multi-GPU (torchrun): every rank solves its own independent cloud (seed +
rank); no collective touches the data path; timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# FP32 operations per interaction, counted from the evaluation source
# (eval_chunks_body.inc: chunk_fwd_parts for every P2P pair, chunk_fwd_nodes
# with quadrupole / monopole); FFMA = 2, FADD/FMUL/MUFU.RSQ = 1.  The deferred
# evaluation of the pairs inside a softening support, padding slots and
# absent targets are extra work and not counted.
FLOP_P2P = 20
FLOP_P2M_QUAD = 53
FLOP_P2M_MONO = 20
# Adjoint (eval_chunks_body.inc: chunk_vjp_parts for every P2P pair,
# chunk_vjp_nodes with quadrupole), same counting rule; the source-side
# rotation shuffles and the deferred softened pairs are not counted.
FLOP_VJP_P2P = 44
FLOP_VJP_P2M_QUAD = 137
# DRAM bytes per launch of the evaluation kernels (dram__bytes_read.sum +
# dram__bytes_write.sum, one ncu capture per list depth), valid only for the
# evaluation sources (sha256 over EVAL_SOURCES), workload and launch shape they
# were taken on; otherwise the line reports null.
EVAL_TRAFFIC = {"sha256": "47d1dda0bfff05e8e772f39b0ba1687f9ddafc886f81e3134f3c5449c9fe7b7b",
                "workload": "paper-20M", "leaf_size": 32, "group_size": 16,
                "by_depth": {1: {"fwd": 14087021312, "vjp": 27807148032},
                             2: {"fwd": 13966775296, "vjp": 28388249344}}}
EVAL_SOURCES = ("walk.cu", "eval_chunks.cuh", "eval_chunks_body.inc")
# Algorithmic HBM bytes per particle of sfg_build (frame 40, keys 36, 8 sort
# passes x 32, gather 94, moments + walk records 150).
BUILD_BYTES_PER_PARTICLE = 576

WORKLOADS = {
    "clumpy-2M": dict(n_gas=1 << 21, n_clumps=512, n_sink=256, theta=0.5, active=0.1, seed_id=2),
    "paper-20M": dict(n_gas=20_000_000, n_clumps=2048, n_sink=1024, theta=0.5, active=0.1, seed_id=5),
    "clumpy-256K": dict(n_gas=1 << 18, n_clumps=128, n_sink=64, theta=0.5, active=0.1, seed_id=2),
}


def eval_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in EVAL_SOURCES:
        with open(os.path.join(ROOT, "paper_2010_11254_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak(sfg, sms: int, sm_max_mhz: float) -> tuple:
    """The FP32 peak the evaluation roofline is taken against: the library's
    FFMA throughput probe (sfg_fp32_peak, best of two launches at the clocks of
    this run), with the figure derived from the unit count and the maximum SM
    clock reported beside it."""
    measured = max(sfg.fp32_peak()["tflops"] for _ in range(2))
    derived = sms * 128 * 2 * sm_max_mhz * 1e6 / 1e12
    return measured, (f"measured: FFMA probe sfg_fp32_peak, {measured:.1f} TFLOP/s; derived: {sms} SMs x 128 "
                      f"FP32 lanes x 2 x {sm_max_mhz:.0f} MHz = {derived:.1f} TFLOP/s"), derived


def make_cloud(wl: dict, rank: int):
    """The workload's cloud; with SFG_CLOUD_CACHE=<dir> the generated arrays are
    kept there (npz) for later runs of the same workload and rank."""
    import gen
    seed = gen.CONFIG_SEED[wl["seed_id"]] + 1000 * rank
    cache = os.environ.get("SFG_CLOUD_CACHE")
    path = None
    if cache:
        path = os.path.join(cache, f"cloud_{wl['n_gas']}_{wl['n_clumps']}_{wl['n_sink']}_{seed}.npz")
        if os.path.exists(path):
            z = np.load(path)
            return gen.Cloud(z["pos"], z["mass"], z["soft"], z["is_sink"], seed, "clumpy (cached)"), seed
    c = gen.clumpy_cloud(wl["n_gas"], n_clumps=wl["n_clumps"], n_sink=wl["n_sink"], seed=seed)
    if path:
        os.makedirs(cache, exist_ok=True)
        np.savez(path, pos=c.pos, mass=c.mass, soft=c.soft, is_sink=c.is_sink)
    return c, seed


def make_active(c, frac: float, seed: int):
    import gen
    act = gen.active_subset(c.n, frac, seed=seed)
    ca, cp = gen.cotangents(act.size, seed=seed + 7)
    return act, ca, cp


def make_inputs(wl: dict, rank: int, frac: float | None):
    c, seed = make_cloud(wl, rank)
    f = wl["active"] if frac is None else frac
    act, ca, cp = make_active(c, f, seed)
    return c, act, ca, cp, f


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(os.environ.get("SFG_BENCH_OUT") or tempfile.gettempdir(),
                                 f"sfg_bench_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# The oracle's tree and group shape for the CPU baselines: the shape the
# autotuner picks for the clumpy workloads on the GPU.
ORACLE_LEAF, ORACLE_GROUP = 32, 16


def cpu_baseline(wl: dict, c, act, ca, cp, sample: int | None = None, seed: int = 0, target_s: float = 20.0) -> dict:
    """The oracle as it stands (FP64, OpenMP) on a bounded sample: the full
    tree build, then the group walks the sampled active rows need and their
    field and adjoint.  The step time is extrapolated per walked group (to
    every group) and per evaluated row (to every active row): a sparse sample
    walks about one group per row, so charging the walk per row would count
    each group's walk once per member.  Without a fixed `sample`, the sample
    grows from 1024 rows until its rows take at least half of `target_s`
    seconds (or every active row is in); the last pass is the one reported."""
    import oracle
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    tr = oracle.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=ORACLE_LEAF)
    t1 = time.perf_counter()

    def timed(f):
        ta = time.perf_counter()
        r = f()
        return r, time.perf_counter() - ta

    def rows_pass(k):
        # every stage once for one row (its fixed cost) and once for the
        # sample; the differences give the cost per walked group and per row
        t_start = time.perf_counter()
        pick = np.sort(rng.choice(act.size, min(k, act.size), replace=False))
        rows = act[pick]
        _, w1 = timed(lambda: tr.walk(act, ORACLE_GROUP, wl["theta"], need=rows[:1]))
        walked1 = int(tr.groups()[:, 3].sum())
        _, a1 = timed(lambda: tr.accel_group(rows[:1]))
        _, v1 = timed(lambda: tr.vjp(rows[:1], ca[pick[:1]], cp[pick[:1]]))
        ng, w = timed(lambda: tr.walk(act, ORACLE_GROUP, wl["theta"], need=rows))
        walked = int(tr.groups()[:, 3].sum())
        _, a = timed(lambda: tr.accel_group(rows))
        _, v = timed(lambda: tr.vjp(rows, ca[pick], cp[pick]))
        dr = max(rows.size - 1, 1)
        per_group = max(0.0, w - w1) / max(walked - walked1, 1)
        per_row = (max(0.0, a - a1) + max(0.0, v - v1)) / dr
        est = (w1 + per_group * (ng - walked1)) + (a1 + v1) + per_row * (act.size - 1)
        return rows.size, walked, ng, est, time.perf_counter() - t_start

    t2 = time.perf_counter()
    if sample is None:
        # grow the sample until its rows take about target_s (or all rows are in)
        k = 1024
        while True:
            t2 = time.perf_counter()
            n_rows, walked, ng, est, took = rows_pass(k)
            if took >= 0.5 * target_s or n_rows >= act.size:
                break
            k = int(min(act.size, k * min(16.0, target_s / max(took, 1e-3))))
    else:
        n_rows, walked, ng, est, _ = rows_pass(sample)
    t3 = time.perf_counter()
    t_build = t1 - t0
    t_step = t_build + est
    return {"value": act.size / t_step, "unit": "evals/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"oracle tree build over all {c.n} particles (leaf {ORACLE_LEAF}), then {walked} of {ng} "
                      f"group walks (groups of <= {ORACLE_GROUP}) and the field and adjoint of {n_rows} of "
                      f"{act.size} active rows; walk cost extrapolated per group, evaluation per row",
            "cpu_seconds_measured": round(t_build + (t3 - t2), 3), "est_step_s": round(t_step, 4),
            "rows": int(n_rows)}


def force_error(c, act, acc, phi, sample: int = 1000, seed: int = 0) -> dict:
    """Median and 99th-percentile relative force error of the GPU result
    against the FP64 direct sum (the oracle) on sampled active rows."""
    import oracle
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(act.size, min(sample, act.size), replace=False))
    ad, pd = oracle.direct(c.pos, c.mass, c.soft, c.is_sink, act[pick])
    e = np.linalg.norm(acc[pick] - ad, axis=1) / np.linalg.norm(ad, axis=1)
    ep = np.abs(phi[pick] - pd) / np.abs(pd)
    return {"vs": "FP64 direct sum", "sample": int(pick.size), "median": float(np.median(e)),
            "p99": float(np.percentile(e, 99)), "phi_median": float(np.median(ep)),
            "phi_p99": float(np.percentile(ep, 99))}


def aggregate(local_ms: float, units_per_rank: int, world: int, dist=None, device=None):
    """Whole-job throughput: every rank did `units_per_rank` in local_ms; the
    job time is the slowest rank's (max over ranks)."""
    t = local_ms
    if dist is not None and world > 1:
        import torch
        v = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        t = float(v.item())
    return t, world * units_per_rank / (t * 1e-3)


def run_reference(args, wl, rank, world):
    """--impl reference: the CPU oracle on this workload (rank 0 only).  One
    step is a bounded sample of the workload: the oracle tree over every
    particle, then the group walks, field and adjoint of a random sample of
    the active rows (sized in the first warm-up step to about 4-8 s of row
    work); ms_per_step is that step's wall time, and the value is the evals/s
    of a whole step extrapolated from it (walks per group, evaluation per
    row)."""
    if rank != 0:
        return
    c, act, ca, cp, frac = make_inputs(wl, 0, args.active_frac)
    # the first warm-up step sizes the row sample (about 8 s of rows per step),
    # the others run it
    sample = None
    for k in range(max(args.warmup, 1)):
        r = cpu_baseline(wl, c, act, ca, cp, sample=sample, seed=1 + k, target_s=8.0)
        sample = r["rows"]
    vals, wall = [], []
    r = None
    for k in range(args.steps):
        t0 = time.perf_counter()
        r = cpu_baseline(wl, c, act, ca, cp, sample=sample, seed=10 + k)
        wall.append(time.perf_counter() - t0)
        vals.append(r["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": "active-particle gravity evaluations per second (build + field + adjoint)",
            "value": v, "unit": "evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(wall), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_particles": int(c.n), "n_active": int(act.size),
                       "leaf_size": ORACLE_LEAF, "group_size": ORACLE_GROUP,
                       "active_frac": frac, "theta": wl["theta"]},
            "cpu_baseline": {"kind": "oracle", "cores": r["cores"],
                             "sample": r["sample"] + "; ms_per_step is the wall time of one such sampled step",
                             "value": v, "est_full_step_s": round(statistics.median(act.size / x for x in vals), 3)},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


ENSEMBLE = dict(n_clouds=256, theta=0.5, seed_id=4)


def ensemble_inputs(rank: int):
    import gen
    clouds = gen.ensemble(ENSEMBLE["n_clouds"], seed=gen.CONFIG_SEED[ENSEMBLE["seed_id"]] + 1000 * rank)
    cat = [np.concatenate([getattr(c, f) for c in clouds]) for f in ("pos", "mass", "soft", "is_sink")]
    off = [0] + [int(x) for x in np.cumsum([c.n for c in clouds])]
    ca, cp = gen.cotangents(off[-1], seed=gen.CONFIG_SEED[ENSEMBLE["seed_id"]] + 7)
    return clouds, cat, off, ca, cp


def oracle_ensemble_sample(clouds, budget: int, seed: int, leaf_size: int = 16, group_size: int = 32) -> dict:
    """The oracle (FP64, OpenMP) on a random sample of whole clouds holding
    about `budget` particles: build, walk, field and adjoint of every particle
    of each sampled cloud; the time per particle is extrapolated to the whole
    ensemble."""
    import gen
    import oracle
    rng = np.random.default_rng(seed)
    picked, total = [], 0
    for k in rng.permutation(len(clouds)):
        if total >= budget:
            break
        picked.append(int(k))
        total += clouds[k].n
    t0 = time.perf_counter()
    for k in picked:
        c = clouds[k]
        rows = np.arange(c.n, dtype=np.int64)
        ca, cp = gen.cotangents(c.n, seed=seed + k)
        tr = oracle.Tree(c.pos, c.mass, c.soft, c.is_sink, leaf_size=leaf_size)
        tr.walk(rows, group_size, ENSEMBLE["theta"])
        tr.accel_group(rows)
        tr.vjp(rows, ca, cp)
    dt = time.perf_counter() - t0
    n_all = sum(c.n for c in clouds)
    est = dt * n_all / total
    return {"value": len(clouds) / est, "unit": "clouds/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{len(picked)} whole clouds ({total} particles, all active) of {len(clouds)}: "
                      f"build + walk + field + adjoint; time per particle extrapolated to {n_all} particles",
            "cpu_seconds_measured": round(dt, 3), "est_step_s": round(est, 3)}


def run_ensemble(args, rank, world, dist, dev):
    """Batched ensemble: 256 independent clouds (uniform recipe, N log-uniform
    in [1e3, 2e5], 0..64 sinks) in one forest, every particle active.  Leaf
    and group size come from the autotuner (untimed).  A step =
    sfg_build_batch + sfg_accel + sfg_accel_vjp of all clouds on the tree just
    built."""
    import torch
    import paper_2010_11254_gb300 as sfg
    from paper_2010_11254_gb300 import autotune
    clouds, cat, off, ca_h, cp_h = ensemble_inputs(rank)
    n = off[-1]
    pos, mass, soft, sink, ca, cp = (torch.from_numpy(x).to(dev) for x in cat + [ca_h, cp_h])
    theta = ENSEMBLE["theta"]
    tuned = autotune.tune(pos, mass, soft, sink, offsets=off, cot_a=ca, cot_phi=cp, theta=theta)
    kw = dict(theta=theta, leaf_size=tuned["leaf_size"], group_size=tuned["group_size"],
              list_depth=tuned.get("list_depth", 0), quadrupole=True, offsets=off)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step(timing: bool):
        t = sfg.Tree(pos, mass, soft, sink, **kw)
        t.set_timing(timing)
        a, p = t.accel(None)
        gp, gm = t.accel_vjp(None, ca, cp)
        return t, a, p, gp, gm

    for _ in range(args.warmup):
        step(True)[0].close()
    torch.cuda.synchronize(dev)
    step_ms = []
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    for k in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t, acc, phi, g_pos, g_mass = step(True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if k < args.steps - 1:
            t.close()
    clocks = sampler.stop()
    st = t.stats()
    fwd_lat, vjp_lat = t.cloud_times()
    t.check()
    t.close()
    launches_per_step = int(st["n_launches"])
    ms, value = aggregate(statistics.mean(step_ms), len(clouds), world, dist, dev)
    peaks, peak_src = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_text, _ = fp32_peak(sfg, sms, float(peaks.get("sm_max_mhz", 2070.0)))
    vflops = st["n_p2p"] * FLOP_VJP_P2P + st["n_p2m"] * FLOP_VJP_P2M_QUAD
    ach = vflops / (st["vjp_walk_ms"] * 1e-3) / 1e12
    # a fixed tree re-evaluated: forward + adjoint captured once in a CUDA graph
    tf = sfg.Tree(pos, mass, soft, sink, **kw)
    a0, _ = tf.accel(None)
    tf.accel_vjp(None, ca, cp)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        a_g, _ = tf.accel(None)
        tf.accel_vjp(None, ca, cp)
    for _ in range(3):
        graph.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    e1.synchronize()
    replay_ms = e0.elapsed_time(e1) / args.steps
    gdiff = float((a_g - a0).abs().max().item() / a0.abs().max().item())
    tf.check()
    tf.close()
    # e2e: pinned host inputs -> device, batched build, field, adjoint, results -> pinned host,
    # pipelined like the single-cloud loop (copy stream, two device slots, L2 flush timed)
    h_in = [torch.from_numpy(x).pin_memory() for x in cat + [ca_h, cp_h]]
    h_out = [torch.empty(tuple(x.shape), dtype=x.dtype).pin_memory() for x in (acc, phi, g_pos, g_mass)]
    copy_s = torch.cuda.Stream(dev)
    slots = [[torch.empty(x.shape, dtype=x.dtype, device=dev) for x in h_in] for _ in range(2)]

    def e2e_run(nsteps: int) -> float:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev_in = [torch.cuda.Event(), torch.cuda.Event()]
        last_use = [None, None]
        e0.record(stream)

        def upload(k):
            sl = k % 2
            copy_s.wait_event(e0)
            if last_use[sl] is not None:
                copy_s.wait_event(last_use[sl])
            with torch.cuda.stream(copy_s):
                for d, h in zip(slots[sl], h_in):
                    d.copy_(h, non_blocking=True)
            ev_in[sl].record(copy_s)

        upload(0)
        for k in range(nsteps):
            sl = k % 2
            stream.wait_event(ev_in[sl])
            flush.fill_(1)
            dv = slots[sl]
            t = sfg.Tree(dv[0], dv[1], dv[2], dv[3], **kw)
            res = t.accel(None) + t.accel_vjp(None, dv[4], dv[5])
            done = torch.cuda.Event()
            done.record(stream)
            last_use[sl] = done
            if k + 1 < nsteps:
                upload(k + 1)
            copy_s.wait_event(done)
            with torch.cuda.stream(copy_s):
                for h, d in zip(h_out, res):
                    d.record_stream(copy_s)
                    h.copy_(d, non_blocking=True)
            t.close()  # synchronizes the compute stream: after the copies are queued
        stream.wait_stream(copy_s)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / nsteps

    e2e_run(args.warmup)
    e2e = [e2e_run(args.steps)]
    e2e_ms, e2e_val = aggregate(statistics.mean(e2e), len(clouds), world, dist, dev)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_ensemble_sample(clouds, 2_000_000, seed=11, leaf_size=kw["leaf_size"],
                                     group_size=kw["group_size"])
    line = {
        "metric": "clouds per second (batched build + field + adjoint of an ensemble)", "value": value,
        "unit": "clouds/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "ensemble-256", "n_clouds": len(clouds), "n_particles": n,
                   "n_min": min(c.n for c in clouds), "n_max": max(c.n for c in clouds), "active": "all",
                   "theta": theta, "leaf_size": kw["leaf_size"], "group_size": kw["group_size"],
                   "list_depth": kw["list_depth"],
                   "autotune": {"key": tuned["key"], "cached": tuned["cached"], "trials": tuned.get("trials")},
                   "l2": "flushed (512 MB write) before every timed step"},
        "phases_ms": {"build": round(st["build_ms"], 4), "fwd": round(st["fwd_ms"], 4),
                      "fwd_walk": round(st["fwd_walk_ms"], 4), "vjp": round(st["vjp_ms"], 4),
                      "vjp_walk": round(st["vjp_walk_ms"], 4)},
        "per_cloud_completion_ms": {"fwd_walk_p50": float(np.percentile(fwd_lat, 50)),
                                    "fwd_walk_p99": float(np.percentile(fwd_lat, 99)),
                                    "fwd_walk_max": float(fwd_lat.max()),
                                    "vjp_walk_p50": float(np.percentile(vjp_lat, 50)),
                                    "vjp_walk_p99": float(np.percentile(vjp_lat, 99)),
                                    "vjp_walk_max": float(vjp_lat.max())},
        "fixed_tree_graph_replay_ms": round(replay_ms, 4), "graph_vs_eager_max_rel_diff": gdiff,
        "roofline": {"bound": "alu",
                     "kernel": "k_eval_chunks<QUAD, MODE_VJP> (adjoint from stored lists, all clouds in one launch)",
                     "achieved": round(ach, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                     "frac": round(ach / peak, 4), "traffic": None, "peak_source": peak_text},
        "interactions": {"p2p": int(st["n_p2p"]), "p2m": int(st["n_p2m"]),
                         "p2p_newtonian_list": int(st["n_p2p_newton"]), "groups": int(st["n_groups"])},
        "particles_per_s": n * world / (ms * 1e-3),
        "e2e": {"value": e2e_val, "unit": "clouds/s",
                "h2d_bytes_per_step": sum(x.numel() * x.element_size() for x in h_in),
                "d2h_bytes_per_step": sum(x.numel() * x.element_size() for x in h_out), "ms_per_step": round(e2e_ms, 3)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference_ensemble(args, rank):
    """--impl reference --workload ensemble-256: the oracle on a bounded
    sample of whole clouds per step (rank 0 only)."""
    if rank != 0:
        return
    clouds, cat, off, ca, cp = ensemble_inputs(0)
    for k in range(args.warmup):
        oracle_ensemble_sample(clouds, 10_000, seed=100 + k)
    vals = [oracle_ensemble_sample(clouds, 40_000, seed=200 + k) for k in range(args.steps)]
    v = statistics.median(r["value"] for r in vals)
    r = vals[-1]
    line = {"impl": "reference", "metric": "clouds per second (batched build + field + adjoint of an ensemble)",
            "value": v, "unit": "clouds/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * len(clouds) / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "ensemble-256", "n_clouds": len(clouds), "n_particles": off[-1],
                       "active": "all", "theta": ENSEMBLE["theta"]},
            "cpu_baseline": {"kind": "oracle", "cores": r["cores"], "sample": r["sample"], "value": v},
            "e2e": {"value": v, "unit": "clouds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_point(args, wl, c, act, ca, cp, frac, rank, world, local, dist, dev):
    """One bench line: warm-up and timed steps, e2e loop, rooflines, error."""
    import torch
    import paper_2010_11254_gb300 as sfg
    d_pos = torch.from_numpy(c.pos).to(dev)
    d_mass = torch.from_numpy(c.mass).to(dev)
    d_soft = torch.from_numpy(c.soft).to(dev)
    d_sink = torch.from_numpy(c.is_sink).to(dev)
    d_act = torch.from_numpy(act).to(dev)
    d_ca = torch.from_numpy(ca).to(dev)
    d_cp = torch.from_numpy(cp).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuned = None
    leaf, group, depth = args.leaf_size, args.group_size, args.list_depth
    if leaf is None or group is None or depth is None:
        # launch shape from the autotuner (untimed; cached per GPU and workload class)
        from paper_2010_11254_gb300 import autotune
        tuned = autotune.tune(d_pos, d_mass, d_soft, d_sink, active=d_act, cot_a=d_ca, cot_phi=d_cp,
                              theta=wl["theta"])
        leaf = tuned["leaf_size"] if leaf is None else leaf
        group = tuned["group_size"] if group is None else group
        depth = tuned.get("list_depth", 0) if depth is None else depth
    kw = dict(theta=wl["theta"], leaf_size=leaf, group_size=group, list_depth=depth, quadrupole=True,
              precision=args.precision, store_lists=bool(args.store_lists))
    lists = bool(args.store_lists) and args.precision == 0
    kname = "k_eval_chunks" if lists else "k_walk"

    def one_step():
        tree = sfg.Tree(d_pos, d_mass, d_soft, d_sink, **kw)
        tree.set_timing(True)
        acc, phi = tree.accel(d_act)
        g_pos, g_mass = tree.accel_vjp(d_act, d_ca, d_cp)
        return tree, (acc, phi, g_pos, g_mass)

    for _ in range(args.warmup):
        tree, out = one_step()
        tree.check()
        tree.close()

    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    times, walk_ms, vjp_walk_ms, fwd_ms, vjp_ms, build_ms = [], [], [], [], [], []
    p2p = p2m = p2p_newt = launches = n_ovf = 0
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tree, out = one_step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        st = tree.stats()
        walk_ms.append(st["fwd_walk_ms"])
        vjp_walk_ms.append(st["vjp_walk_ms"])
        fwd_ms.append(st["fwd_ms"])
        vjp_ms.append(st["vjp_ms"])
        build_ms.append(st["build_ms"])
        p2p, p2m, p2p_newt = st["n_p2p"], st["n_p2m"], st["n_p2p_newton"]
        n_ovf = st["n_overflow"]
        launches += st["n_launches"]
        tree.check()
        tree.close()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    acc_h, phi_h = out[0].cpu().numpy(), out[1].cpu().numpy()
    if dist is not None:
        dist.barrier()
    ms_per_step, value = aggregate(sum(times) / args.steps, act.size, world, dist, dev)

    # end to end: pinned host inputs -> device, the three calls, results -> pinned host.
    # Steps are pipelined as a serving loop would run them: the next step's
    # inputs go up on a copy stream into the other of two device slots while
    # this step computes, and this step's results come down on the copy
    # stream while the next one computes.  Every step's copies are inside
    # the timed region; L2 is flushed at the start of every step (timed).
    h_in = [torch.from_numpy(x).pin_memory() for x in (c.pos, c.mass, c.soft, c.is_sink, act, ca, cp)]
    h_out = [torch.empty((act.size, 3), dtype=torch.float64).pin_memory(),
             torch.empty(act.size, dtype=torch.float64).pin_memory(),
             torch.empty((c.n, 3), dtype=torch.float64).pin_memory(),
             torch.empty(c.n, dtype=torch.float64).pin_memory()]
    bi = sum(x.numel() * x.element_size() for x in h_in)
    bo = sum(x.numel() * x.element_size() for x in h_out)
    copy_s = torch.cuda.Stream(dev)
    slots = [[torch.empty(x.shape, dtype=x.dtype, device=dev) for x in h_in] for _ in range(2)]

    def e2e_run(nsteps: int) -> float:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ev_in = [torch.cuda.Event(), torch.cuda.Event()]
        last_use = [None, None]
        e0.record(stream)

        def upload(k):
            sl = k % 2
            copy_s.wait_event(e0)
            if last_use[sl] is not None:
                copy_s.wait_event(last_use[sl])
            with torch.cuda.stream(copy_s):
                for d, h in zip(slots[sl], h_in):
                    d.copy_(h, non_blocking=True)
            ev_in[sl].record(copy_s)

        upload(0)
        for k in range(nsteps):
            sl = k % 2
            stream.wait_event(ev_in[sl])
            flush.fill_(1)
            dv = slots[sl]
            tree = sfg.Tree(dv[0], dv[1], dv[2], dv[3], **kw)
            acc, phi = tree.accel(dv[4])
            g_pos, g_mass = tree.accel_vjp(dv[4], dv[5], dv[6])
            done = torch.cuda.Event()
            done.record(stream)
            last_use[sl] = done
            if k + 1 < nsteps:
                upload(k + 1)
            copy_s.wait_event(done)
            with torch.cuda.stream(copy_s):
                for h, d in zip(h_out, (acc, phi, g_pos, g_mass)):
                    d.record_stream(copy_s)
                    h.copy_(d, non_blocking=True)
            tree.close()  # synchronizes the compute stream: after the copies are queued
        stream.wait_stream(copy_s)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / nsteps

    e2e_run(args.warmup)
    e2e_times = [e2e_run(args.steps)]
    e2e_ms, e2e_value = aggregate(statistics.mean(e2e_times), act.size, world, dist, dev)

    peaks, peak_src = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak, peak_text, _ = fp32_peak(sfg, sms, sm_max)
    same_src = EVAL_TRAFFIC["sha256"] is not None and EVAL_TRAFFIC["sha256"] == eval_sources_sha256()

    def roof(kernel, flops, ms, traffic_key, model):
        a = flops / (ms * 1e-3) / 1e12
        return {"bound": "alu", "kernel": kernel, "achieved": round(a, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(a / peak, 4),
                "traffic": EVAL_TRAFFIC["by_depth"].get(depth or 1, {}).get(traffic_key)
                if (same_src and args.workload == EVAL_TRAFFIC["workload"]
                    and (leaf, group) == (EVAL_TRAFFIC["leaf_size"], EVAL_TRAFFIC["group_size"])) else None,
                "peak_source": peak_text,
                "flops_per_launch": int(flops), "launch_ms": round(ms, 4), "flop_model": model}

    wk = statistics.mean(walk_ms)
    vk = statistics.mean(vjp_walk_ms)
    r_fwd = roof(f"{kname}<QUAD, MODE_EVAL> (forward FP32 evaluation{' from stored lists' if lists else ''})",
                 p2p * FLOP_P2P + p2m * FLOP_P2M_QUAD, wk, "fwd",
                 f"P2P {FLOP_P2P}, P2M quadrupole {FLOP_P2M_QUAD} FP32 flops per interaction")
    r_vjp = roof(f"{kname}<QUAD, MODE_VJP> (adjoint FP32 tidal-tensor products{' from stored lists' if lists else ''})",
                 p2p * FLOP_VJP_P2P + p2m * FLOP_VJP_P2M_QUAD, vk, "vjp",
                 f"P2P {FLOP_VJP_P2P}, P2M quadrupole {FLOP_VJP_P2M_QUAD} FP32 flops per interaction")
    dominant, other = (r_vjp, r_fwd) if vk >= wk else (r_fwd, r_vjp)
    line = {
        "metric": "active-particle gravity evaluations per second (build + field + adjoint)",
        "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == 0 else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_particles": int(c.n), "n_sinks": int(c.n_sink),
                   "n_active": int(act.size), "active_frac": frac, "theta": wl["theta"],
                   "leaf_size": leaf, "group_size": group,
                   "list_depth": depth or 1, "quadrupole": True,
                   "precision": args.precision, "store_lists": bool(args.store_lists),
                   "autotune": None if tuned is None else {"key": tuned["key"], "cached": tuned["cached"],
                                                            "trials": tuned.get("trials")},
                   "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": f"independent clouds x{world}"},
        "roofline": dominant,
        "roofline_other_walk": other,
        "phases_ms": {"build": round(statistics.mean(build_ms), 4), "fwd": round(statistics.mean(fwd_ms), 4),
                      "fwd_walk": round(wk, 4), "vjp": round(statistics.mean(vjp_ms), 4),
                      "vjp_walk": round(statistics.mean(vjp_walk_ms), 4)},
        "adjoint_over_forward": round(statistics.mean(vjp_ms) / statistics.mean(fwd_ms), 3),
        "interactions": {"p2p": int(p2p), "p2m": int(p2m), "p2p_newtonian_list": int(p2p_newt),
                         "per_active": round((p2p + p2m) / act.size, 1), "overflowed_groups": int(n_ovf),
                         "fwd_per_s": round((p2p + p2m) / (statistics.mean(fwd_ms) * 1e-3), 1)},
        "build_hbm": {"algorithmic_GBps": round(BUILD_BYTES_PER_PARTICLE * c.n / (statistics.mean(build_ms) * 1e-3)
                                                / 1e9, 1), "peak_GBps": peaks.get("hbm_gbs")},
        "particles_per_s": c.n * world / (ms_per_step * 1e-3),
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo, "ms_per_step": round(e2e_ms, 3)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0:
        line["force_error"] = force_error(c, act, acc_h, phi_h, sample=args.error_sample)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, c, act, ca, cp)
    return line


def run_opening_curve(args, wl, c, act, dev):
    """Accuracy against cost of the opening rules of Sec. 2.2 on one cloud:
    the Theta rule alone over a range of Theta, and Theta together with the
    acceleration-based relative clause over a range of alpha.  |g_prev| is the
    field of an accurate pass (Theta = 0.2) standing in for the previous
    step's.  One JSON line per point: the forward time of sfg_accel (groups,
    walk, evaluation; the build is the same for every point and excluded),
    interactions per active row, and the force error against the FP64 direct
    sum on sampled active rows (the direct sums are taken once)."""
    import torch
    import oracle
    import paper_2010_11254_gb300 as sfg
    d_pos = torch.from_numpy(c.pos).to(dev)
    d_mass = torch.from_numpy(c.mass).to(dev)
    d_soft = torch.from_numpy(c.soft).to(dev)
    d_sink = torch.from_numpy(c.is_sink).to(dev)
    d_act = torch.from_numpy(act).to(dev)
    leaf = args.leaf_size or 32
    group = args.group_size or 16
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(act.size, min(args.error_sample, act.size), replace=False))
    ad, _ = oracle.direct(c.pos, c.mass, c.soft, c.is_sink, act[pick])
    t = sfg.Tree(d_pos, d_mass, d_soft, d_sink, theta=0.2, leaf_size=leaf, group_size=group)
    acc, _ = t.accel(d_act)
    t.check()
    t.close()
    g_prev = torch.zeros(c.n, dtype=torch.float64, device=dev)
    g_prev[d_act] = torch.linalg.vector_norm(acc, dim=1)
    points = [(th, 0.0) for th in (0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 1.0)]
    points += [(th, al) for th in (0.7, 1.0) for al in (0.001, 0.0025, 0.005, 0.01, 0.02)]
    for theta, alpha in points:
        fwd = []
        for k in range(args.warmup + args.steps):
            t = sfg.Tree(d_pos, d_mass, d_soft, d_sink, theta=theta, leaf_size=leaf, group_size=group)
            if alpha > 0.0:
                t.set_relative(g_prev, alpha)
            t.set_timing(True)
            acc, _ = t.accel(d_act)
            torch.cuda.synchronize(dev)
            st = t.stats()
            t.check()
            t.close()
            if k >= args.warmup:
                fwd.append(st["fwd_ms"])
        a = acc.cpu().numpy()[pick]
        e = np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1)
        print(json.dumps({
            "metric": "opening-rule accuracy vs cost", "workload": args.workload, "theta": theta,
            "rule": "theta" if alpha == 0.0 else "theta + relative", "alpha": alpha or None,
            "leaf_size": leaf, "group_size": group, "fwd_ms": round(statistics.median(fwd), 4),
            "interactions_per_active": round((st["n_p2p"] + st["n_p2m"]) / act.size, 1),
            "p2p_per_active": round(st["n_p2p"] / act.size, 1), "p2m_per_active": round(st["n_p2m"] / act.size, 1),
            "force_error": {"vs": "FP64 direct sum", "sample": int(pick.size), "median": float(np.median(e)),
                            "p99": float(np.percentile(e, 99)), "max": float(e.max())}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper-20M", choices=sorted(WORKLOADS) + ["ensemble-256"])
    ap.add_argument("--active-frac", type=float, default=None)
    ap.add_argument("--active-fracs", default=None,
                    help="comma-separated active fractions: one line each on the same cloud")
    ap.add_argument("--error-sample", type=int, default=10000,
                    help="active rows checked against the FP64 direct sum")
    ap.add_argument("--store-lists", type=int, default=1, choices=[0, 1])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--leaf-size", type=int, default=None, help="default: the autotuner's choice")
    ap.add_argument("--group-size", type=int, default=None, help="default: the autotuner's choice")
    ap.add_argument("--list-depth", type=int, default=None, choices=[1, 2, 4],
                    help="evaluation chunk depth (sources staged per lane); default: the autotuner's choice")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1],
                    help="0: FP32 pair arithmetic with FP64 frame/moments/potential sums; 1: all FP64")
    ap.add_argument("--opening-curve", action="store_true",
                    help="accuracy vs cost of the Theta and relative opening rules (one line per point)")
    args = ap.parse_args()
    wl = WORKLOADS.get(args.workload)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if wl is None:
            run_reference_ensemble(args, rank)
        else:
            run_reference(args, wl, rank, world)
        return

    import torch
    import paper_2010_11254_gb300 as sfg

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    os.environ.setdefault("SFG_TIMING", "1")
    if args.workload == "ensemble-256":
        run_ensemble(args, rank, world, dist, dev)
        if dist is not None:
            dist.destroy_process_group()
        return

    c, seed = make_cloud(wl, rank)
    if args.opening_curve:
        act, _, _ = make_active(c, wl["active"] if args.active_frac is None else args.active_frac, seed)
        run_opening_curve(args, wl, c, act, dev)
        return
    fracs = ([float(x) for x in args.active_fracs.split(",")] if args.active_fracs
             else [wl["active"] if args.active_frac is None else args.active_frac])
    for frac in fracs:
        act, ca, cp = make_active(c, frac, seed)
        line = run_point(args, wl, c, act, ca, cp, frac, rank, world, local, dist, dev)
        if rank == 0:
            print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
