"""Benchmark of the ELSR VNS hot path on GB300.

Headline workload: plain GVNS on one synthetic instance with K=50 products and
T=52 periods (generator seed 1), 2000 shaking iterations, kmax=3, mode P
(Algorithm 1's product-parallel VND).  One step = one whole GVNS run through
the C ABI (stage the instance, VND, 2000 x (shake, VND, accept)), i.e. every
step of the hot path.  Metric: candidate moves evaluated per second (the sum
over neighbourhood evaluations of |N_j|, counted exactly as the oracle counts
them); VNS instances/s is reported beside it.

The same JSON line carries `workloads`: the batched forms measured in the same
run, each with its own CUDA-event timing, clocks, integer roofline and CPU
baseline on every host core -- `batch` (1024 instances K ~ U{5..100},
T ~ U{12..52}, 500 iterations each, one persistent launch), `multistart`
(K=100 x T=104, 4096 starts x 1000 iterations, device best-of) and `serve`
(a Poisson stream of 2000 requests/s, K ~ U{5..200}, T ~ U{12..104}, 300
iterations each, p50/p99 latency).  The integer roofline's peak is measured
on the device (elsr_int_issue_probe) with the SM clock sampled.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload batch|multistart|serve   (one workload's record)

``--impl reference`` times the CPU oracle (plain single-threaded C) on a
bounded sample of the headline workload.  Under torchrun (N > 1) every rank
runs independent replicas (one instance, its own seed) and rank 0 prints one
line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The serving workload launches many small kernels side by side on separate
# streams; more hardware work queues than the default 8 keep them from
# queueing behind one another.  Read when CUDA starts, so set it first.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

WORKLOAD = {
    "workload": "plain GVNS, one instance K=50 products x T=52 periods, seed 1, "
                "2000 shaking iterations, kmax=3, mode P",
    "K": 50, "T": 52, "gen_seed": 1, "vns_seed": 1, "iters": 2000, "kmax": 3, "mode": "P",
}
# Paper-shaped instance (the size of the paper's benchmark set: K=300
# products, T=52 periods), secondary measurement via --instance paper.
WORKLOAD_PAPER = {
    "workload": "plain GVNS, one instance K=300 products x T=52 periods (paper-shaped), "
                "seed 3, 1000 shaking iterations, kmax=3, mode P",
    "K": 300, "T": 52, "gen_seed": 3, "vns_seed": 1, "iters": 1000, "kmax": 3, "mode": "P",
}
METRIC = "candidate moves evaluated/s"
UNIT = "moves/s"
INT_OPS_PER_STEP = 16         # algorithmic integer operations per decode step
# DRAM bytes (read + written) per launch, from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on the current kernels.  The speculative kernel of
# the plain run is not profiled: its figure is a one-team launch of the same
# run (100 iterations: 280,580 B read, 0 written) scaled by the iterations, an
# upper bound since the instance is staged once per run.
TRAFFIC_PLAIN_PER_100_ITERS = 280_580
TRAFFIC_BATCH_LAUNCH = 16_460_000 + 12_140_000  # batch workload's timed launch (500 iterations)
LANES_PER_SM = 128            # 32-bit integer lanes per SM (4 SMSPs x 32), for context
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="elsr_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(iters: int):
    """The oracle as it stands, single-threaded, on the first `iters`
    iterations of the workload (a bounded sample)."""
    import oracle
    from paper_1704_05132_gb300 import gen
    inst = oracle.Instance.from_arrays(gen.plain_medium())
    t0 = time.perf_counter()
    r = oracle.vns(inst, WORKLOAD["vns_seed"], iters, WORKLOAD["kmax"], 0)
    dt = time.perf_counter() - t0
    return {"value": r.counters["moves_evaluated"] / dt, "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": f"first {iters} of {WORKLOAD['iters']} iterations of the workload "
                      f"({r.counters['moves_evaluated']} moves, {dt:.2f} s)"}


def _oracle_job(job):
    """One oracle GVNS run (in a spawned worker): job = (kind, ident, seed, iters)."""
    import oracle
    from paper_1704_05132_gb300 import gen
    kind, ident, seed, iters = job
    if kind == "batch":
        g = gen.make_instance(0, ident, K_range=(5, 100), T_range=(12, 52))
    elif kind == "multistart":
        g = gen.multistart_large()
    else:
        g = gen.serving_request(ident)
    t0 = time.perf_counter()
    r = oracle.vns(oracle.Instance.from_arrays(g), seed, iters, 3, 0)
    return r.counters["moves_evaluated"], time.perf_counter() - t0


def cpu_baseline_pool(jobs, sample: str):
    """The oracle as it stands on every host core: one independent run per
    worker process (spawned, so no CUDA state is inherited), on a bounded
    sample of a batched workload."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_job, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    moves = sum(m for m, _ in res)
    per_run = sorted(dt for _, dt in res)
    busy = sum(per_run)
    return {"value": moves / wall, "unit": UNIT, "cores": n, "kind": "oracle",
            "instances_per_s": len(jobs) / wall, "p50_run_s": per_run[len(per_run) // 2],
            "one_core": {"value": moves / busy, "unit": UNIT,
                         "instances_per_s": len(jobs) / busy,
                         "note": "the same runs' moves over the sum of their own run "
                                 "times (each run is single-threaded; runs sharing the "
                                 "host's caches make this a slight underestimate)"},
            "sample": sample + f" ({len(jobs)} runs, {moves} moves, {wall:.1f} s wall)"}


def extrapolate_full(cb, runs, iter_scale, how):
    """Add to a pool baseline `cb` the oracle's time for the full workload:
    `runs` runs, each `iter_scale` times the sample's iterations, at the
    sample's runs per second on the same cores."""
    cb["full_workload_s_extrapolated"] = runs * iter_scale / cb["instances_per_s"]
    cb["extrapolation"] = how
    return cb


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1704_05132_gb300 import gen
    oracle.build()
    inst = oracle.Instance.from_arrays(gen.plain_medium())
    iters = args.ref_iters
    for _ in range(args.warmup):
        oracle.vns(inst, WORKLOAD["vns_seed"], iters, WORKLOAD["kmax"], 0)
    moves, t = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.vns(inst, WORKLOAD["vns_seed"], iters, WORKLOAD["kmax"], 0)
        t += time.perf_counter() - t0
        moves += r.counters["moves_evaluated"]
    v = moves / t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": dict(WORKLOAD, sample_iters=iters),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: the first {iters} of {WORKLOAD['iters']} "
                                   "iterations of the workload"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_int_peak(torch, dev, stream):
    """Integer-issue peak of this GPU, measured: elsr_int_issue_probe (eight
    independent chains of add / min / xor / multiply-add per thread, 8 CTAs
    of 256 threads per SM) timed with CUDA events on `stream` over about a
    second, the SM clock sampled meanwhile."""
    import ctypes
    from paper_1704_05132_gb300 import _native as nat
    lib = nat.load()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = sms * 8, 2048
    src = torch.arange(3, 39, dtype=torch.int32, device=dev)
    sink = torch.empty(blocks * 256, dtype=torch.int32, device=dev)
    ops = ctypes.c_int64()

    def launch():
        nat.check(lib.elsr_int_issue_probe(ctypes.c_void_p(stream.cuda_stream), blocks, iters,
                                           ctypes.c_void_p(src.data_ptr()),
                                           ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops)))

    for _ in range(3):
        launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 0
    with ClockSampler(dev.index or 0) as clk:
        t_end = time.perf_counter() + 1.0
        e0.record(stream)
        while time.perf_counter() < t_end or n < 10:
            launch()
            n += 1
            if n % 8 == 0:
                stream.synchronize()
        e1.record(stream)
        e1.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    tops = ops.value * n / (ms / 1e3) / 1e12
    mhz = clocks.get("sm_mhz")
    per_clk = tops * 1e12 / (sms * mhz * 1e6) if mhz else None
    return {"value": tops, "unit": "Tintop/s", "sms": sms, "launches": n, "ms": ms,
            "ops_per_launch": ops.value, "clocks": clocks,
            "int_ops_per_sm_per_clock": per_clk,
            "how": "elsr_int_issue_probe: 8 CTAs x 256 threads per SM, 8 independent chains "
                   "of add, min, xor, multiply-add per thread; CUDA events over ~1 s"}


def roofline_alu(steps, kernel_s, peak, traffic=None, note=""):
    """Integer roofline of a launch: INT_OPS_PER_STEP ops per decode step."""
    achieved = INT_OPS_PER_STEP * steps / kernel_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak["value"], "unit": "Tintop/s",
            "frac": achieved / peak["value"], "traffic": traffic,
            "peak_source": "measured on this GPU (elsr_int_issue_probe, median SM clock "
                           f"{peak['clocks'].get('sm_mhz')} MHz)",
            "note": f"{INT_OPS_PER_STEP} int ops per decode step x {steps} decode steps per "
                    f"launch (device counter, equal to the oracle's definition, taken in a "
                    f"warm-up launch of the same run; the timed launches, whose trajectory is "
                    f"the same, run with the counter off) / launch time" +
                    (f"; {note}" if note else "")}


def _timed_steps(torch, stream, step, steps, warmup, flush, dev):
    """CUDA-event time of each of `steps` calls after `warmup` untimed ones,
    L2 flushed (untimed) before each, clocks sampled meanwhile."""
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(dev.index or 0) as clk:
        for _ in range(steps):
            flush.add_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    return ms, clk.summary()


def bench_staging(torch, stream, flush, dev, b, insts, reps=20):
    """The staging pass alone on the batch's instances: every row's prefix
    tables built in device memory by the stage kernel (the row loader the
    GVNS launch stages shared memory with), CUDA-event timed, L2 flushed
    before each launch.  HBM bytes: D and R read, hM and hR read, tables
    ((T + 1) int2 per row) and C0 (one int64 per row) written."""
    rows = sum(g.K for g in insts)
    cells = sum(g.K * g.T for g in insts)
    nbytes = 8 * cells + 8 * rows + 8 * (cells + rows) + 8 * rows
    ms, _ = _timed_steps(torch, stream, b.stage_tables, reps, 3, flush, dev)
    ms.sort()
    med = ms[len(ms) // 2] / 1e3
    hbm = _peaks().get("hbm_gbs")
    gbs = nbytes / med / 1e9
    return {"kernel": "stage_kernel", "bytes": nbytes, "rows": rows, "cells": cells,
            "ms_median": med * 1e3, "ms_min": ms[0], "launches": reps, "gbs": gbs,
            "hbm_peak_gbs": hbm, "frac": gbs / hbm if hbm else None,
            "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}


def bench_batch(torch, dev, stream, flush, peak, steps, warmup, args, cpu=True):
    """1024 independent instances K ~ U{5..100}, T ~ U{12..52} (seed 0, ids
    0..1023), 500 iterations each, in one persistent launch per step."""
    from paper_1704_05132_gb300 import elsr, gen
    n = args.n or 1024
    iters = args.iters if args.iters is not None else 500
    insts = gen.batch_uneven(n)
    tuned = None
    if not (args.lanes or args.threads or args.cluster):
        from paper_1704_05132_gb300 import autotune  # the Batch below takes its choice
        # probes long enough that the initial descent does not dominate them
        tuned = autotune.tune_batch(insts, probe_iters=100)
    b = elsr.Batch(insts, stream=stream, lanes=args.lanes, threads=args.threads,
                   cluster=args.cluster)
    seeds = np.arange(n, dtype=np.uint64)
    b.run(seeds, iters, 3, 0)          # decode steps counted once, untimed
    counted = b.results()
    segs = sum(r["segments"] for r in counted)
    b.set_count_steps(False)           # the counting launch was the first warm-up
    ms, clocks = _timed_steps(torch, stream, lambda: b.run(seeds, iters, 3, 0), steps,
                              max(0, warmup - 1), flush, dev)
    st = b.results()
    assert all(r["status"] == 0 for r in st)
    assert [r["traj_hash"] for r in st] == [r["traj_hash"] for r in counted]
    moves = sum(r["moves_evaluated"] for r in st)
    t = sum(ms) / 1e3
    stage_bytes = sum(4 * (2 * g.K * g.T + 4 * g.K) for g in insts)
    staging = bench_staging(torch, stream, flush, dev, b, insts)
    rec = {"metric": METRIC, "value": moves * steps / t, "unit": UNIT,
           "instances_per_s": n * steps / t, "ms_per_step": 1e3 * t / steps,
           "steps": steps, "warmup": warmup, "higher_is_better": True,
           "config": {"workload": f"batch of {n} instances, K ~ U{{5..100}}, T ~ U{{12..52}}, "
                                  f"{iters} iterations each, kmax=3, mode P, one persistent "
                                  "launch", "instances": n, "iters": iters,
                      "l2": "flushed between steps (256 MiB device write, untimed)"},
           "moves_per_step": moves, "segments_per_step": segs,
           "launch_shape": b.launch_shape(), "autotuned": tuned, "clocks": clocks,
           "gpu_launches": steps,
           "staging": dict(staging, launch_bytes=stage_bytes,
                           launch_note="instance bytes the GVNS launch reads from HBM "
                                       "(D, R, costs), staged with the same row loader"),
           "roofline": roofline_alu(segs, t / steps, peak,
                                    traffic=TRAFFIC_BATCH_LAUNCH if (n, iters) == (1024, 500)
                                    else None)}
    b.close()
    if cpu and not args.no_cpu_baseline:
        m = min(n, 64)
        rec["cpu_baseline"] = cb = cpu_baseline_pool(
            [("batch", i, i, iters) for i in range(m)],
            f"the first {m} of the {n} instances, {iters} iterations each")
        extrapolate_full(cb, n, 1.0, f"all {n} instances at the sample's instances/s on the "
                                     "same cores (the sample is the workload's first instances)")
    return rec


def bench_multistart(torch, dev, stream, flush, peak, steps, warmup, args, cpu=True):
    """One instance K=100, T=104 (seed 0, id 0), 4096 starts seeded 0..4095,
    1000 iterations each, best-of reduced on the device; one launch per step."""
    from paper_1704_05132_gb300 import elsr, gen
    n = args.n or 4096
    iters = args.iters if args.iters is not None else 1000
    g = gen.multistart_large()
    sv = elsr.Solver(g, stream=stream, lanes=args.lanes, threads=args.threads,
                     cluster=args.cluster)
    box = {}

    def step():
        box["best"] = sv.multistart(0, n, iters, 3, 0)

    step()                             # decode steps counted once, untimed
    counted = sv.multistart_stats(n)
    segs = sum(r["segments"] for r in counted)
    sv.set_count_steps(False)          # the counting launch was the first warm-up
    ms, clocks = _timed_steps(torch, stream, step, steps, max(0, warmup - 1), flush, dev)
    st = sv.multistart_stats(n)
    assert all(r["status"] == 0 for r in st)
    assert [r["traj_hash"] for r in st] == [r["traj_hash"] for r in counted]
    moves = sum(r["moves_evaluated"] for r in st)
    t = sum(ms) / 1e3
    rec = {"metric": METRIC, "value": moves * steps / t, "unit": UNIT,
           "instances_per_s": n * steps / t, "ms_per_step": 1e3 * t / steps,
           "steps": steps, "warmup": warmup, "higher_is_better": True,
           "config": {"workload": f"multi-start, one instance K=100 x T=104, {n} starts "
                                  f"(seeds 0..{n - 1}), {iters} iterations each, device "
                                  "best-of", "starts": n, "iters": iters,
                      "l2": "flushed between steps (256 MiB device write, untimed)"},
           "best_of": {"cost": box["best"][0], "start": box["best"][1]},
           "moves_per_step": moves, "segments_per_step": segs,
           "launch_shape": sv.launch_shape(), "clocks": clocks, "gpu_launches": 2 * steps,
           "roofline": roofline_alu(segs, t / steps, peak)}
    sv.close()
    if cpu and not args.no_cpu_baseline:
        m, it_s = 16, min(iters, 200)
        rec["cpu_baseline"] = cb = cpu_baseline_pool(
            [("multistart", 0, s, it_s) for s in range(m)],
            f"starts 0..{m - 1}, {it_s} of the {iters} iterations each")
        extrapolate_full(cb, n, iters / it_s,
                         f"all {n} starts at {iters} iterations: the sample's time per start "
                         f"scaled by {iters}/{it_s} iterations (an estimate: the early "
                         "iterations include the longer initial descent)")
    return rec


def bench_serve(torch, dev, peak, args, cpu=True):
    """Poisson arrivals (mean `--rate` requests/s) of instances K ~ U{5..200},
    T ~ U{12..104} (seed 5, id = request id), 300 iterations each; p50/p99
    latency (completion - arrival on the host clock) and instances/s."""
    from paper_1704_05132_gb300 import serve
    n = args.requests
    iters = args.iters if args.iters is not None else 300
    warm = serve.poisson_requests(64, args.rate, iters, seed=5, id0=10 ** 6)
    serve.Server(slots=args.slots, max_runs=args.max_runs).run(warm, realtime=False)
    reqs = serve.poisson_requests(n, args.rate, iters, seed=5)
    srv = serve.Server(slots=args.slots, max_runs=args.max_runs)
    with ClockSampler(dev.index or 0) as clk:
        stats = srv.run(reqs)
    s = stats.summary()
    rec = {"metric": METRIC, "value": s["moves_per_s"], "unit": UNIT,
           "instances_per_s": s["instances_per_s"], "offered_per_s": args.rate,
           "p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"], "mean_ms": s["mean_ms"],
           "higher_is_better": True,
           "config": {"workload": f"serving, Poisson arrivals mean {args.rate:g} req/s, "
                                  f"{n} requests K ~ U{{5..200}}, T ~ U{{12..104}}, "
                                  f"{iters} iterations each", "requests": n, "iters": iters,
                      "slots": args.slots, "max_runs_per_team": args.max_runs,
                      "batching": "continuous: requests join running launches through "
                                  "device queues and retire one by one"},
           "launches": s["batches"], "max_inflight": s["max_inflight"], "span_s": s["span_s"],
           "clocks": clk.summary(), "timing": "host clock, arrival to result on the host"}
    if cpu and not args.no_cpu_baseline:
        m = 16
        rec["cpu_baseline"] = cpu_baseline_pool(
            [("serve", r, r, iters) for r in range(m)],
            f"requests 0..{m - 1} solved one per core, {iters} iterations each "
            "(p50_run_s is the oracle's per-request solve time)")
    return rec


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world, rank, local = _dist()
    torch.cuda.set_device(local)  # before the process group: its barriers use this device
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_1704_05132_gb300 import build, elsr, gen
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()

    wl = dict(WORKLOAD_PAPER if args.instance == "paper" else WORKLOAD)
    g = gen.paper_shaped() if args.instance == "paper" else gen.plain_medium()
    mode = 1 if args.mode == "G" else 0
    wl["mode"] = args.mode
    wl["workload"] = wl["workload"].replace("mode P", f"mode {args.mode}")
    if args.workers:
        wl["workload"] = ("fork-join " + wl["workload"] +
                          f", {args.workers} workers per iteration (Algorithm 2, Section 3)")
        wl["workers"] = args.workers
    K, T = g.K, g.T
    seed = wl["vns_seed"] + rank  # replicas: one seed per rank
    stream = torch.cuda.current_stream(dev)
    solver = elsr.Solver(g, stream=stream, lanes=args.lanes, threads=args.threads,
                         cluster=args.cluster, speculation=args.speculation)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    iters = args.iters if args.iters is not None else wl["iters"]

    def step():
        if args.workers:
            solver.vns_forkjoin_run(seed, iters, wl["kmax"], mode, args.workers)
        else:
            solver.vns_run(seed, iters, wl["kmax"], mode)

    for _ in range(args.warmup):
        step()
    st = solver.result(solution=False, traj=False)
    moves_per_step = st["moves_evaluated"]
    segs_per_step = st["segments"]       # decode steps, counted in the warm-up run
    solver.set_count_steps(False)        # the timed runs skip that bookkeeping

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.add_(1)                       # L2 flush between steps (untimed)
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    st2 = solver.result(solution=False, traj=False)
    assert st2["moves_evaluated"] == moves_per_step and st2["status"] == 0
    assert st2["best_cost"] == st["best_cost"] and st2["traj_hash"] == st["traj_hash"]
    solver.set_count_steps(True)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_local = sum(step_ms) / 1e3
    t_max = t_local
    moves_total = moves_per_step * args.steps
    if world > 1:
        tt = torch.tensor([t_local], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
        mv = torch.tensor([moves_total], dtype=torch.float64, device=dev)
        dist.all_reduce(mv, op=dist.ReduceOp.SUM)
        moves_total = float(mv.item())
    value = moves_total / t_max
    kernel_s = t_local / args.steps

    # ---- one full-neighbourhood evaluation (N1 u N2 u N3) per launch ----
    solver.set_state()
    ev_moves = K * (2 * T + 2 * (T - 1))
    for _ in range(3):
        solver.eval_neighbourhood(0b111, 0)
    ev_n = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev_ms = 0.0
    for _ in range(ev_n):
        e0.record(stream)
        solver.eval_neighbourhood(0b111, 0)
        e1.record(stream)
        e1.synchronize()
        ev_ms += e0.elapsed_time(e1)
    eval_launch = {"moves_per_launch": ev_moves, "us_per_launch": 1e3 * ev_ms / ev_n,
                   "moves_per_s": ev_moves * ev_n / (ev_ms / 1e3),
                   "state": "initial solution (all setups open)",
                   "note": "one elsr_eval_neighbourhood call incl. its result copies"}

    # ---- end to end through the public API, host buffers, copies inside ----
    pinned = {f: torch.from_numpy(np.ascontiguousarray(getattr(g, f))).pin_memory()
              for f in ("D", "R", "kM", "kR", "hM", "hR")}
    host = gen.ElsrInstance(*(pinned[f].numpy() for f in ("D", "R", "kM", "kR", "hM", "hR")))
    h2d = sum(int(a.numel()) * 4 for a in pinned.values())
    d2h = 80 + K * 32 + 8  # run statistics, solution bits, best cost
    e2e_moves, e2e_t = 0, 0.0
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 5))
    for i in range(e2e_steps + 1 if e2e_steps else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = elsr.Solver(host, stream=stream, lanes=args.lanes, threads=args.threads,
                         cluster=args.cluster, speculation=args.speculation)
        s2.set_count_steps(False)
        if args.workers:
            s2.vns_forkjoin_run(seed, iters, wl["kmax"], mode, args.workers)
        else:
            s2.vns_run(seed, iters, wl["kmax"], mode)
        r2 = s2.result(solution=True, traj=False)
        s2.close()
        dt = time.perf_counter() - t0
        if i > 0:  # first one is a warm-up
            e2e_t += dt
            e2e_moves += r2["moves_evaluated"]
    e2e_value = e2e_moves / e2e_t * world if e2e_t else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    clocks = clk.summary()
    peak = measure_int_peak(torch, dev, stream)
    sms = peak["sms"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": dict(wl, iters=iters, parallelism=f"replicas x{world}",
                       l2="flushed between steps (256 MiB device write, untimed)",
                       launch="one persistent launch per GVNS run"),
        "instances_per_s": world * args.steps / t_max,
        "moves_per_step": moves_per_step,
        "segments_per_step": segs_per_step,
        "eval_launch": eval_launch,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "launch_shape": solver.launch_shape(),
        "roofline": roofline_alu(
            segs_per_step, kernel_s, peak,
            traffic=(TRAFFIC_PLAIN_PER_100_ITERS * iters // 100
                     if args.instance == "medium" and not args.workers and mode == 0 else None),
            note="traffic: one-team launch of the same run under ncu, scaled by the "
                 "iterations (upper bound)"),
        "int_peak": dict(peak, unit_count_tops=sms * LANES_PER_SM *
                         (peak["clocks"].get("sm_mhz") or 0) * 1e6 / 1e12,
                         unit_count_note=f"{sms} SMs x {LANES_PER_SM} lanes x median SM "
                                         "clock, for context"),
    }
    if not args.no_cpu_baseline and world == 1 and args.instance == "medium" \
            and not args.workers and mode == 0:
        line["cpu_baseline"] = cpu_baseline(args.cpu_iters)
    if world == 1 and not args.no_workloads and args.instance == "medium" \
            and not args.workers and mode == 0 and args.iters is None:
        sub = argparse.Namespace(**vars(args))
        sub.n, sub.lanes, sub.threads, sub.cluster = 0, 0, 0, 0
        wsteps, wwarm = max(1, args.steps // 2), min(args.warmup, 3)
        line["workloads"] = {
            "batch": bench_batch(torch, dev, stream, flush, peak, wsteps, wwarm, sub),
            "multistart": bench_multistart(torch, dev, stream, flush, peak,
                                           min(args.steps, 3), wwarm, sub),
            "serve": bench_serve(torch, dev, peak, sub),
        }
        # the same stream at a load the server sustains, for its latency there
        sub_low = argparse.Namespace(**vars(sub))
        sub_low.rate = args.rate / 2
        line["workloads"]["serve_half_rate"] = bench_serve(torch, dev, peak, sub_low, cpu=False)
        b, ms_ = line["workloads"]["batch"], line["workloads"]["multistart"]
        line["workloads"]["note"] = (
            "instances/s at the workloads' own budgets: plain one run at a time "
            f"{line['instances_per_s']:.1f}/s (2000 iterations), batch "
            f"{b['instances_per_s']:.1f}/s (500), multi-start {ms_['instances_per_s']:.1f}/s "
            "(1000); moves/s compares the forms at equal work")
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_workload(args):
    """One batched workload's record as a line of its own (profiling)."""
    import torch
    from paper_1704_05132_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    peak = measure_int_peak(torch, dev, stream)
    if args.workload == "batch":
        rec = bench_batch(torch, dev, stream, flush, peak, args.steps, args.warmup, args)
    elif args.workload == "multistart":
        rec = bench_multistart(torch, dev, stream, flush, peak, args.steps, args.warmup, args)
    else:
        rec = bench_serve(torch, dev, peak, args)
    rec.update({"n_gpus": 1, "dtype": "int32", "data": "synthetic", "int_peak": peak})
    print(json.dumps(rec), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=1000)
    ap.add_argument("--ref-iters", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the batch / multi-start / serving records of the default run")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per row (0: automatic)")
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0: automatic)")
    ap.add_argument("--cluster", type=int, default=0, help="CTAs per run (0: automatic)")
    ap.add_argument("--speculation", type=int, default=0,
                    help="speculative teams for the single run (0: automatic, 1: off)")
    ap.add_argument("--instance", default="medium", choices=["medium", "paper"],
                    help="plain workload instance: K=50 x T=52 (default) or the paper-shaped "
                         "K=300 x T=52")
    ap.add_argument("--mode", default="P", choices=["P", "G"],
                    help="VND mode of the plain workload (P: Algorithm 1, G: single argmin)")
    ap.add_argument("--workers", type=int, default=0,
                    help="fork-join workers per iteration (0: the sequential GVNS)")
    ap.add_argument("--workload", default="plain",
                    choices=["plain", "batch", "multistart", "serve"])
    ap.add_argument("--rate", type=float, default=2000.0, help="serving arrivals per second")
    ap.add_argument("--requests", type=int, default=2000, help="serving requests")
    ap.add_argument("--slots", type=int, default=2048, help="serving requests in flight at most")
    ap.add_argument("--max-runs", type=int, default=1,
                    help="serving requests a team solves before it leaves its SMs")
    ap.add_argument("--n", type=int, default=0, help="instances / starts of a batched workload")
    ap.add_argument("--iters", type=int, default=None,
                    help="override the iteration budget (profiling of small cases only)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "plain":
        run_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
