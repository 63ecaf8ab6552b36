"""Autotuner for the persistent GVNS launch shape.

Knobs (none changes a result; only speed):
  lanes    -- lanes that share one product row (4..32 within a warp; 64 or
              128 = a row group of 2 or 4 warps; 0 = automatic, which lets
              each run of a batch pick its own): each lane evaluates
              about |row moves| / lanes candidates per sweep;
  threads  -- threads per CTA (rows in flight per CTA = threads / lanes);
  cluster  -- CTAs that share one run (1 for batches of small instances;
              larger clusters split a big instance's rows over several SMs);
  runs_per_cta -- instances per CTA of a batch (1, 2 or 4): small runs
              share a CTA, each in a partition of its threads;
  teams    -- speculative teams for a single run (0: as many as are
              resident, up to 16).
A probe runs each candidate for a few iterations of the real workload and
times it with CUDA events; the best moves/s wins.  Choices are cached per
workload signature (bucketed K, T and batch size) in memory and, optionally,
in a JSON file (``cache_file``, or the file named by ELSR_AUTOTUNE_CACHE).
A Batch created with every knob left at 0 takes the cached choice for its
signature when there is one (``lookup_batch``), without probing.
"""
from __future__ import annotations

import json
import os

import numpy as np

from .elsr import Batch, Solver

_cache: dict = {}


def _bucket(x: int) -> int:
    return 1 << max(0, int(x - 1).bit_length())


def signature(insts, kind: str) -> str:
    K = max(int(i.D.shape[0]) for i in insts)
    T = max(int(i.D.shape[1]) for i in insts)
    return f"{kind}:K{_bucket(K)}:T{_bucket(T)}:n{_bucket(len(insts))}"


def _timed(fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out


# lanes = 0: every run of the batch picks its own row-group width
BATCH_CANDIDATES = [dict(lanes=l, threads=t, cluster=1, runs_per_cta=p) for l in (0, 8, 16)
                    for t in (512, 1024) for p in (1, 2, 4)]
SINGLE_CANDIDATES = [dict(lanes=l, cluster=c, teams=0) for l in (32, 64)
                     for c in (6, 8, 9, 10, 12, 16)]


def tune_batch(insts, probe_iters: int = 10, candidates=None, cache_file: str | None = None):
    """Best launch shape for a batch of instances (dict lanes/threads/cluster)."""
    key = signature(insts, "batch")
    hit = _lookup(key, cache_file)
    if hit:
        return hit
    seeds = np.arange(len(insts), dtype=np.uint64)
    best, best_rate, err = None, -1.0, None
    for cand in candidates or BATCH_CANDIDATES:
        b = None
        try:
            b = Batch(insts, lanes=cand["lanes"], threads=cand["threads"],
                      cluster=cand["cluster"], runs_per_cta=cand.get("runs_per_cta", 0))
            b.run(seeds, 1, 3, 0)  # warm-up (kernel attributes, first touch)
            b.results()
            ms, _ = _timed(lambda: b.run(seeds, probe_iters, 3, 0))
            rate = sum(r["moves_evaluated"] for r in b.results()) / ms
        except Exception as e:  # a shape this device or batch cannot run
            rate, err = -1.0, e
        finally:
            if b is not None:
                b.close()
        if rate > best_rate:
            best, best_rate = dict(cand), rate
    return _chosen(key, best, err, cache_file)


def tune_single(inst, probe_iters: int = 100, candidates=None, cache_file: str | None = None):
    """Best launch shape for one GVNS run (dict lanes/cluster/teams)."""
    key = signature([inst], "single")
    hit = _lookup(key, cache_file)
    if hit:
        return hit
    best, best_rate, err = None, -1.0, None
    for cand in candidates or SINGLE_CANDIDATES:
        s = None
        try:
            s = Solver(inst, lanes=cand["lanes"], cluster=cand["cluster"],
                       speculation=cand["teams"])
            s.vns(0, 2, 3, 0, traj=False, solution=False)
            ms, _ = _timed(lambda: s.vns_run(0, probe_iters, 3, 0))
            rate = s.result(traj=False, solution=False)["moves_evaluated"] / ms
        except Exception as e:  # a shape this device or instance cannot run
            rate, err = -1.0, e
        finally:
            if s is not None:
                s.close()
        if rate > best_rate:
            best, best_rate = dict(cand), rate
    return _chosen(key, best, err, cache_file)


def _chosen(key, best, err, cache_file):
    """Cache and return the winning shape; no shape that ran is an error."""
    if best is None:
        raise RuntimeError(f"autotune: no candidate launch shape ran for {key}") from err
    _store(key, best, cache_file)
    return best


def lookup_batch(insts, cache_file: str | None = None):
    """The cached launch shape for this batch's signature, or None (no
    probing)."""
    return _lookup(signature(insts, "batch"), cache_file)


def _lookup(key, cache_file):
    cache_file = cache_file or os.environ.get("ELSR_AUTOTUNE_CACHE")
    if key in _cache:
        return _cache[key]
    if cache_file and os.path.exists(cache_file):
        with open(cache_file) as f:
            disk = json.load(f)
        if key in disk:
            _cache[key] = disk[key]
            return disk[key]
    return None


def _store(key, value, cache_file):
    cache_file = cache_file or os.environ.get("ELSR_AUTOTUNE_CACHE")
    _cache[key] = value
    if cache_file:
        disk = {}
        if os.path.exists(cache_file):
            with open(cache_file) as f:
                disk = json.load(f)
        disk[key] = value
        tmp = cache_file + ".tmp"
        with open(tmp, "w") as f:
            json.dump(disk, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_file)
