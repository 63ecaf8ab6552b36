"""Continuous-batching server for GVNS solves of independent instances.

Requests (an instance, a seed, an iteration budget) arrive over time.  The
server keeps a pool of CUDA streams ("slots").  Whenever a slot is free, every
waiting request that fits the device-memory budget is admitted (first come,
first served) and solved by one persistent batched launch on that slot; while
it runs, new arrivals queue up and are admitted by the next free slot, so the
work of several batches overlaps on the device.  Requests whose rows do not
fit one CTA's shared memory are launched separately (they use CTA clusters),
so they do not force clusters on small instances.  A batch's device memory
(instance data, tables, solutions) is held from admission until its results
are read, and admission never lets the resident bytes exceed the budget.

Every request's result depends only on its instance, seed and budget, so it
is the same whether it is solved alone or in any mix (tested).

Latency of a request = completion time - arrival time, on the host clock.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

from . import _native as nat
from .elsr import Batch

SMEM_ONE_CTA = 227 * 1024 - 1024  # dynamic shared bytes per CTA (static control words < 1 KB)


@dataclass
class Request:
    rid: int
    inst: object          # ElsrInstance (D, R, kM, kR, hM, hR)
    seed: int
    iters: int
    arrival: float = 0.0  # seconds after the start of the stream


@dataclass
class Result:
    rid: int
    best_cost: int
    traj_hash: int
    moves_evaluated: int
    status: int
    arrival: float
    admitted: float
    done: float
    batch: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    batches: int = 0
    max_resident_bytes: int = 0
    wall_s: float = 0.0

    def summary(self) -> dict:
        if not self.results:  # an empty request stream
            return {"requests": 0, "batches": self.batches, "p50_ms": None, "p99_ms": None,
                    "mean_ms": None, "instances_per_s": 0.0, "moves_per_s": 0.0,
                    "max_resident_bytes": self.max_resident_bytes, "span_s": 0.0}
        lat = np.array([r.latency for r in self.results]) * 1e3
        moves = sum(r.moves_evaluated for r in self.results)
        first = min(r.arrival for r in self.results)
        last = max(r.done for r in self.results)
        span = max(last - first, 1e-9)
        return {"requests": len(self.results), "batches": self.batches,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "instances_per_s": len(self.results) / span,
                "moves_per_s": moves / span, "max_resident_bytes": self.max_resident_bytes,
                "span_s": span}


def footprint(K: int, T: int):
    """(shared bytes per CTA at one CTA per run, device bytes while resident)."""
    lib = nat.load()
    sm = ctypes.c_int32()
    dv = ctypes.c_int64()
    nat.check(lib.elsr_run_footprint(K, T, ctypes.byref(sm), ctypes.byref(dv)))
    return int(sm.value), int(dv.value)


class Server:
    """Serve requests with `slots` concurrent batches under a device-memory
    budget of `mem_budget` bytes."""

    def __init__(self, slots: int = 4, mem_budget: int = 256 << 20, max_batch: int = 4096,
                 kmax: int = 3, mode: int = nat.MODE_P):
        import torch
        self.torch = torch
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.mem_budget = mem_budget
        self.max_batch = max_batch
        self.kmax = kmax
        self.mode = mode

    def _launch(self, reqs, stream, now):
        insts = [r.inst for r in reqs]
        b = Batch(insts, stream=stream)
        seeds = np.array([r.seed for r in reqs], dtype=np.uint64)
        iters = reqs[0].iters
        b.run(seeds, iters, self.kmax, self.mode)
        ev = self.torch.cuda.Event()
        ev.record(stream)
        return b, ev

    def run(self, requests, realtime: bool = True) -> ServeStats:
        """Serve `requests` (arrival times relative to now when realtime, else
        all available at once).  Requests of one batch share an iteration
        budget, so batches are formed per budget.  On an error every slot is
        drained before the error propagates (no work is left in flight)."""
        try:
            return self._run(requests, realtime)
        finally:
            for s in self.streams:
                s.synchronize()

    def _run(self, requests, realtime: bool) -> ServeStats:
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting = collections.deque()
        inflight = {}  # slot -> (list of (Batch, event, reqs)), admitted time, bytes
        free = list(range(len(self.streams)))
        resident = 0
        stats = ServeStats()
        sizes = {}
        for r in pending:  # a request that can never be admitted is refused up front
            key = (r.inst.K, r.inst.T)
            if key not in sizes:
                sizes[key] = footprint(*key)
            if sizes[key][1] > self.mem_budget:
                raise ValueError(f"request {r.rid} (K={key[0]}, T={key[1]}) needs "
                                 f"{sizes[key][1]} device bytes, more than the budget of "
                                 f"{self.mem_budget}")
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: float("inf"))
        while pending or waiting or inflight:
            now = clock()
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # completions
            for slot in list(inflight):
                parts, admitted, nbytes = inflight[slot]
                if all(ev.query() for _, ev, _ in parts):
                    done = time.perf_counter() - t0
                    for b, _, reqs in parts:
                        for r, st in zip(reqs, b.results()):
                            stats.results.append(Result(
                                r.rid, st["best_cost"], st["traj_hash"], st["moves_evaluated"],
                                st["status"], r.arrival if realtime else 0.0, admitted, done,
                                stats.batches))
                        b.close()
                    resident -= nbytes
                    del inflight[slot]
                    free.append(slot)
            # admissions
            while free and waiting:
                iters = waiting[0].iters
                take, nbytes = [], 0
                for r in list(waiting):
                    if r.iters != iters or len(take) >= self.max_batch:
                        continue
                    fb = sizes[(r.inst.K, r.inst.T)][1]
                    if resident + nbytes + fb > self.mem_budget:
                        break
                    take.append(r)
                    nbytes += fb
                if not take:
                    break
                for r in take:
                    waiting.remove(r)
                slot = free.pop()
                stream = self.streams[slot]
                small = [r for r in take if sizes[(r.inst.K, r.inst.T)][0] <= SMEM_ONE_CTA]
                large = [r for r in take if sizes[(r.inst.K, r.inst.T)][0] > SMEM_ONE_CTA]
                parts = []
                with torch.cuda.stream(stream):
                    for grp in (small, large):
                        if grp:
                            b, ev = self._launch(grp, stream, now)
                            parts.append((b, ev, grp))
                resident += nbytes
                stats.max_resident_bytes = max(stats.max_resident_bytes, resident)
                inflight[slot] = (parts, time.perf_counter() - t0, nbytes)
                stats.batches += 1
            if not (free and waiting):
                nxt = pending[0].arrival - clock() if pending else 0.0
                time.sleep(min(max(nxt, 0.0), 2e-4) if nxt > 0 or inflight else 0.0)
        stats.wall_s = time.perf_counter() - t0
        return stats


def poisson_requests(n: int, rate: float, iters: int, seed: int = 5, id0: int = 0,
                     arrival_seed: int = 12345):
    """n requests of the serving workload: instance (seed, id) with K ~ U{5..200},
    T ~ U{12..104}, VNS seed = request id, exponential inter-arrival gaps of
    mean 1/rate drawn on the harness side."""
    from .gen import serving_request
    rng = np.random.default_rng(arrival_seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    return [Request(id0 + i, serving_request(id0 + i, seed), id0 + i, iters, float(t[i]))
            for i in range(n)]
