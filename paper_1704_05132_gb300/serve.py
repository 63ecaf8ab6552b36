"""Serving GVNS requests with continuous batching.

Requests (an instance, a seed, an iteration budget) arrive over time.  Each
is submitted to the library's server (``elsr_server_*`` in the C ABI) as soon
as it has arrived and fits: the server admits a request by its footprint in
fixed-size device pools (a slot, K*T cells, K rows) and answers "busy" when
they are full, in which case the request waits, in arrival order, for
completions to free room.  On the device a submitted request joins the
kernels already running: a team that finishes a request takes the next one
queued for its size class, so requests of different sizes and arrival times
are solved side by side, and each one retires on its own as soon as its run
ends (its statistics land in host memory that the loop polls without
synchronising any stream).

Every request's result depends only on its instance, seed and budget, so it
is the same whether it is served alone or in any mix (tested).

Latency of a request = completion time - arrival time, on the host clock.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

from . import _native as nat


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
    batch: int = 0        # kernel launches issued before it retired

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    batches: int = 0            # kernel launches of the server
    max_resident_bytes: int = 0
    max_inflight: int = 0
    wall_s: float = 0.0

    def summary(self) -> dict:
        if not self.results:  # an empty request stream
            return {"requests": 0, "batches": self.batches, "p50_ms": None, "p99_ms": None,
                    "mean_ms": None, "instances_per_s": 0.0, "moves_per_s": 0.0,
                    "max_resident_bytes": self.max_resident_bytes,
                    "max_inflight": self.max_inflight, "span_s": 0.0}
        lat = np.array([r.latency for r in self.results]) * 1e3
        moves = sum(r.moves_evaluated for r in self.results)
        first = min(r.arrival for r in self.results)
        last = max(r.done for r in self.results)
        span = max(last - first, 1e-9)
        return {"requests": len(self.results), "batches": self.batches,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "instances_per_s": len(self.results) / span,
                "moves_per_s": moves / span, "max_resident_bytes": self.max_resident_bytes,
                "max_inflight": self.max_inflight, "span_s": span}


def footprint(K: int, T: int) -> int:
    """Device bytes a request holds in the server's pools while in flight:
    D and R (K*T int32 each) and four int32 costs per product."""
    return 8 * K * T + 16 * K


class NativeServer:
    """The C ABI's server (argument marshalling only)."""

    def __init__(self, slots: int = 0, cells: int = 0, rows: int = 0, threads: int = 0,
                 max_runs: int = 0, acc64: bool = False, count_steps: bool = False,
                 keep_solutions: bool = False):
        self._lib = nat.load()
        cfg = nat.ServerConfig(slots, threads, cells, rows, max_runs, int(acc64),
                               int(count_steps), int(keep_solutions))
        h = ctypes.c_void_p()
        nat.check(self._lib.elsr_server_create(ctypes.byref(h), ctypes.byref(cfg)))
        self._h = h
        self.slots = slots or 2048
        self.cells = cells or (8 << 20)
        self.rows = rows or (512 << 10)
        self._tk = np.zeros(1, np.int64)

    def _chk(self, code):
        return nat.check(code, self._h, server=True)

    def submit(self, inst, seed: int, iters: int, kmax: int = 3, mode: int = nat.MODE_P):
        """Ticket of the request, or None when the server is full now."""
        arr = [np.ascontiguousarray(getattr(inst, f), dtype=np.int32)
               for f in ("D", "R", "kM", "kR", "hM", "hR")]
        K, T = arr[0].shape
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        code = self._lib.elsr_server_submit(self._h, K, T, *[p(a) for a in arr],
                                            seed & ((1 << 64) - 1), iters, kmax, mode,
                                            self._tk.ctypes.data_as(ctypes.c_void_p))
        if code == nat.ELSR_E_BUSY:
            return None
        self._chk(code)
        return int(self._tk[0])

    def poll(self, max_n: int = 1024):
        """[(ticket, stats dict)] of requests retired since the last poll."""
        tk = np.zeros(max_n, np.int64)
        st = (nat.Stats * max_n)()
        n = self._chk(self._lib.elsr_server_poll(self._h, max_n,
                                                 tk.ctypes.data_as(ctypes.c_void_p), st))
        return [(int(tk[i]), st[i].as_dict()) for i in range(n)]

    def solution(self, ticket: int, K: int, T: int):
        gm = np.zeros((K, T), np.uint8)
        gr = np.zeros((K, T), np.uint8)
        self._chk(self._lib.elsr_server_solution(self._h, ticket,
                                                 gm.ctypes.data_as(ctypes.c_void_p),
                                                 gr.ctypes.data_as(ctypes.c_void_p)))
        return gm, gr

    def release(self, ticket: int):
        self._chk(self._lib.elsr_server_release(self._h, ticket))

    def info(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._chk(self._lib.elsr_server_info(self._h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.elsr_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over the library's device queues.

    slots / cells / rows size the device pools (requests in flight, demand
    and return values, product rows); a request is admitted when its
    footprint fits and waits otherwise."""

    def __init__(self, slots: int = 2048, cells: int = 8 << 20, rows: int = 512 << 10,
                 max_runs: int = 1, kmax: int = 3, mode: int = nat.MODE_P,
                 acc64: bool = False, native=None):
        self.slots, self.cells, self.rows = slots, cells, rows
        self.max_runs = max_runs
        self.kmax = kmax
        self.mode = mode
        self.acc64 = acc64
        self._native = native  # a stand-in for NativeServer (tests)

    def _make(self):
        if self._native is not None:
            return self._native(self.slots, self.cells, self.rows)
        return NativeServer(self.slots, self.cells, self.rows, max_runs=self.max_runs,
                            acc64=self.acc64)

    def run(self, requests, realtime: bool = True) -> ServeStats:
        """Serve `requests` (arrival times relative to now when realtime, else
        all available at once) and return per-request results."""
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        for r in pending:  # a request that can never be admitted is refused up front
            K, T = r.inst.D.shape
            if K * T > self.cells or K > self.rows:
                raise ValueError(f"request {r.rid} (K={K}, T={T}) needs {footprint(K, T)} "
                                 f"pool bytes, more than the server's pools hold")
        stats = ServeStats()
        if not pending:
            return stats
        srv = self._make()
        try:
            return self._serve(srv, pending, realtime, stats)
        finally:
            srv.close()

    # a request that has not retired this long after its admission is an error
    RETIRE_LIMIT_S = 120.0

    def _serve(self, srv, pending, realtime, stats):
        waiting = collections.deque()
        inflight = {}  # ticket -> (request, admitted, bytes)
        resident = 0
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: float("inf"))
        while pending or waiting or inflight:
            now = clock()
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            progressed = False
            # admissions, in arrival order: stop at the first that does not fit
            while waiting:
                r = waiting[0]
                tk = srv.submit(r.inst, r.seed, r.iters, self.kmax, self.mode)
                if tk is None:
                    break
                waiting.popleft()
                K, T = r.inst.D.shape
                nb = footprint(K, T)
                inflight[tk] = (r, time.perf_counter() - t0, nb)
                resident += nb
                stats.max_resident_bytes = max(stats.max_resident_bytes, resident)
                stats.max_inflight = max(stats.max_inflight, len(inflight))
                progressed = True
            # retirements
            done = srv.poll(1024)
            if done:
                t_done = time.perf_counter() - t0
                launches = srv.info()[1]
                for tk, st in done:
                    r, admitted, nb = inflight.pop(tk)
                    resident -= nb
                    stats.results.append(Result(
                        r.rid, st["best_cost"], st["traj_hash"], st["moves_evaluated"],
                        st["status"], r.arrival if realtime else 0.0, admitted, t_done,
                        launches))
                progressed = True
            if not progressed:
                if inflight:
                    oldest = min(a for _, a, _ in inflight.values())
                    if time.perf_counter() - t0 - oldest > self.RETIRE_LIMIT_S:
                        raise RuntimeError(f"{len(inflight)} requests have not retired "
                                           f"{self.RETIRE_LIMIT_S:.0f} s after admission")
                nxt = pending[0].arrival - clock() if pending and not waiting else 0.0
                time.sleep(min(max(nxt, 0.0), 1e-4) if nxt > 0 else 2e-5)
        stats.batches = srv.info()[1]
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
