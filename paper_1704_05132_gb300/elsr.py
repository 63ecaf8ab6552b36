"""Python API over the C ABI (argument marshalling only).

``Solver`` wraps one instance handle (``elsr_t``), ``Batch`` a set of
instances solved by one persistent launch (``elsr_batch_t``).  Inputs are
numpy arrays; every step of the search runs in the CUDA kernels of
``libelsr.so``.  Work is issued on a CUDA stream: by default PyTorch's current
stream when PyTorch is importable, else the legacy default stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat
from ._native import check, load

P = ctypes.c_void_p
SHAPE_KEYS = ("lanes", "threads", "cluster", "blocks", "smem", "tables_in_smem", "words",
              "teams")


# elsr_traj_t; "worker" is the fork-join winner (the C field `reserved`)
TRAJ_DTYPE = np.dtype([("it", np.int32), ("k", np.int32), ("cost", np.int64),
                       ("accepted", np.int32), ("worker", np.int32)])


def _p(a: np.ndarray):
    return a.ctypes.data_as(P)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _instance_arrays(inst):
    """The instance's arrays as contiguous int32, their shapes checked
    against one another before any pointer reaches the library (which reads
    K*T and K entries): D, R [K][T]; kM, kR, hM, hR [K]; pM, pR [K] or None."""
    D, R = _i32(inst.D), _i32(inst.R)
    if D.ndim != 2 or R.shape != D.shape:
        raise ValueError(f"D and R must be [K][T] arrays of one shape, got {D.shape}, {R.shape}")
    K = D.shape[0]
    rows = []
    for f in ("kM", "kR", "hM", "hR", "pM", "pR"):
        v = getattr(inst, f, None)
        if v is None and f in ("pM", "pR"):
            rows.append(None)
            continue
        a = _i32(v)
        if a.shape != (K,):
            raise ValueError(f"{f} must have shape ({K},), got {a.shape}")
        rows.append(a)
    return [D, R] + rows[:4], rows[4], rows[5]


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Solver:
    """One ELSR instance resident on the device (``elsr_create``)."""

    def __init__(self, inst, stream=None, lanes: int = 0, threads: int = 0,
                 cluster: int = 0, speculation: int = 0):
        arrs, pm, pr = _instance_arrays(inst)
        lib = load()
        self.K, self.T = int(arrs[0].shape[0]), int(arrs[0].shape[1])
        h = P()
        if pm is None and pr is None:
            check(lib.elsr_create(ctypes.byref(h), self.K, self.T, *[_p(a) for a in arrs]), None)
        else:  # unit production costs (Algorithm 1's p_M, p_R)
            arrs += [_i32(pm if pm is not None else np.zeros(self.K)),
                     _i32(pr if pr is not None else np.zeros(self.K))]
            check(lib.elsr_create_ex(ctypes.byref(h), self.K, self.T,
                                     *[_p(a) for a in arrs]), None)
        self._h = h
        self._lib = lib
        self.set_stream(stream)
        if lanes or threads:
            self.set_launch(lanes, threads)
        if cluster:
            self.set_cluster(cluster)
        if speculation:
            self.set_speculation(speculation)
        self._last_iters = 0
        self._base_it = 0

    # -- plumbing --
    def _chk(self, code):
        return check(code, self._h)

    def set_stream(self, stream=None):
        s = _stream_handle(stream)
        self._chk(self._lib.elsr_set_stream(self._h, P(s) if s else None))

    def set_launch(self, lanes: int = 0, threads: int = 0):
        self._chk(self._lib.elsr_set_launch(self._h, lanes, threads))

    def set_cluster(self, cluster: int = 0):
        self._chk(self._lib.elsr_set_cluster(self._h, cluster))

    def set_speculation(self, teams: int = 0):
        self._chk(self._lib.elsr_set_speculation(self._h, teams))

    def set_count_steps(self, on: bool = True):
        """Decode-step counter of the next runs (off while timing)."""
        self._chk(self._lib.elsr_set_count_steps(self._h, 1 if on else 0))

    def launch_shape(self) -> dict:
        v = np.zeros(8, np.int32)
        self._chk(self._lib.elsr_launch_shape(self._h, _p(v)))
        return dict(zip(SHAPE_KEYS, v.tolist()))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.elsr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- state --
    def set_state(self, gM=None, gR=None):
        if gM is None and gR is None:
            self._chk(self._lib.elsr_set_state(self._h, None, None))
            return
        gm, gr = _u8(gM).reshape(self.K, self.T), _u8(gR).reshape(self.K, self.T)
        self._chk(self._lib.elsr_set_state(self._h, _p(gm), _p(gr)))

    def get_state(self):
        gm = np.zeros((self.K, self.T), np.uint8)
        gr = np.zeros((self.K, self.T), np.uint8)
        self._chk(self._lib.elsr_get_state(self._h, _p(gm), _p(gr)))
        return gm, gr

    def cost(self):
        rc = np.zeros(self.K, np.int64)
        tot = np.zeros(1, np.int64)
        self._chk(self._lib.elsr_cost(self._h, _p(rc), _p(tot)))
        return int(tot[0]), rc

    # -- Algorithm 1: one neighbourhood evaluation --
    def eval_neighbourhood(self, mask: int = 0b111, mode: int = nat.MODE_P):
        """(best cost, best move, per-product costs [K], per-product moves [K]);
        the four outputs share one buffer, passed as raw addresses."""
        K = self.K
        out = np.empty(2 + 2 * K, np.int64)
        a = out.__array_interface__["data"][0]
        self._chk(self._lib.elsr_eval_neighbourhood(self._h, mask, mode, a, a + 8, a + 16,
                                                    a + 16 + 8 * K))
        return int(out[0]), int(out[1]), out[2:2 + K], out[2 + K:]

    def move_costs(self, j: int):
        n = self.K * (2 * (self.T - 1) if j == 3 else self.T)
        c = np.zeros(max(n, 1), np.int64)
        w = np.zeros(max(n, 1), np.int32)
        self._chk(self._lib.elsr_move_costs(self._h, j, _p(c), _p(w)))
        return c[:n], w[:n]

    # -- Algorithm 2: GVNS --
    def vns_run(self, seed: int, iters: int, kmax: int = 3, mode: int = nat.MODE_P):
        """Queue a GVNS run on the stream (asynchronous)."""
        self._chk(self._lib.elsr_vns_run(self._h, seed & ((1 << 64) - 1), iters, kmax, mode))
        self._last_iters = iters
        self._base_it = 0

    def vns_forkjoin_run(self, seed: int, iters: int, kmax: int = 3, mode: int = nat.MODE_P,
                         workers: int = 2):
        """Queue a fork-join GVNS run (Algorithm 2 with `workers` shakes +
        VNDs per iteration, the least result kept) on the stream."""
        self._chk(self._lib.elsr_vns_forkjoin_run(self._h, seed & ((1 << 64) - 1), iters, kmax,
                                                  mode, workers))
        self._last_iters = iters
        self._base_it = 0

    def vns_forkjoin(self, seed: int, iters: int, kmax: int = 3, mode: int = nat.MODE_P,
                     workers: int = 2, **kw):
        self.vns_forkjoin_run(seed, iters, kmax, mode, workers)
        return self.result(**kw)

    # -- checkpoint / resume and the wall-clock budget --
    def set_time_limit(self, us: int = 0):
        """Wall-clock budget of the next runs in microseconds (0: none)."""
        self._chk(self._lib.elsr_set_time_limit(self._h, int(us)))

    def checkpoint(self) -> dict:
        """Loop state of the last run (waits for it) plus its incumbent x as
        arrays "gM", "gR"; plain data (see save_checkpoint)."""
        ck = nat.Checkpoint()
        gm = np.zeros((self.K, self.T), np.uint8)
        gr = np.zeros((self.K, self.T), np.uint8)
        code = self._lib.elsr_checkpoint(self._h, ctypes.byref(ck), _p(gm), _p(gr))
        if code not in (nat.ELSR_E_CAP, nat.ELSR_E_TIMEOUT, nat.ELSR_E_STATE):
            self._chk(code)
        d = ck.as_dict()
        d["gM"], d["gR"] = gm, gr
        return d

    def vns_resume_run(self, ck: dict, iters: int):
        """Queue iterations ck["next_it"] .. + iters - 1 of a checkpointed run."""
        c = nat.Checkpoint.from_dict(ck)
        gm, gr = _u8(ck["gM"]).reshape(self.K, self.T), _u8(ck["gR"]).reshape(self.K, self.T)
        self._chk(self._lib.elsr_vns_resume(self._h, ctypes.byref(c), _p(gm), _p(gr), iters))
        self._last_iters = iters
        self._base_it = int(ck["next_it"])

    def vns_resume(self, ck: dict, iters: int, **kw):
        self.vns_resume_run(ck, iters)
        return self.result(**kw)

    def result(self, solution: bool = True, plan: bool = False, traj: bool = True):
        st = nat.Stats()
        st.status = 1  # stays 1 unless the library fills the statistics
        gm = np.zeros((self.K, self.T), np.uint8) if solution else None
        gr = np.zeros((self.K, self.T), np.uint8) if solution else None
        pl = np.zeros((4, self.K, self.T), np.int32) if plan else None
        n = self._last_iters if traj else 0
        tr = np.zeros(max(n, 1), TRAJ_DTYPE)
        code = self._lib.elsr_result(self._h, ctypes.byref(st),
                                     _p(gm) if solution else None,
                                     _p(gr) if solution else None,
                                     _p(pl) if plan else None,
                                     _p(tr) if n else None, n)
        # a run that ended with a status (cap, timeout, mismatched resume)
        # still reports its statistics
        if not (code in (nat.ELSR_E_CAP, nat.ELSR_E_TIMEOUT, nat.ELSR_E_STATE)
                and st.status == code):
            self._chk(code)
        out = st.as_dict()
        if solution:
            out["gM"], out["gR"] = gm, gr
        if plan:
            out["plan"] = pl
        if n:
            ran = out["iterations"] - self._base_it  # entries this run wrote
            out["traj"] = tr[:max(0, min(n, ran))].copy()
        return out

    def vns(self, seed: int, iters: int, kmax: int = 3, mode: int = nat.MODE_P, **kw):
        self.vns_run(seed, iters, kmax, mode)
        return self.result(**kw)

    def multistart(self, seed0: int, nstarts: int, iters: int, kmax: int = 3,
                   mode: int = nat.MODE_P, costs: bool = False):
        bc = np.zeros(1, np.int64)
        bs = np.zeros(1, np.int32)
        cs = np.zeros(nstarts, np.int64) if costs else None
        self._chk(self._lib.elsr_multistart_run(self._h, seed0, nstarts, iters, kmax, mode,
                                                _p(bc), _p(bs), _p(cs) if costs else None))
        self._last_iters = 0
        self._base_it = 0
        return int(bc[0]), int(bs[0]), cs

    def multistart_stats(self, n: int):
        st = (nat.Stats * max(n, 1))()
        self._chk(self._lib.elsr_multistart_stats(self._h, st, n))
        return [s.as_dict() for s in st[:n]]

    def moves_evaluated(self) -> int:
        v = np.zeros(1, np.int64)
        self._chk(self._lib.elsr_counters(self._h, _p(v)))
        return int(v[0])


def save_checkpoint(path: str, ck: dict) -> None:
    """Store a checkpoint (loop state and incumbent) in an .npz file."""
    np.savez(path, **{k: np.asarray(v) for k, v in ck.items()})


def load_checkpoint(path: str) -> dict:
    with np.load(path) as z:
        return {k: (z[k] if z[k].ndim else int(z[k])) for k in z.files}


class Batch:
    """Many instances of uneven size solved by one persistent launch."""

    def __init__(self, insts, stream=None, lanes: int = 0, threads: int = 0,
                 cluster: int = 0, runs_per_cta: int = 0):
        insts = list(insts)
        if not insts:
            raise ValueError("a batch needs at least one instance")
        for i in insts:
            _instance_arrays(i)
        lib = load()
        self._lib = lib
        self.n = len(insts)
        self.Ks = np.array([i.D.shape[0] for i in insts], np.int32)
        self.Ts = np.array([i.D.shape[1] for i in insts], np.int32)
        cat = lambda f: _i32(np.concatenate([np.ravel(getattr(i, f)) for i in insts]))
        arrs = [cat("D"), cat("R"), cat("kM"), cat("kR"), cat("hM"), cat("hR")]
        if not (lanes or threads or cluster or runs_per_cta):
            from . import autotune  # a tuned shape for this signature, when cached
            hit = autotune.lookup_batch(insts)
            if hit:
                lanes, threads = hit.get("lanes", 0), hit.get("threads", 0)
                cluster, runs_per_cta = hit.get("cluster", 0), hit.get("runs_per_cta", 0)
        b = P()
        sh = _stream_handle(stream)
        if any(getattr(i, "pM", None) is not None or getattr(i, "pR", None) is not None
               for i in insts):
            pc = lambda f: _i32(np.concatenate([
                np.ravel(getattr(i, f)) if getattr(i, f, None) is not None
                else np.zeros(i.D.shape[0]) for i in insts]))
            arrs += [pc("pM"), pc("pR")]
            code = lib.elsr_batch_create_ex(ctypes.byref(b), self.n, _p(self.Ks), _p(self.Ts),
                                            *[_p(a) for a in arrs], P(sh) if sh else None)
        else:
            code = lib.elsr_batch_create_on(ctypes.byref(b), self.n, _p(self.Ks), _p(self.Ts),
                                            *[_p(a) for a in arrs], P(sh) if sh else None)
        check(code, None, batch=True)
        self._b = b
        if lanes or threads:
            self.set_launch(lanes, threads)
        if cluster:
            self._chk(self._lib.elsr_batch_set_cluster(self._b, cluster))
        if runs_per_cta:
            self.set_runs_per_cta(runs_per_cta)

    def _chk(self, code):
        return check(code, self._b, batch=True)

    def launch_shape(self) -> dict:
        v = np.zeros(8, np.int32)
        self._chk(self._lib.elsr_batch_launch_shape(self._b, _p(v)))
        out = dict(zip(SHAPE_KEYS, v.tolist()))
        pk = np.zeros(2, np.int32)
        self._chk(self._lib.elsr_batch_packing(self._b, _p(pk[:1]), _p(pk[1:])))
        out["runs_per_cta"], out["whole_cta_runs"] = int(pk[0]), int(pk[1])
        return out

    def set_count_steps(self, on: bool = True):
        """Decode-step counter of the next runs (off while timing)."""
        self._chk(self._lib.elsr_batch_set_count_steps(self._b, 1 if on else 0))

    def stage_tables(self):
        """(Re)build every row's prefix tables in device memory, on the
        batch's stream (asynchronous)."""
        self._chk(self._lib.elsr_batch_stage_tables(self._b))

    def set_runs_per_cta(self, runs_per_cta: int = 0):
        """Instances per CTA (0: the library's choice)."""
        self._chk(self._lib.elsr_batch_set_runs_per_cta(self._b, runs_per_cta))

    def set_stream(self, stream=None):
        s = _stream_handle(stream)
        self._chk(self._lib.elsr_batch_set_stream(self._b, P(s) if s else None))

    def set_launch(self, lanes: int = 0, threads: int = 0):
        self._chk(self._lib.elsr_batch_set_launch(self._b, lanes, threads))

    def run(self, seeds, iters: int, kmax: int = 3, mode: int = nat.MODE_P):
        s = np.ascontiguousarray(seeds, dtype=np.uint64)
        if s.shape != (self.n,):
            raise ValueError(f"one seed per instance: expected shape ({self.n},), got {s.shape}")
        self._seeds = s
        self._chk(self._lib.elsr_batch_run(self._b, _p(s), iters, kmax, mode))

    def results(self):
        st = (nat.Stats * self.n)()
        code = self._lib.elsr_batch_results(self._b, st)
        if code != nat.ELSR_E_CAP:
            self._chk(code)
        return [s.as_dict() for s in st]

    def solution(self, i: int):
        K, T = int(self.Ks[i]), int(self.Ts[i])
        gm = np.zeros((K, T), np.uint8)
        gr = np.zeros((K, T), np.uint8)
        self._chk(self._lib.elsr_batch_solution(self._b, i, _p(gm), _p(gr)))
        return gm, gr

    def close(self):
        if getattr(self, "_b", None):
            self._lib.elsr_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
