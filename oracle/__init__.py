"""CPU oracle for the ELSR variable neighbourhood search (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library never loads it, and it shares no code with the CUDA path.

The arithmetic lives in ``elsr_oracle.c`` (plain single-threaded C, one full
per-period decode per candidate move).  This module compiles it with gcc and
exposes thin ctypes wrappers.  Each wrapper names the passage of Antoniadis &
Sifaleras (2017) that the C function follows:

* ``decode_row`` / ``total_cost``    -- Section 2 objective and the decode reading
* ``move_costs`` / ``eval_neighbourhood`` -- Algorithm 1, best-neighbour search
* ``vnd``                            -- Algorithm 1 (pipe VND)
* ``shake`` / ``draw``               -- Algorithm 2, Shake(x, k)
* ``vns`` / ``multistart``           -- Algorithm 2 (GVNS) and the best-of of Section 3
* ``shake_worker`` / ``vns_forkjoin`` -- Algorithm 2 as the paper runs it: P
  workers shake and descend from the same x, the minimum is kept (Section 3)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "elsr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
# ELSR_ORACLE_SANITIZE=1 (set by tests/test_host_sanitized.py) builds and
# loads a separate copy under AddressSanitizer and UBSan.
_SANITIZE = os.environ.get("ELSR_ORACLE_SANITIZE") == "1"
_LIB_PATH = os.path.join(_BUILD, "libelsr_oracle_san.so" if _SANITIZE else "libelsr_oracle.so")
_lock = threading.Lock()
_lib = None

INF = np.iinfo(np.int64).max


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libelsr_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    opt = (["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
            "-fno-sanitize-recover=all"] if _SANITIZE else ["-O2"])
    subprocess.check_call(["gcc"] + opt + ["-std=c11", "-shared", "-fPIC",
                           "-Wall", "-Wextra", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Instance(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("T", ctypes.c_int32),
                ("D", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("kM", ctypes.c_void_p), ("kR", ctypes.c_void_p),
                ("hM", ctypes.c_void_p), ("hR", ctypes.c_void_p),
                ("pM", ctypes.c_void_p), ("pR", ctypes.c_void_p)]


class _Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("moves_evaluated", "evals", "vnd_cycles", "applied",
                 "iterations", "accepted")]


TRAJ_DTYPE = np.dtype([("it", np.int32), ("k", np.int32), ("cost", np.int64),
                       ("accepted", np.int32), ("pad", np.int32)])


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, u32, u64 = (ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_uint32, ctypes.c_uint64)
            sig = {
                "orc_decode_row": (i64, [P, i32, P, P, P]),
                "orc_total_cost": (i64, [P, P, P, P]),
                "orc_nb_size": (i64, [i32, i32, i32]),
                "orc_row_moves": (i64, [i32, i32]),
                "orc_apply_row_move": (None, [i32, i32, i64, P, P]),
                "orc_apply_move": (None, [i32, i32, i32, i64, P, P]),
                "orc_move_costs": (None, [P, P, P, i32, P]),
                "orc_eval_neighbourhood": (i64, [P, P, P, u32, i32, P, P, P, P]),
                "orc_vnd": (i32, [P, P, P, i32, P]),
                "orc_splitmix64": (u64, [u64]),
                "orc_draw": (u64, [u64, u64, u64, u64]),
                "orc_shake": (None, [i32, i32, P, P, u64, i64, i32]),
                "orc_vns": (i32, [P, P, P, u64, i32, i32, i32, P, P, P, P]),
                "orc_shake_worker": (None, [i32, i32, P, P, u64, i64, i32, i32]),
                "orc_vns_forkjoin": (i32, [P, P, P, u64, i32, i32, i32, i32, P, P, P, P]),
                "orc_initial_solution": (None, [i32, i32, P, P]),
                "orc_decode_steps": (i64, [P, i32, P, P, i32, i64]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Instance:
    """Problem data of Section 2: D, R int32 [K][T]; kM, kR, hM, hR int32 [K];
    optional unit production costs pM, pR int32 [K] (Algorithm 1's p_M, p_R;
    None = 0)."""
    D: np.ndarray
    R: np.ndarray
    kM: np.ndarray
    kR: np.ndarray
    hM: np.ndarray
    hR: np.ndarray
    pM: np.ndarray | None = None
    pR: np.ndarray | None = None

    def __post_init__(self):
        fields = ["D", "R", "kM", "kR", "hM", "hR"]
        fields += [f for f in ("pM", "pR") if getattr(self, f) is not None]
        for f in fields:
            setattr(self, f, np.ascontiguousarray(getattr(self, f), dtype=np.int32))
        if self.D.ndim != 2 or self.D.shape != self.R.shape:
            raise ValueError("D and R must be [K][T]")
        K = self.D.shape[0]
        for f in fields[2:]:
            if getattr(self, f).shape != (K,):
                raise ValueError(f"{f} must have shape [K]")
        ptr = lambda a: a.ctypes.data if a is not None else None
        self._c = _Instance(self.K, self.T, self.D.ctypes.data, self.R.ctypes.data,
                            self.kM.ctypes.data, self.kR.ctypes.data,
                            self.hM.ctypes.data, self.hR.ctypes.data,
                            ptr(self.pM), ptr(self.pR))

    @property
    def K(self) -> int:
        return int(self.D.shape[0])

    @property
    def T(self) -> int:
        return int(self.D.shape[1])

    @classmethod
    def from_arrays(cls, arrs) -> "Instance":
        """From any object with D, R, kM, kR, hM, hR (and optionally pM, pR)
        attributes."""
        return cls(arrs.D, arrs.R, arrs.kM, arrs.kR, arrs.hM, arrs.hR,
                   getattr(arrs, "pM", None), getattr(arrs, "pR", None))

    def row(self, k: int) -> "Instance":
        """The single-product instance made of product k alone."""
        s = slice(k, k + 1)
        sub = lambda a: a[s] if a is not None else None
        return Instance(self.D[s], self.R[s], self.kM[s], self.kR[s],
                        self.hM[s], self.hR[s], sub(self.pM), sub(self.pR))

    @property
    def cref(self):
        return ctypes.byref(self._c)


def _bits(g, K, T):
    a = np.ascontiguousarray(g, dtype=np.uint8).reshape(K, T)
    if a.size and a.max() > 1:
        raise ValueError("setup bits must be 0/1")
    return a


def initial_solution(K: int, T: int):
    """All setups open (reading of the omitted initialisation method)."""
    return np.ones((K, T), np.uint8), np.ones((K, T), np.uint8)


def decode_row(inst: Instance, k: int, gM_row, gR_row):
    """Section 2 / decode reading: (cost, plan[4][T] = xM, xR, yM, yR)."""
    lib = _load()
    gm = _bits(gM_row, 1, inst.T)
    gr = _bits(gR_row, 1, inst.T)
    plan = np.zeros((4, inst.T), np.int64)
    c = lib.orc_decode_row(inst.cref, k, _ptr(gm), _ptr(gr), _ptr(plan))
    return int(c), plan


def total_cost(inst: Instance, gM, gR):
    """Section 2 objective: (total, rowcost[K]); INF marks infeasibility."""
    lib = _load()
    gm, gr = _bits(gM, inst.K, inst.T), _bits(gR, inst.K, inst.T)
    rc = np.zeros(inst.K, np.int64)
    t = lib.orc_total_cost(inst.cref, _ptr(gm), _ptr(gr), _ptr(rc))
    return int(t), rc


def nb_size(K: int, T: int, j: int) -> int:
    return int(_load().orc_nb_size(K, T, j))


def row_moves(T: int, j: int) -> int:
    return int(_load().orc_row_moves(T, j))


def apply_move(K, T, j, m, gM, gR):
    """Apply global move m of N_j in place (arrays [K][T] uint8)."""
    _load().orc_apply_move(K, T, j, int(m), _ptr(gM), _ptr(gR))


def move_costs(inst: Instance, gM, gR, j: int) -> np.ndarray:
    """New cost of the moved row for every move of N_j (global layout)."""
    lib = _load()
    gm, gr = _bits(gM, inst.K, inst.T), _bits(gR, inst.K, inst.T)
    out = np.zeros(nb_size(inst.K, inst.T, j), np.int64)
    lib.orc_move_costs(inst.cref, _ptr(gm), _ptr(gr), j, _ptr(out))
    return out


def eval_neighbourhood(inst: Instance, gM, gR, mask: int, mode: int):
    """Algorithm 1's best-neighbour search without applying anything.

    Returns (best_cost, best_move, pp_cost[K], pp_move[K], moves_evaluated)."""
    lib = _load()
    gm, gr = _bits(gM, inst.K, inst.T), _bits(gR, inst.K, inst.T)
    bc = np.zeros(1, np.int64)
    bm = np.zeros(1, np.int64)
    pc = np.zeros(inst.K, np.int64)
    pm = np.zeros(inst.K, np.int64)
    n = lib.orc_eval_neighbourhood(inst.cref, _ptr(gm), _ptr(gr), mask, mode,
                                   _ptr(bc), _ptr(bm), _ptr(pc), _ptr(pm))
    return int(bc[0]), int(bm[0]), pc, pm, int(n)


def _counters_dict(c: _Counters) -> dict:
    return {n: int(getattr(c, n)) for n, _ in _Counters._fields_}


def vnd(inst: Instance, gM, gR, mode: int = 0):
    """Algorithm 1 (pipe VND).  Returns (gM, gR, counters) with new arrays."""
    lib = _load()
    gm = _bits(gM, inst.K, inst.T).copy()
    gr = _bits(gR, inst.K, inst.T).copy()
    cnt = _Counters()
    rc = lib.orc_vnd(inst.cref, _ptr(gm), _ptr(gr), mode, ctypes.byref(cnt))
    if rc != 0:
        raise RuntimeError("oracle VND hit its cycle cap")
    return gm, gr, _counters_dict(cnt)


def splitmix64(z: int) -> int:
    return int(_load().orc_splitmix64(z & 0xFFFFFFFFFFFFFFFF))


def draw(seed: int, it: int, k: int, j: int) -> int:
    return int(_load().orc_draw(seed, it, k, j))


def shake(K, T, gM, gR, seed, it, k):
    """Algorithm 2's Shake(x, k) in place."""
    _load().orc_shake(K, T, _ptr(gM), _ptr(gR), seed, it, k)


@dataclass
class VnsResult:
    best_cost: int
    gM: np.ndarray
    gR: np.ndarray
    counters: dict
    traj: np.ndarray
    traj_hash: int


def vns(inst: Instance, seed: int, iters: int, kmax: int = 3, mode: int = 0,
        gM=None, gR=None) -> VnsResult:
    """Algorithm 2 (GVNS reading) from the given start (default: all open)."""
    lib = _load()
    if gM is None or gR is None:
        gM, gR = initial_solution(inst.K, inst.T)
    gm = _bits(gM, inst.K, inst.T).copy()
    gr = _bits(gR, inst.K, inst.T).copy()
    cnt = _Counters()
    log = np.zeros(max(iters, 1), TRAJ_DTYPE)
    bc = np.zeros(1, np.int64)
    h = np.zeros(1, np.uint64)
    rc = lib.orc_vns(inst.cref, _ptr(gm), _ptr(gr), seed & 0xFFFFFFFFFFFFFFFF,
                     iters, kmax, mode, ctypes.byref(cnt), _ptr(log), _ptr(bc), _ptr(h))
    if rc != 0:
        raise RuntimeError("oracle VNS hit a VND cycle cap")
    return VnsResult(int(bc[0]), gm, gr, _counters_dict(cnt), log[:iters], int(h[0]))


def shake_worker(K, T, gM, gR, seed, it, k, worker):
    """Shake(x, k) of fork-join worker p, in place (draws keyed p << 8 | j)."""
    _load().orc_shake_worker(K, T, _ptr(gM), _ptr(gR), seed, it, k, worker)


def vns_forkjoin(inst: Instance, seed: int, iters: int, kmax: int = 3, mode: int = 0,
                 workers: int = 2, gM=None, gR=None) -> VnsResult:
    """Algorithm 2 with P workers per iteration (Section 3's fork-join model):
    every worker shakes the incumbent with its own draws and runs VND, the
    least (f, worker) is kept when it improves.  traj["pad"] = the winner."""
    lib = _load()
    if gM is None or gR is None:
        gM, gR = initial_solution(inst.K, inst.T)
    gm = _bits(gM, inst.K, inst.T).copy()
    gr = _bits(gR, inst.K, inst.T).copy()
    cnt = _Counters()
    log = np.zeros(max(iters, 1), TRAJ_DTYPE)
    bc = np.zeros(1, np.int64)
    h = np.zeros(1, np.uint64)
    rc = lib.orc_vns_forkjoin(inst.cref, _ptr(gm), _ptr(gr), seed & 0xFFFFFFFFFFFFFFFF,
                              iters, kmax, mode, workers, ctypes.byref(cnt), _ptr(log),
                              _ptr(bc), _ptr(h))
    if rc != 0:
        raise RuntimeError("oracle fork-join GVNS hit a VND cycle cap")
    return VnsResult(int(bc[0]), gm, gr, _counters_dict(cnt), log[:iters], int(h[0]))


def multistart(inst: Instance, seeds, iters: int, kmax: int = 3, mode: int = 0):
    """Independent starts (same instance, same initial solution, one seed
    each); the best is the lexicographic minimum of (cost, start index)."""
    results = [vns(inst, int(s), iters, kmax, mode) for s in seeds]
    best = min(range(len(results)), key=lambda i: (results[i].best_cost, i))
    return best, results


def decode_steps(inst: Instance, k: int, gM_row, gR_row, j: int, local: int) -> int:
    """Work measure (not part of the method): setup segments of the moved row
    that a re-decode visits before the rest of the row is known from the row
    before the move (defined in ``orc_decode_steps``)."""
    gm = _bits(gM_row, 1, inst.T)
    gr = _bits(gR_row, 1, inst.T)
    return int(_load().orc_decode_steps(inst.cref, k, _ptr(gm), _ptr(gr), j, local))
