"""ctypes binding of the C ABI in include/elsr.h (argument marshalling only).

The library is the in-tree ``_build/libelsr.so`` compiled by ``build.py``.
Loading fails loudly when it is missing or when no CUDA device is present:
there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libelsr.so")

ELSR_OK = 0
ELSR_E_ARG = -1
ELSR_E_RANGE = -2
ELSR_E_NOMEM = -3
ELSR_E_CUDA = -4
ELSR_E_CAP = -5
ELSR_E_STATE = -6
ELSR_E_TIMEOUT = -7
ELSR_E_BUSY = -8
MODE_P = 0
MODE_G = 1
T_MAX = 128
INF = (1 << 63) - 1


class Stats(ctypes.Structure):
    _fields_ = [("best_cost", ctypes.c_int64), ("traj_hash", ctypes.c_uint64),
                ("moves_evaluated", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("vnd_cycles", ctypes.c_int64), ("applied", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("segments", ctypes.c_int64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "reserved"}


class Checkpoint(ctypes.Structure):
    """elsr_checkpoint_t: Algorithm 2's loop state between two iterations."""
    _fields_ = [("seed", ctypes.c_uint64), ("kmax", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("workers", ctypes.c_int32), ("next_it", ctypes.c_int32), ("k", ctypes.c_int32),
                ("status", ctypes.c_int32), ("cost", ctypes.c_int64),
                ("traj_hash", ctypes.c_uint64), ("moves_evaluated", ctypes.c_int64),
                ("evals", ctypes.c_int64), ("vnd_cycles", ctypes.c_int64),
                ("applied", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("segments", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}

    @classmethod
    def from_dict(cls, d: dict) -> "Checkpoint":
        c = cls()
        for n, _ in cls._fields_:
            setattr(c, n, int(d[n]))
        return c


class Traj(ctypes.Structure):
    _fields_ = [("it", ctypes.c_int32), ("k", ctypes.c_int32), ("cost", ctypes.c_int64),
                ("accepted", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# (restype, argtypes) of every entry point declared in include/elsr.h
P = ctypes.c_void_p
i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
SIGNATURES = {
    "elsr_version": (ctypes.c_int, []),
    "elsr_run_footprint": (ctypes.c_int, [i32, i32, P, P]),
    "elsr_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "elsr_last_error": (ctypes.c_char_p, [P]),
    "elsr_create": (ctypes.c_int, [ctypes.POINTER(P), i32, i32, P, P, P, P, P, P]),
    "elsr_create_ex": (ctypes.c_int, [ctypes.POINTER(P), i32, i32, P, P, P, P, P, P, P, P]),
    "elsr_destroy": (None, [P]),
    "elsr_set_stream": (ctypes.c_int, [P, P]),
    "elsr_set_launch": (ctypes.c_int, [P, i32, i32]),
    "elsr_set_cluster": (ctypes.c_int, [P, i32]),
    "elsr_set_speculation": (ctypes.c_int, [P, i32]),
    "elsr_launch_shape": (ctypes.c_int, [P, P]),
    "elsr_set_state": (ctypes.c_int, [P, P, P]),
    "elsr_get_state": (ctypes.c_int, [P, P, P]),
    "elsr_cost": (ctypes.c_int, [P, P, P]),
    "elsr_eval_neighbourhood": (ctypes.c_int, [P, u32, i32, P, P, P, P]),
    "elsr_move_costs": (ctypes.c_int, [P, i32, P, P]),
    "elsr_vns_run": (ctypes.c_int, [P, u64, i32, i32, i32]),
    "elsr_vns_forkjoin_run": (ctypes.c_int, [P, u64, i32, i32, i32, i32]),
    "elsr_set_time_limit": (ctypes.c_int, [P, i64]),
    "elsr_checkpoint": (ctypes.c_int, [P, P, P, P]),
    "elsr_vns_resume": (ctypes.c_int, [P, P, P, P, i32]),
    "elsr_result": (ctypes.c_int, [P, P, P, P, P, P, i32]),
    "elsr_multistart_run": (ctypes.c_int, [P, u64, i32, i32, i32, i32, P, P, P]),
    "elsr_counters": (ctypes.c_int, [P, P]),
    "elsr_multistart_stats": (ctypes.c_int, [P, P, i32]),
    "elsr_eval_neighbourhood_static": (ctypes.c_int, [i32, i32, P, P, P, P, P, P, P, P,
                                                      u32, i32, P, P, P, P]),
    "elsr_batch_create": (ctypes.c_int, [ctypes.POINTER(P), i32, P, P, P, P, P, P, P, P]),
    "elsr_batch_create_on": (ctypes.c_int, [ctypes.POINTER(P), i32, P, P, P, P, P, P, P, P, P]),
    "elsr_batch_create_ex": (ctypes.c_int, [ctypes.POINTER(P), i32, P, P, P, P, P, P, P, P,
                                            P, P, P]),
    "elsr_batch_destroy": (None, [P]),
    "elsr_batch_last_error": (ctypes.c_char_p, [P]),
    "elsr_batch_set_stream": (ctypes.c_int, [P, P]),
    "elsr_batch_set_launch": (ctypes.c_int, [P, i32, i32]),
    "elsr_batch_set_cluster": (ctypes.c_int, [P, i32]),
    "elsr_batch_launch_shape": (ctypes.c_int, [P, P]),
    "elsr_batch_set_runs_per_cta": (ctypes.c_int, [P, i32]),
    "elsr_batch_set_count_steps": (ctypes.c_int, [P, i32]),
    "elsr_batch_stage_tables": (ctypes.c_int, [P]),
    "elsr_set_count_steps": (ctypes.c_int, [P, i32]),
    "elsr_batch_packing": (ctypes.c_int, [P, P, P]),
    "elsr_batch_run": (ctypes.c_int, [P, P, i32, i32, i32]),
    "elsr_batch_results": (ctypes.c_int, [P, P]),
    "elsr_batch_solution": (ctypes.c_int, [P, i32, P, P]),
    "elsr_int_issue_probe": (ctypes.c_int, [P, i32, i32, P, P, P]),
    "elsr_server_create": (ctypes.c_int, [ctypes.POINTER(P), P]),
    "elsr_server_destroy": (None, [P]),
    "elsr_server_last_error": (ctypes.c_char_p, [P]),
    "elsr_server_submit": (ctypes.c_int, [P, i32, i32, P, P, P, P, P, P, u64, i32, i32, i32,
                                          P]),
    "elsr_server_poll": (ctypes.c_int, [P, i32, P, P]),
    "elsr_server_solution": (ctypes.c_int, [P, i64, P, P]),
    "elsr_server_release": (ctypes.c_int, [P, i64]),
    "elsr_server_info": (ctypes.c_int, [P, P, P]),
}


class ServerConfig(ctypes.Structure):
    """elsr_server_config_t."""
    _fields_ = [("slots", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("cells", ctypes.c_int64), ("rows", ctypes.c_int64),
                ("max_runs", ctypes.c_int32), ("acc64", ctypes.c_int32),
                ("count_steps", ctypes.c_int32), ("keep_solutions", ctypes.c_int32)]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return LIB_PATH


def load(path: str | None = None):
    """Load libelsr.so (raises when it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"{p} is missing: build it with paper_1704_05132_gb300.build.build() "
                    "(the engine has no CPU fallback)")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


class ElsrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"elsr error {code}: {msg}")
        self.code = code


def check(code: int, handle=None, batch=False, server=False) -> int:
    if code < 0:
        lib = load()
        msg = (lib.elsr_server_last_error(handle) if server
               else lib.elsr_batch_last_error(handle) if batch
               else lib.elsr_last_error(handle))
        base = lib.elsr_strerror(code).decode()
        detail = msg.decode() if msg else ""
        raise ElsrError(code, f"{base}: {detail}" if detail else base)
    return code
