"""Run many independent oracle GVNS runs on every host core (test helper).

The pool is started with the "spawn" method, so no worker inherits the
parent's CUDA state.  A job is (instance arrays, seed, iters, start bits or
None[, want_bits]); the result is the run's best cost, trajectory hash and
counters, plus its solution (gM, gR) when want_bits is set.
"""
from __future__ import annotations

import multiprocessing as mp
import os


def _job(job):
    import oracle
    (D, R, kM, kR, hM, hR), seed, iters, start = job[:4]
    inst = oracle.Instance(D, R, kM, kR, hM, hR)
    gm, gr = start if start is not None else (None, None)
    r = oracle.vns(inst, int(seed), int(iters), 3, 0, gM=gm, gR=gr)
    if len(job) > 4 and job[4]:
        return r.best_cost, r.traj_hash, r.counters, r.gM, r.gR
    return r.best_cost, r.traj_hash, r.counters


def arrays(g):
    return (g.D, g.R, g.kM, g.kR, g.hM, g.hR)


def run_many(jobs):
    """Results of oracle.vns for every job, in order, on all host cores."""
    import oracle
    oracle.build()
    n = max(1, min(len(jobs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_job, jobs, chunksize=max(1, len(jobs) // (8 * n)))
