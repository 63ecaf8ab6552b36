"""Checkpoint / resume of GVNS runs and the wall-clock budget (Algorithm 2's
stopping test on elapsed time), against the oracle's uninterrupted runs.

A run of N iterations, a checkpoint and a resume of M iterations must give
exactly the oracle's run of N + M iterations: every trajectory entry, the
final solution, the trajectory hash and the totals.  A budgeted run stops at
an iteration boundary, so it must equal the oracle's run of as many
iterations as it reports.
"""
import numpy as np
import pytest

import oracle
from paper_1704_05132_gb300 import gen

pytestmark = pytest.mark.gpu

COUNTERS = ("moves_evaluated", "evals", "vnd_cycles", "applied", "iterations", "accepted")


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_05132_gb300 import build, elsr
    build.build()
    oracle.build()
    return elsr


def _oracle(g, seed, iters, mode, workers):
    inst = oracle.Instance.from_arrays(g)
    if workers:
        return oracle.vns_forkjoin(inst, seed=seed, iters=iters, kmax=3, mode=mode,
                                   workers=workers)
    return oracle.vns(inst, seed=seed, iters=iters, kmax=3, mode=mode)


def _run(s, seed, iters, mode, workers):
    if workers:
        return s.vns_forkjoin(seed=seed, iters=iters, kmax=3, mode=mode, workers=workers)
    return s.vns(seed=seed, iters=iters, kmax=3, mode=mode)


def _check_final(r, o):
    assert r["status"] == 0
    assert r["best_cost"] == o.best_cost
    assert r["traj_hash"] == o.traj_hash
    np.testing.assert_array_equal(r["gM"], o.gM)
    np.testing.assert_array_equal(r["gR"], o.gR)
    for key in COUNTERS:
        assert r[key] == o.counters[key], key


CASES = [("medium_P", gen.plain_medium, 1, 0, 0, 300, 200),
         ("small_G", gen.plain_small, 0, 1, 0, 120, 80),
         ("small_fj3", gen.plain_small, 0, 0, 3, 100, 100),
         ("K20_fj2_G", lambda: gen.make_instance(6, 4, K=20, T=24), 2, 1, 2, 40, 35)]


@pytest.mark.parametrize("name,mk,seed,mode,workers,n1,n2", CASES, ids=[c[0] for c in CASES])
def test_resume_equals_uninterrupted(E, tmp_path, name, mk, seed, mode, workers, n1, n2):
    g = mk()
    o = _oracle(g, seed, n1 + n2, mode, workers)
    with E.Solver(g) as s:
        r1 = _run(s, seed, n1, mode, workers)
        ck = s.checkpoint()
    assert ck["next_it"] == n1 and ck["status"] == 0 and ck["workers"] == workers
    assert ck["cost"] == r1["best_cost"] and ck["traj_hash"] == r1["traj_hash"]
    path = str(tmp_path / "ck.npz")
    E.save_checkpoint(path, ck)
    ck2 = E.load_checkpoint(path)
    with E.Solver(g) as s2:  # a fresh handle, as after a restart
        r2 = s2.vns_resume(ck2, n2)
        ck3 = s2.checkpoint()
    traj = np.concatenate([r1["traj"], r2["traj"]])
    np.testing.assert_array_equal(traj["it"], np.arange(n1 + n2))
    np.testing.assert_array_equal(traj["cost"], o.traj["cost"])
    np.testing.assert_array_equal(traj["k"], o.traj["k"])
    np.testing.assert_array_equal(traj["accepted"], o.traj["accepted"])
    if workers:
        np.testing.assert_array_equal(traj["worker"], o.traj["pad"])
    _check_final(r2, o)
    assert ck3["next_it"] == n1 + n2 and ck3["moves_evaluated"] == o.counters["moves_evaluated"]


@pytest.mark.parametrize("workers", [0, 4])
def test_time_limit_stops_on_an_iteration_boundary(E, workers):
    """A budget of a few milliseconds ends the run early; what it ran is the
    oracle's run of that many iterations, and a resume completes it."""
    g = gen.plain_medium()
    with E.Solver(g) as s:
        s.set_time_limit(4000)
        r = _run(s, 1, 1_000_000, 0, workers)
        n = r["iterations"]
        assert 0 < n < 1_000_000
        ck = s.checkpoint()
        s.set_time_limit(0)
        r2 = s.vns_resume(ck, 20)
    o = _oracle(g, 1, n, 0, workers)
    assert r["best_cost"] == o.best_cost and r["traj_hash"] == o.traj_hash
    np.testing.assert_array_equal(r["traj"]["cost"][:n], o.traj["cost"])
    o2 = _oracle(g, 1, n + 20, 0, workers)
    _check_final(r2, o2)


def test_resume_rejects_a_state_that_does_not_match(E):
    """A checkpoint whose cost does not belong to the given solution stops
    before its first iteration (status ELSR_E_STATE); the handle stays usable."""
    g = gen.plain_small()
    with E.Solver(g) as s:
        s.vns(seed=0, iters=30, kmax=3, mode=0)
        ck = s.checkpoint()
        bad = dict(ck, cost=ck["cost"] + 1)
        r = s.vns_resume(bad, 10)
        assert r["status"] == E.nat.ELSR_E_STATE
        with pytest.raises(Exception):
            s.vns_resume(dict(ck, k=4), 10)  # k beyond kmax: refused on the host
        r2 = s.vns_resume(ck, 10)
        assert r2["status"] == 0 and r2["iterations"] == 40


def test_multistart_after_resume_and_budget_starts_fresh(E):
    """Run descriptors of a resume or a budgeted run do not leak into a later
    multi-start on the same handle: every start equals the oracle's run."""
    g = gen.plain_small()
    inst = oracle.Instance.from_arrays(g)
    want = [oracle.vns(inst, seed=i, iters=40, kmax=3, mode=0).best_cost for i in range(8)]
    with E.Solver(g) as s:
        s.vns(seed=0, iters=30, kmax=3, mode=0)
        ck = s.checkpoint()
        for step in ("resume", "budget"):
            if step == "resume":
                s.vns_resume(ck, 10)
            else:
                s.set_time_limit(2000)
                s.vns(seed=1, iters=50, kmax=3, mode=0)
            s.set_state()  # back to every setup open
            best, start, costs = s.multistart(0, 8, 40, 3, 0, costs=True)
            np.testing.assert_array_equal(costs, want)
            assert (best, start) == min((c, i) for i, c in enumerate(want))
