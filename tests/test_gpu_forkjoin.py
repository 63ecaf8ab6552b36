"""Fork-join GVNS on the GPU vs the oracle (Algorithm 2 as the paper runs it:
every worker shakes the same incumbent with its own draws and runs VND, the
least (cost, worker) is kept when it improves).

Bit-exact: per-iteration (k, cost, accepted, winning worker), final solution,
counters (every worker's VND counts) and the trajectory hash.
"""
import numpy as np
import pytest

import oracle
from paper_1704_05132_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_05132_gb300 import build, elsr
    build.build()
    oracle.build()
    return elsr


def _check(r, o):
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    np.testing.assert_array_equal(r["traj"]["k"], o.traj["k"])
    np.testing.assert_array_equal(r["traj"]["accepted"], o.traj["accepted"])
    np.testing.assert_array_equal(r["traj"]["worker"], o.traj["pad"])
    assert r["best_cost"] == o.best_cost
    np.testing.assert_array_equal(r["gM"], o.gM)
    np.testing.assert_array_equal(r["gR"], o.gR)
    for key in ("moves_evaluated", "evals", "vnd_cycles", "applied", "iterations", "accepted"):
        assert r[key] == o.counters[key], key
    assert r["traj_hash"] == o.traj_hash
    assert r["status"] == 0


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("workers", [1, 2, 5, 16])
def test_forkjoin_small(E, mode, workers):
    """K=5 products, T=12 periods, seed 0, 200 iterations."""
    g = gen.plain_small()
    o = oracle.vns_forkjoin(oracle.Instance.from_arrays(g), seed=0, iters=200, kmax=3,
                            mode=mode, workers=workers)
    with E.Solver(g) as s:
        r = s.vns_forkjoin(seed=0, iters=200, kmax=3, mode=mode, workers=workers)
        assert s.launch_shape()["teams"] == workers
    _check(r, o)


def test_forkjoin_one_worker_equals_sequential_run(E):
    g = gen.make_instance(3, 3, K=17, T=30)
    with E.Solver(g) as s:
        a = s.vns(seed=5, iters=300, kmax=3, mode=0)
        b = s.vns_forkjoin(seed=5, iters=300, kmax=3, mode=0, workers=1)
    for key in ("best_cost", "traj_hash", "moves_evaluated", "applied", "accepted", "segments"):
        assert a[key] == b[key], key
    np.testing.assert_array_equal(a["gM"], b["gM"])
    np.testing.assert_array_equal(a["traj"]["cost"], b["traj"]["cost"])


@pytest.fixture(scope="module")
def medium_fj():
    g = gen.plain_medium()
    return g, oracle.vns_forkjoin(oracle.Instance.from_arrays(g), seed=1, iters=100, kmax=3,
                                  mode=0, workers=4)


@pytest.mark.parametrize("cluster,lanes", [(0, 0), (1, 32), (2, 16), (8, 64)])
def test_forkjoin_medium(E, medium_fj, cluster, lanes):
    """K=50, T=52, 4 workers, 100 iterations, across team shapes."""
    g, o = medium_fj
    with E.Solver(g, cluster=cluster, lanes=lanes) as s:
        r = s.vns_forkjoin(seed=1, iters=100, kmax=3, mode=0, workers=4)
    _check(r, o)
    assert r["segments"] > 0


def test_forkjoin_mode_g_cluster(E):
    """Mode G inside each worker, workers of 4 CTAs (K=40, T=36)."""
    g = gen.make_instance(12, 1, K=40, T=36)
    o = oracle.vns_forkjoin(oracle.Instance.from_arrays(g), seed=2, iters=25, kmax=3,
                            mode=1, workers=3)
    with E.Solver(g, cluster=4) as s:
        r = s.vns_forkjoin(seed=2, iters=25, kmax=3, mode=1, workers=3)
        assert s.launch_shape()["cluster"] == 4
    _check(r, o)


def test_forkjoin_rejects_more_workers_than_resident(E):
    """More workers than the device holds at once is refused on the host
    (nothing is launched), and the handle stays usable."""
    g = gen.plain_medium()
    with E.Solver(g, cluster=8) as s:
        with pytest.raises(Exception) as ei:
            s.vns_forkjoin_run(seed=1, iters=10, kmax=3, mode=0, workers=4000)
        assert "resident" in str(ei.value)
        r = s.vns_forkjoin(seed=1, iters=10, kmax=3, mode=0, workers=2)
        assert r["status"] == 0 and r["iterations"] == 10
