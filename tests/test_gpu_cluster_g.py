"""Mode G (one best move over the whole neighbourhood) on multi-CTA teams.

The single argmin of mode G spans every product of the instance.  When a
run's rows are spread over the CTAs of a thread-block cluster, the CTAs'
best keys meet through distributed shared memory once per neighbourhood.
These tests check, bit for bit against the oracle, that the cluster size,
the lanes per row and the placement of the prefix tables change nothing:
GVNS trajectories, final solutions and counters, up to the paper's
instance size (K = 300 products; T = 104 periods here, twice the paper's 52).
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
    assert r["best_cost"] == o.best_cost
    np.testing.assert_array_equal(r["gM"], o.gM)
    np.testing.assert_array_equal(r["gR"], o.gR)
    for key in ("moves_evaluated", "evals", "vnd_cycles", "applied", "iterations", "accepted"):
        assert r[key] == o.counters[key], key
    assert r["traj_hash"] == o.traj_hash


@pytest.fixture(scope="module")
def medium_g():
    """Oracle: mode-G GVNS on the medium instance (K=50, T=52), 40 iterations."""
    g = gen.plain_medium()
    return g, oracle.vns(oracle.Instance.from_arrays(g), seed=1, iters=40, kmax=3, mode=1)


@pytest.mark.parametrize("cluster,lanes,threads",
                         [(1, 32, 256), (2, 16, 256), (4, 32, 128), (8, 8, 64),
                          (8, 64, 128), (16, 32, 96), (3, 128, 256)])
def test_mode_g_cluster_trajectory(E, medium_g, cluster, lanes, threads):
    g, o = medium_g
    with E.Solver(g, cluster=cluster, lanes=lanes, threads=threads) as s:
        r = s.vns(seed=1, iters=40, kmax=3, mode=1)
        shape = s.launch_shape()
    assert shape["cluster"] == cluster and shape["lanes"] == lanes
    _check(r, o)


def test_mode_g_cluster_vnd_from_random_states(E):
    """Mode-G VND alone (iters = 0) from random, partly infeasible states on a
    4-CTA team: the objective bookkeeping across CTAs starts from rows that
    fall short."""
    g = gen.make_instance(8, 3, K=29, T=40)
    inst = oracle.Instance.from_arrays(g)
    rng = np.random.default_rng(5)
    for i in range(4):
        gm = (rng.random((inst.K, inst.T)) < 0.4).astype(np.uint8)
        gr = (rng.random((inst.K, inst.T)) < 0.4).astype(np.uint8)
        gm[:, 0] = 1
        if i == 1:
            gm[3, :] = 0  # one infeasible row: only a move in it can help
            gr[3, :] = 0
        om, orr, cnt = oracle.vnd(inst, gm, gr, 1)
        with E.Solver(g, cluster=4, lanes=16, threads=128) as s:
            s.set_state(gm, gr)
            r = s.vns(seed=0, iters=0, kmax=3, mode=1)
        np.testing.assert_array_equal(r["gM"], om)
        np.testing.assert_array_equal(r["gR"], orr)
        for key in ("moves_evaluated", "evals", "vnd_cycles", "applied"):
            assert r[key] == cnt[key], key


@pytest.fixture(scope="module")
def paper_scale():
    """K=300, T=104: a mode-P local optimum (oracle VND from all open) as the
    start of a short mode-G GVNS, both from the oracle."""
    g = gen.make_instance(9, 7, K=300, T=104)
    inst = oracle.Instance.from_arrays(g)
    gm0, gr0 = oracle.initial_solution(inst.K, inst.T)
    sm, sr, _ = oracle.vnd(inst, gm0, gr0, 0)
    o = oracle.vns(inst, seed=3, iters=6, kmax=3, mode=1, gM=sm, gR=sr)
    return g, sm, sr, o


@pytest.mark.parametrize("cluster", [0, 4, 16])
def test_mode_g_paper_scale(E, paper_scale, cluster):
    """Mode-G GVNS at K=300, T=104 across cluster sizes (4 CTAs keep the
    prefix tables in global memory; 0 = automatic)."""
    g, sm, sr, o = paper_scale
    with E.Solver(g, cluster=cluster) as s:
        s.set_state(sm, sr)
        r = s.vns(seed=3, iters=6, kmax=3, mode=1)
        shape = s.launch_shape()
    assert shape["cluster"] >= 4
    if cluster == 4:
        assert shape["tables_in_smem"] == 0
    _check(r, o)


def test_mode_p_paper_scale_vnd(E, paper_scale):
    """The mode-P VND that produced the start, on the GPU (K=300, T=104)."""
    g, sm, sr, _ = paper_scale
    with E.Solver(g) as s:
        r = s.vns(seed=0, iters=0, kmax=3, mode=0)
    np.testing.assert_array_equal(r["gM"], sm)
    np.testing.assert_array_equal(r["gR"], sr)


@pytest.mark.parametrize("teams,cluster", [(2, 1), (5, 2), (16, 4), (0, 0), (31, 1)])
def test_mode_g_speculative_run_matches_oracle(E, teams, cluster):
    """Mode-G runs speculate like mode-P ones: teams run consecutive
    iterations and commit them in order up to the first acceptance, so the
    trajectory, solution and counters equal the sequential run's."""
    g = gen.make_instance(6, 1, K=20, T=30)
    o = oracle.vns(oracle.Instance.from_arrays(g), seed=9, iters=150, kmax=3, mode=1)
    with E.Solver(g, cluster=cluster, speculation=teams) as s:
        r = s.vns(seed=9, iters=150, kmax=3, mode=1)
        shape = s.launch_shape()
    if teams != 1:
        assert shape["teams"] > 1
    _check(r, o)
    assert r["segments"] > 0


def test_mode_g_speculation_counts_committed_work_only(E):
    g = gen.make_instance(6, 2, K=24, T=40)
    res = []
    for teams in (1, 12):
        with E.Solver(g, speculation=teams) as s:
            r = s.vns(seed=2, iters=120, kmax=3, mode=1)
        res.append((r["best_cost"], r["traj_hash"], r["moves_evaluated"], r["segments"],
                    r["applied"], r["vnd_cycles"], r["iterations"], r["accepted"]))
    assert res[0] == res[1]
