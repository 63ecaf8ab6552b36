"""Unit production costs pM, pR (Algorithm 1's p_M, p_R) on the GPU vs the
oracle, bit for bit: per-move row costs and decode steps, neighbourhood
evaluations in modes P and G, VND, GVNS trajectories (speculative, cluster,
fork-join and batched launches), with pR - pM of both signs and values large
enough to need 64-bit row accumulators.
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


def _big(g):
    """Production costs large enough that rows need 64-bit accumulators."""
    K = g.D.shape[0]
    return gen.ElsrInstance(g.D, g.R, g.kM, g.kR, g.hM, g.hR,
                            np.full(K, 2_000_000, np.int32), np.full(K, 900_000, np.int32))


CASES = [("K5_T12", lambda: gen.with_production_costs(gen.plain_small(), 1)),
         ("K9_T40", lambda: gen.with_production_costs(gen.make_instance(3, 1, K=9, T=40), 2,
                                                      pR_range=(0, 400))),
         ("K6_T65", lambda: gen.with_production_costs(gen.make_instance(3, 2, K=6, T=65), 3)),
         ("K4_T104_acc64", lambda: _big(gen.make_instance(3, 3, K=4, T=104)))]


def _states(rng, K, T, n):
    yield np.ones((K, T), np.uint8), np.ones((K, T), np.uint8)
    for i in range(n):
        gm = (rng.random((K, T)) < rng.uniform(0.1, 0.8)).astype(np.uint8)
        gr = (rng.random((K, T)) < rng.uniform(0.1, 0.8)).astype(np.uint8)
        if i % 2 == 0:
            gm[:, 0] = 1
        yield gm, gr


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_move_costs_and_evaluation(E, name, mk):
    g = mk()
    inst = oracle.Instance.from_arrays(g)
    rng = np.random.default_rng(len(name))
    with E.Solver(g) as s:
        for gm, gr in _states(rng, inst.K, inst.T, 4):
            s.set_state(gm, gr)
            tot, rc = s.cost()
            otot, orc = oracle.total_cost(inst, gm, gr)
            assert tot == otot
            np.testing.assert_array_equal(rc, orc)
            for j in (1, 2, 3):
                c, w = s.move_costs(j)
                np.testing.assert_array_equal(c, oracle.move_costs(inst, gm, gr, j))
            for mode in (0, 1):
                got = s.eval_neighbourhood(7, mode)
                bc, bm, pc, pm, _ = oracle.eval_neighbourhood(inst, gm, gr, 7, mode)
                assert got[:2] == (bc, bm)
                np.testing.assert_array_equal(got[2], pc)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_vns_trajectory(E, name, mk, mode):
    g = mk()
    o = oracle.vns(oracle.Instance.from_arrays(g), seed=4, iters=120, kmax=3, mode=mode)
    with E.Solver(g) as s:
        r = s.vns(seed=4, iters=120, kmax=3, mode=mode)
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    assert r["best_cost"] == o.best_cost and r["traj_hash"] == o.traj_hash
    np.testing.assert_array_equal(r["gM"], o.gM)
    np.testing.assert_array_equal(r["gR"], o.gR)
    for key in ("moves_evaluated", "applied", "accepted"):
        assert r[key] == o.counters[key], key


def test_medium_speculative_cluster_and_forkjoin(E):
    """K=50, T=52 with production costs: the default speculative launch, a
    mode-G cluster run and a fork-join run."""
    g = gen.with_production_costs(gen.plain_medium(), 5)
    inst = oracle.Instance.from_arrays(g)
    o = oracle.vns(inst, seed=1, iters=200, kmax=3, mode=0)
    with E.Solver(g) as s:
        r = s.vns(seed=1, iters=200, kmax=3, mode=0)
        assert s.launch_shape()["teams"] > 1
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    assert r["traj_hash"] == o.traj_hash and r["moves_evaluated"] == o.counters["moves_evaluated"]
    og = oracle.vns(inst, seed=2, iters=15, kmax=3, mode=1)
    with E.Solver(g, cluster=4) as s:
        rg = s.vns(seed=2, iters=15, kmax=3, mode=1)
    assert rg["traj_hash"] == og.traj_hash and rg["best_cost"] == og.best_cost
    of = oracle.vns_forkjoin(inst, seed=3, iters=40, kmax=3, mode=0, workers=3)
    with E.Solver(g) as s:
        rf = s.vns_forkjoin(seed=3, iters=40, kmax=3, mode=0, workers=3)
    assert rf["traj_hash"] == of.traj_hash and rf["best_cost"] == of.best_cost
    np.testing.assert_array_equal(rf["gM"], of.gM)


def test_batch_mixing_instances_with_and_without_production_costs(E):
    insts = []
    for i in range(12):
        g = gen.make_instance(8, i, K_range=(5, 30), T_range=(12, 40))
        insts.append(gen.with_production_costs(g, 8, 100 + i) if i % 2 else g)
    b = E.Batch(insts)
    seeds = np.arange(12, dtype=np.uint64) + 7
    b.run(seeds, iters=40, kmax=3, mode=0)
    res = b.results()
    for i in (0, 1, 4, 7, 11):
        o = oracle.vns(oracle.Instance.from_arrays(insts[i]), seed=7 + i, iters=40, kmax=3,
                       mode=0)
        assert res[i]["best_cost"] == o.best_cost and res[i]["traj_hash"] == o.traj_hash
    b.close()
