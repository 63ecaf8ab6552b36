"""Degenerate instances on the GPU vs the oracle, bit for bit.

* rows with no demand and no returns (every pattern feasible, the empty
  pattern optimal);
* rows whose returns exceed demand (nothing manufactured once every gR is
  open; the returns stock only grows);
* zero holding costs and zero setup costs, where most moves tie and the
  lowest index must win, per product and across products;
* identical products, where mode G's argmin ties across products and, on a
  multi-CTA team, across the CTAs of a cluster;
* an instance with no cost at all, where no GVNS iteration is ever
  accepted (every speculative team's iteration commits).

Each case runs the neighbourhood evaluation, VND and GVNS trajectories
(speculative, cluster, fork-join and batched launches).
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


def _inst(D, R, kM, kR, hM, hR):
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    return gen.ElsrInstance(i32(D), i32(R), i32(kM), i32(kR), i32(hM), i32(hR))


def mixed_rows():
    """K=12, T=30: rows 0, 5, 11 without demand or returns, rows 3 and 8 with
    returns above demand, the rest as generated."""
    g = gen.make_instance(41, 0, K=12, T=30)
    D, R = g.D.copy(), g.R.copy()
    D[[0, 5, 11]] = 0
    R[[0, 5, 11]] = 0
    R[[3, 8]] = D[[3, 8]] + 13
    return _inst(D, R, g.kM, g.kR, g.hM, g.hR)


def zero_holding():
    g = gen.make_instance(42, 0, K=10, T=26)
    z = np.zeros(10)
    return _inst(g.D, g.R, g.kM, g.kR, z, z)


def zero_setup():
    g = gen.make_instance(43, 0, K=10, T=26)
    z = np.zeros(10)
    return _inst(g.D, g.R, z, z, g.hM, g.hR)


def identical_products(K=40, T=30):
    g = gen.make_instance(44, 0, K=1, T=T)
    rep = lambda a: np.repeat(a, K, axis=0)
    return _inst(rep(g.D), rep(g.R), rep(g.kM), rep(g.kR), rep(g.hM), rep(g.hR))


def no_cost():
    g = gen.make_instance(45, 0, K=8, T=20)
    z = np.zeros(8)
    return _inst(g.D, g.R, z, z, z, z)


CASES = [("mixed_rows", mixed_rows), ("zero_holding", zero_holding),
         ("zero_setup", zero_setup), ("identical", identical_products),
         ("no_cost", no_cost)]
IDS = [c[0] for c in CASES]


def _states(rng, K, T, n):
    yield np.ones((K, T), np.uint8), np.ones((K, T), np.uint8)
    yield np.zeros((K, T), np.uint8), np.zeros((K, T), np.uint8)
    for _ in range(n):
        gm = (rng.random((K, T)) < rng.uniform(0.1, 0.7)).astype(np.uint8)
        gr = (rng.random((K, T)) < rng.uniform(0.1, 0.7)).astype(np.uint8)
        gm[:, 0] = 1
        yield gm, gr


def _check_run(r, o):
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    np.testing.assert_array_equal(r["traj"]["k"], o.traj["k"])
    np.testing.assert_array_equal(r["traj"]["accepted"], o.traj["accepted"])
    assert r["best_cost"] == o.best_cost and r["traj_hash"] == o.traj_hash
    np.testing.assert_array_equal(r["gM"], o.gM)
    np.testing.assert_array_equal(r["gR"], o.gR)
    for key in ("moves_evaluated", "evals", "vnd_cycles", "applied", "iterations", "accepted"):
        assert r[key] == o.counters[key], key


@pytest.mark.parametrize("name,mk", CASES, ids=IDS)
def test_evaluation(E, name, mk):
    g = mk()
    inst = oracle.Instance.from_arrays(g)
    rng = np.random.default_rng(len(name))
    with E.Solver(g) as s:
        for gm, gr in _states(rng, inst.K, inst.T, 3):
            s.set_state(gm, gr)
            tot, rc = s.cost()
            otot, orc = oracle.total_cost(inst, gm, gr)
            assert tot == otot
            np.testing.assert_array_equal(rc, orc)
            for j in (1, 2, 3):
                c, _ = s.move_costs(j)
                np.testing.assert_array_equal(c, oracle.move_costs(inst, gm, gr, j))
            for mode in (0, 1):
                for mask in (1, 4, 7):
                    got = s.eval_neighbourhood(mask, mode)
                    bc, bm, pc, pm, _ = oracle.eval_neighbourhood(inst, gm, gr, mask, mode)
                    assert got[:2] == (bc, bm), (mode, mask)
                    np.testing.assert_array_equal(got[2], pc)
                    np.testing.assert_array_equal(got[3], pm)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,mk", CASES, ids=IDS)
def test_gvns_default_launch(E, name, mk, mode):
    g = mk()
    iters = 150 if mode == 0 else 60
    o = oracle.vns(oracle.Instance.from_arrays(g), seed=6, iters=iters, kmax=3, mode=mode)
    with E.Solver(g) as s:
        r = s.vns(seed=6, iters=iters, kmax=3, mode=mode)
    _check_run(r, o)
    if name == "no_cost":
        assert o.counters["accepted"] == 0


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_identical_products_mode_g_on_clusters(E, cluster):
    """Every product offers the same best move: the lowest product index
    must win even when the tied products sit on different CTAs."""
    g = identical_products()
    o = oracle.vns(oracle.Instance.from_arrays(g), seed=2, iters=30, kmax=3, mode=1)
    with E.Solver(g, cluster=cluster) as s:
        r = s.vns(seed=2, iters=30, kmax=3, mode=1)
        assert s.launch_shape()["cluster"] == cluster
    _check_run(r, o)


@pytest.mark.parametrize("name,mk", CASES, ids=IDS)
def test_forkjoin(E, name, mk):
    """Fork-join workers whose results tie: the lowest worker wins."""
    g = mk()
    o = oracle.vns_forkjoin(oracle.Instance.from_arrays(g), seed=8, iters=40, kmax=3,
                            mode=0, workers=4)
    with E.Solver(g) as s:
        r = s.vns_forkjoin(seed=8, iters=40, kmax=3, mode=0, workers=4)
    _check_run(r, o)
    np.testing.assert_array_equal(r["traj"]["worker"], o.traj["pad"])


def test_batch(E):
    insts = [mk() for _, mk in CASES] + [identical_products(3, 12), gen.plain_small()]
    seeds = np.arange(len(insts), dtype=np.uint64) + 30
    b = E.Batch(insts)
    b.run(seeds, iters=80, kmax=3, mode=0)
    res = b.results()
    for i, g in enumerate(insts):
        o = oracle.vns(oracle.Instance.from_arrays(g), seed=30 + i, iters=80, kmax=3, mode=0)
        assert res[i]["status"] == 0
        assert res[i]["best_cost"] == o.best_cost and res[i]["traj_hash"] == o.traj_hash, i
        gm, gr = b.solution(i)
        np.testing.assert_array_equal(gm, o.gM)
        np.testing.assert_array_equal(gr, o.gR)
    b.close()
