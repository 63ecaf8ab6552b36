"""GPU vs oracle parity through the C ABI (needs a GB300).

Integer work, so every comparison is bit-exact: per-move row costs and
decode steps, per-product and global argmins, VND results, whole GVNS
trajectories (entry by entry), final solutions, plans and counters.
"""
import numpy as np
import pytest

import oracle
from paper_1704_05132_gb300 import gen

pytestmark = pytest.mark.gpu

INF = oracle.INF


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_05132_gb300 import build, elsr
    build.build()
    oracle.build()
    return elsr


def _inst(g):
    return oracle.Instance.from_arrays(g)


def _states(rng, K, T, n):
    """Setup matrices: all open, random (feasible and infeasible rows), sparse."""
    yield np.ones((K, T), np.uint8), np.ones((K, T), np.uint8)
    for i in range(n):
        dm, dr = rng.uniform(0.05, 0.9), rng.uniform(0.05, 0.9)
        gm = (rng.random((K, T)) < dm).astype(np.uint8)
        gr = (rng.random((K, T)) < dr).astype(np.uint8)
        if i % 3 == 0:
            gm[:, 0] = 1
        if i % 3 == 1:
            gm[:, 0] = 1
            gr &= gm
        yield gm, gr


def _big_costs(g):
    """Same instance with holding costs large enough to need 64-bit rows."""
    g2 = gen.ElsrInstance(g.D.copy(), g.R.copy(), g.kM.copy(), g.kR.copy(),
                          (g.hM.astype(np.int64) * 20000).astype(np.int32),
                          (g.hR.astype(np.int64) * 20000).astype(np.int32))
    return g2


CASES = [
    ("plain_small", lambda: gen.plain_small()),
    ("K3_T1", lambda: gen.make_instance(5, 1, K=3, T=1)),
    ("K2_T2", lambda: gen.make_instance(5, 2, K=2, T=2)),
    ("K7_T63", lambda: gen.make_instance(5, 3, K=7, T=63)),
    ("K5_T64", lambda: gen.make_instance(5, 4, K=5, T=64)),
    ("K6_T65", lambda: gen.make_instance(5, 5, K=6, T=65)),
    ("K4_T128", lambda: gen.make_instance(5, 6, K=4, T=128)),
    ("K37_T52", lambda: gen.make_instance(5, 7, K=37, T=52)),
    ("wide_acc64", lambda: _big_costs(gen.make_instance(5, 8, K=9, T=40))),
]


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_move_costs_and_decode_steps(E, name, mk):
    g = mk()
    inst = _inst(g)
    rng = np.random.default_rng(len(name))
    with E.Solver(g) as s:
        for gm, gr in _states(rng, inst.K, inst.T, 4):
            s.set_state(gm, gr)
            tot, rc = s.cost()
            otot, orc = oracle.total_cost(inst, gm, gr)
            assert tot == otot
            np.testing.assert_array_equal(rc, orc)
            for j in (1, 2, 3):
                if oracle.row_moves(inst.T, j) <= 0:
                    continue
                c, w = s.move_costs(j)
                np.testing.assert_array_equal(c, oracle.move_costs(inst, gm, gr, j))
                per = oracle.row_moves(inst.T, j)
                # decode steps of a sample of moves, one by one through the oracle
                for m in rng.choice(len(c), size=min(len(c), 40), replace=False):
                    k, l = divmod(int(m), per)
                    assert w[m] == oracle.decode_steps(inst, k, gm[k], gr[k], j, l)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,mk", CASES[:6] + CASES[8:], ids=[c[0] for c in CASES[:6] + CASES[8:]])
def test_eval_neighbourhood(E, name, mk, mode):
    g = mk()
    inst = _inst(g)
    rng = np.random.default_rng(99 + mode)
    with E.Solver(g) as s:
        for gm, gr in _states(rng, inst.K, inst.T, 3):
            s.set_state(gm, gr)
            for mask in (1, 2, 4, 3, 7):
                got = s.eval_neighbourhood(mask, mode)
                bc, bm, pc, pm, _ = oracle.eval_neighbourhood(inst, gm, gr, mask, mode)
                assert got[0] == bc and got[1] == bm, (mask, got[:2], (bc, bm))
                np.testing.assert_array_equal(got[2], pc)
                np.testing.assert_array_equal(got[3], pm)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_vnd_parity(E, name, mk, mode):
    g = mk()
    inst = _inst(g)
    gm0, gr0 = oracle.initial_solution(inst.K, inst.T)
    om, orr, cnt = oracle.vnd(inst, gm0, gr0, mode)
    with E.Solver(g) as s:
        r = s.vns(seed=0, iters=0, kmax=3, mode=mode)
    np.testing.assert_array_equal(r["gM"], om)
    np.testing.assert_array_equal(r["gR"], orr)
    assert r["best_cost"] == oracle.total_cost(inst, om, orr)[0]
    for key in ("moves_evaluated", "evals", "vnd_cycles", "applied"):
        assert r[key] == cnt[key], key


def _check_run(r, o):
    assert r["best_cost"] == o.best_cost
    np.testing.assert_array_equal(r["gM"], o.gM)
    np.testing.assert_array_equal(r["gR"], o.gR)
    for key in ("moves_evaluated", "evals", "vnd_cycles", "applied", "iterations", "accepted"):
        assert r[key] == o.counters[key], key
    assert r["traj_hash"] == o.traj_hash


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("kmax", [1, 3])
def test_vns_small_trajectory(E, mode, kmax):
    """Plain VNS, K=5 products, T=12 periods, seed 0, 200 iterations."""
    g = gen.plain_small()
    inst = _inst(g)
    o = oracle.vns(inst, seed=0, iters=200, kmax=kmax, mode=mode)
    with E.Solver(g) as s:
        r = s.vns(seed=0, iters=200, kmax=kmax, mode=mode)
    np.testing.assert_array_equal(r["traj"]["it"], o.traj["it"])
    np.testing.assert_array_equal(r["traj"]["k"], o.traj["k"])
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    np.testing.assert_array_equal(r["traj"]["accepted"], o.traj["accepted"])
    _check_run(r, o)


@pytest.mark.parametrize("name,mk", [c for c in CASES if c[0] not in ("plain_small",)],
                         ids=[c[0] for c in CASES if c[0] not in ("plain_small",)])
def test_vns_edge_shapes(E, name, mk):
    g = mk()
    inst = _inst(g)
    iters = 40 if inst.K * inst.T < 1000 else 10
    o = oracle.vns(inst, seed=7, iters=iters, kmax=3, mode=0)
    with E.Solver(g) as s:
        r = s.vns(seed=7, iters=iters, kmax=3, mode=0)
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    _check_run(r, o)


def test_vns_medium_full_trajectory(E):
    """Plain VNS, K=50 products, T=52 periods, seed 1, 2000 iterations: the
    benchmark's workload and launch shape, compared entry by entry."""
    g = gen.plain_medium()
    inst = _inst(g)
    with E.Solver(g) as s:
        r = s.vns(seed=1, iters=2000, kmax=3, mode=0, plan=True)
    o = oracle.vns(inst, seed=1, iters=2000, kmax=3, mode=0)
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    np.testing.assert_array_equal(r["traj"]["accepted"], o.traj["accepted"])
    _check_run(r, o)
    for k in range(inst.K):
        c, plan = oracle.decode_row(inst, k, o.gM[k], o.gR[k])
        assert c != INF
        np.testing.assert_array_equal(r["plan"][:, k, :], plan)
    # the step counter: the sum of per-move decode steps of every evaluation
    assert r["segments"] > 0


def test_segments_equal_oracle_decode_steps(E):
    """The kernel's step counter equals the sum of the oracle's per-move
    decode steps over every neighbourhood evaluation of a VND."""
    g = gen.make_instance(31, 0, K=6, T=20)
    inst = _inst(g)
    gm, gr = oracle.initial_solution(inst.K, inst.T)
    total = 0
    # replay the oracle's mode-P VND, summing decode steps at each evaluation
    while True:
        imp = False
        for j in (1, 2, 3):
            per = oracle.row_moves(inst.T, j)
            for k in range(inst.K):
                for l in range(per):
                    total += oracle.decode_steps(inst, k, gm[k], gr[k], j, l)
            c = oracle.move_costs(inst, gm, gr, j).reshape(inst.K, per)
            _, rc = oracle.total_cost(inst, gm, gr)
            for k in range(inst.K):
                l = int(np.argmin(c[k]))
                if c[k, l] < rc[k]:
                    gm1, gr1 = gm[k:k + 1].copy(), gr[k:k + 1].copy()
                    oracle.apply_move(1, inst.T, j, l, gm1, gr1)
                    gm[k], gr[k] = gm1[0], gr1[0]
                    imp = True
        if not imp:
            break
    with E.Solver(g) as s:
        r = s.vns(seed=0, iters=0, kmax=3, mode=0)
    assert r["segments"] == total
    np.testing.assert_array_equal(r["gM"], gm)


def test_plan_matches_oracle_decode(E):
    g = gen.make_instance(17, 0, K=8, T=30)
    inst = _inst(g)
    with E.Solver(g) as s:
        r = s.vns(seed=3, iters=20, kmax=3, mode=0, plan=True)
    for k in range(inst.K):
        c, plan = oracle.decode_row(inst, k, r["gM"][k], r["gR"][k])
        np.testing.assert_array_equal(r["plan"][:, k, :], plan)


def test_multistart_best_of(E):
    """Independent starts with seeds seed0 + s; device best-of = the
    lexicographic (cost, start) minimum of the oracle's starts."""
    g = gen.make_instance(0, 0, K=12, T=26)
    inst = _inst(g)
    seeds = list(range(40, 56))
    best, outs = oracle.multistart(inst, seeds, iters=30, kmax=3, mode=0)
    with E.Solver(g) as s:
        bc, bs, costs = s.multistart(40, len(seeds), 30, 3, 0, costs=True)
        r = s.result(traj=False)
    np.testing.assert_array_equal(costs, [o.best_cost for o in outs])
    assert (bc, bs) == (outs[best].best_cost, best)
    np.testing.assert_array_equal(r["gM"], outs[best].gM)
    assert r["traj_hash"] == outs[best].traj_hash


def test_multistart_large_instance_sample(E):
    """Multi-start case: K=100, T=104 (seed 0, id 0), the same launch shape as
    the 4096-start workload; starts checked one by one against the oracle."""
    g = gen.multistart_large()
    inst = _inst(g)
    with E.Solver(g) as s:
        bc, bs, costs = s.multistart(0, 64, 3, 3, 0, costs=True)
    for sidx in (0, 37):
        o = oracle.vns(inst, seed=sidx, iters=3, kmax=3, mode=0)
        assert costs[sidx] == o.best_cost
    assert bc == costs.min() and bs == int(np.argmin(costs))


def test_batch_uneven_sample(E):
    """Batching: 1024 instances K ~ U{5..100}, T ~ U{12..52} in one persistent
    launch; a sample of instances checked one by one against the oracle."""
    insts = gen.batch_uneven(1024)
    seeds = np.arange(1024, dtype=np.uint64)
    b = E.Batch(insts)
    b.run(seeds, iters=60, kmax=3, mode=0)
    res = b.results()
    sizes = np.array([i.K * i.T for i in insts])
    sample = list(np.argsort(sizes)[:6]) + [int(np.argmax(sizes)), 500]
    for i in sample:
        inst = _inst(insts[i])
        o = oracle.vns(inst, seed=int(seeds[i]), iters=60, kmax=3, mode=0)
        assert res[i]["best_cost"] == o.best_cost, i
        assert res[i]["traj_hash"] == o.traj_hash, i
        gm, gr = b.solution(i)
        np.testing.assert_array_equal(gm, o.gM)
        np.testing.assert_array_equal(gr, o.gR)
    for r in res:
        assert r["status"] == 0 and r["iterations"] == 60
    b.close()


def test_batch_with_global_tables(E):
    """Instances too large for shared-memory prefix tables (K=200, T=104) use
    tables staged in global memory; parity with the oracle still holds."""
    insts = [gen.make_instance(9, i, K=200, T=104) for i in range(2)] + \
            [gen.make_instance(9, 5, K=7, T=13)]
    b = E.Batch(insts)
    b.run(np.array([3, 4, 5], np.uint64), iters=2, kmax=3, mode=0)
    res = b.results()
    for i, g in enumerate(insts):
        o = oracle.vns(_inst(g), seed=3 + i, iters=2, kmax=3, mode=0)
        assert res[i]["best_cost"] == o.best_cost
        assert res[i]["traj_hash"] == o.traj_hash
    b.close()


def test_staging_pass_rebuilds_the_same_tables(E):
    """The stage kernel finds each row's instance by binary search over the
    instances' first rows: 61 instances of 1..40 products (single-product
    instances at both ends and in the middle) and one that forces tables into
    global memory, staged explicitly and again after a run, give the oracle's
    results on every instance."""
    rng = np.random.default_rng(11)
    insts = [gen.make_instance(11, 0, K=1, T=9)]
    insts += [gen.make_instance(11, i, K=int(rng.integers(1, 41)), T=int(rng.integers(2, 60)))
              for i in range(1, 30)]
    insts += [gen.make_instance(11, 30, K=1, T=64), gen.make_instance(11, 31, K=200, T=104)]
    insts += [gen.make_instance(11, i, K=int(rng.integers(1, 41)), T=int(rng.integers(2, 60)))
              for i in range(32, 61)]
    insts += [gen.make_instance(11, 61, K=1, T=3)]
    seeds = np.arange(len(insts), dtype=np.uint64) + 40
    b = E.Batch(insts)
    b.stage_tables()
    b.run(seeds, iters=3, kmax=3, mode=0)
    first = [(r["best_cost"], r["traj_hash"]) for r in b.results()]
    assert b.launch_shape()["tables_in_smem"] == 0
    b.stage_tables()
    b.stage_tables()
    b.run(seeds, iters=3, kmax=3, mode=0)
    assert [(r["best_cost"], r["traj_hash"]) for r in b.results()] == first
    b.close()
    for i, g in enumerate(insts):
        o = oracle.vns(_inst(g), seed=int(seeds[i]), iters=3, kmax=3, mode=0)
        assert first[i] == (o.best_cost, o.traj_hash), i


def test_staging_pass_over_many_instances(E):
    """1100 small instances and one whose tables go to global memory (three
    levels of the stage kernel's 32-way search): a sample of runs, the first
    and last instances among them, equals the oracle."""
    rng = np.random.default_rng(12)
    insts = [gen.make_instance(12, i, K=int(rng.integers(1, 9)), T=int(rng.integers(2, 20)))
             for i in range(1100)]
    insts.insert(700, gen.make_instance(12, 5000, K=200, T=104))
    seeds = np.arange(len(insts), dtype=np.uint64)
    b = E.Batch(insts)
    b.stage_tables()
    b.run(seeds, iters=2, kmax=3, mode=0)
    res = b.results()
    assert b.launch_shape()["tables_in_smem"] == 0
    b.close()
    for i in [0, 1, 31, 32, 33, 699, 700, 701, 1023, 1024, 1025] + list(range(1090, 1101)):
        o = oracle.vns(_inst(insts[i]), seed=int(seeds[i]), iters=2, kmax=3, mode=0)
        assert (res[i]["best_cost"], res[i]["traj_hash"]) == (o.best_cost, o.traj_hash), i


SHAPES = [(4, 64, 1), (8, 256, 1), (16, 512, 1), (32, 512, 1), (16, 384, 1),
          (32, 64, 2), (16, 128, 3), (32, 224, 8), (8, 64, 16), (32, 32, 16),
          (64, 128, 1), (64, 448, 8), (128, 256, 4), (128, 512, 2), (64, 64, 16),
          (16, 1024, 1), (32, 768, 2), (64, 960, 1), (8, 1024, 3)]


@pytest.mark.parametrize("T", [40, 90])
def test_launch_shapes_give_identical_results(E, T):
    """Lanes per row, block size and CTAs per cluster change only speed."""
    g = gen.make_instance(2, 2, K=23, T=T)
    ref = None
    for lanes, threads, cluster in SHAPES:
        with E.Solver(g, lanes=lanes, threads=threads, cluster=cluster, speculation=1) as s:
            r = s.vns(seed=11, iters=50, kmax=3, mode=0)
            shape = s.launch_shape()
        assert shape["cluster"] == cluster and shape["threads"] == threads
        key = (r["best_cost"], r["traj_hash"], r["moves_evaluated"], r["segments"],
               r["applied"])
        if ref is None:
            ref = key
        assert key == ref, (lanes, threads, cluster)
        np.testing.assert_array_equal(r["traj"]["cost"][:5], r["traj"]["cost"][:5])


@pytest.mark.parametrize("teams,cluster", [(2, 1), (5, 2), (16, 8), (0, 0), (31, 4)])
def test_speculative_run_matches_oracle(E, teams, cluster):
    """Speculative teams commit iterations in order: the trajectory, solution
    and counters equal the sequential run's."""
    g = gen.make_instance(6, 1, K=20, T=30)
    inst = _inst(g)
    o = oracle.vns(inst, seed=9, iters=400, kmax=3, mode=0)
    with E.Solver(g, cluster=cluster, speculation=teams) as s:
        r = s.vns(seed=9, iters=400, kmax=3, mode=0)
        shape = s.launch_shape()
    if teams > 1:
        assert shape["teams"] > 1
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    np.testing.assert_array_equal(r["traj"]["k"], o.traj["k"])
    np.testing.assert_array_equal(r["traj"]["accepted"], o.traj["accepted"])
    _check_run(r, o)
    assert r["segments"] > 0


def test_speculation_counts_committed_work_only(E):
    """Work counters of a speculative run equal those of a one-team run."""
    g = gen.make_instance(6, 2, K=30, T=40)
    res = []
    for teams in (1, 12):
        with E.Solver(g, speculation=teams) as s:
            r = s.vns(seed=2, iters=300, kmax=3, mode=0)
        res.append((r["best_cost"], r["traj_hash"], r["moves_evaluated"], r["segments"],
                    r["applied"], r["vnd_cycles"], r["iterations"], r["accepted"]))
    assert res[0] == res[1]


def test_cluster_run_matches_oracle(E):
    """The medium plain workload on an 8-CTA cluster, 300 iterations."""
    g = gen.plain_medium()
    inst = _inst(g)
    o = oracle.vns(inst, seed=1, iters=300, kmax=3, mode=0)
    with E.Solver(g, cluster=8) as s:
        r = s.vns(seed=1, iters=300, kmax=3, mode=0)
        assert s.launch_shape()["cluster"] == 8
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    _check_run(r, o)


def test_invalid_state_rejected(E):
    g = gen.plain_small()
    with E.Solver(g) as s:
        bad = np.full((g.K, g.T), 2, np.uint8)
        with pytest.raises(E.nat.ElsrError if hasattr(E, "nat") else Exception):
            s.set_state(bad, bad)
        with pytest.raises(Exception):
            s.vns_run(0, 10, kmax=4)


def test_batch_small_instances_use_wide_row_groups(E):
    """A batch with automatic lanes gives each run its own row-group width
    (wider for instances with few products); every run still equals the
    oracle's.  Sizes from 2 to 40 products cover 16-, 32- and 128-lane
    groups in 1024-thread blocks."""
    insts = [gen.make_instance(13, i, K=k, T=t)
             for i, (k, t) in enumerate([(2, 12), (5, 40), (8, 52), (9, 20), (16, 33),
                                         (31, 52), (33, 12), (40, 52), (3, 64), (7, 65)])]
    b = E.Batch(insts, threads=1024)
    seeds = np.arange(len(insts), dtype=np.uint64) + 100
    b.run(seeds, iters=60, kmax=3, mode=0)
    res = b.results()
    for i, g in enumerate(insts):
        o = oracle.vns(_inst(g), seed=100 + i, iters=60, kmax=3, mode=0)
        assert res[i]["best_cost"] == o.best_cost, i
        assert res[i]["traj_hash"] == o.traj_hash, i
        assert res[i]["moves_evaluated"] == o.counters["moves_evaluated"], i
        gm, gr = b.solution(i)
        np.testing.assert_array_equal(gm, o.gM)
    b.close()


def test_eval_graph_replay_follows_state_launch_and_stream(E):
    """elsr_eval_neighbourhood replays a recorded CUDA graph per (mode, mask):
    its results follow the solution set between calls, a change of lanes per
    row records the graph again (both kernels of the evaluation), and a
    replay on another stream stays ordered after that stream's state copy."""
    import torch
    g = gen.make_instance(5, 9, K=21, T=44)
    inst = _inst(g)
    rng = np.random.default_rng(17)
    states = list(_states(rng, inst.K, inst.T, 4))
    side = torch.cuda.Stream()
    with E.Solver(g) as s:
        for step, lanes in enumerate((0, 8, 32, 0)):
            s.set_launch(lanes=lanes)
            if step == 3:
                s.set_stream(side)
            for gm, gr in states:
                s.set_state(gm, gr)
                for mode in (0, 1):
                    for mask in (7, 2, 7):
                        got = s.eval_neighbourhood(mask, mode)
                        bc, bm, pc, pm, _ = oracle.eval_neighbourhood(inst, gm, gr, mask, mode)
                        assert got[:2] == (bc, bm), (lanes, mode, mask)
                        np.testing.assert_array_equal(got[2], pc)
                        np.testing.assert_array_equal(got[3], pm)


def test_stream_switch_waits_for_work_in_flight(E):
    """A run queued on one stream, then the handle moved to another stream
    before the run has finished: the results read on the new stream are the
    finished run's (elsr_set_stream orders the new stream after the old)."""
    import torch
    g = gen.plain_medium()
    o = oracle.vns(_inst(g), seed=1, iters=400, kmax=3, mode=0)
    first, second = torch.cuda.Stream(), torch.cuda.Stream()
    with E.Solver(g, stream=first, speculation=1) as s:
        s.vns_run(1, 400, 3, 0)   # about 10 ms on one team: still running below
        s.set_stream(second)
        r = s.result()
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    _check_run(r, o)


def test_step_counter_switch_changes_no_result(E):
    """Runs timed with the decode-step counter off give the same trajectory,
    solution and every other counter, and report no steps; switched back on,
    the count is the oracle's again (single run and batch)."""
    g = gen.make_instance(8, 8, K=12, T=30)
    inst = _inst(g)
    with E.Solver(g) as s:
        on = s.vns(seed=4, iters=60, kmax=3, mode=0)
        s.set_count_steps(False)
        off = s.vns(seed=4, iters=60, kmax=3, mode=0)
        s.set_count_steps(True)
        again = s.vns(seed=4, iters=60, kmax=3, mode=0)
    keys = ("best_cost", "traj_hash", "moves_evaluated", "applied", "accepted", "vnd_cycles")
    assert [on[k] for k in keys] == [off[k] for k in keys] == [again[k] for k in keys]
    assert off["segments"] == 0 and on["segments"] == again["segments"] > 0
    np.testing.assert_array_equal(on["gM"], off["gM"])
    insts = gen.batch_uneven(12, seed=4)
    b = E.Batch(insts)
    seeds = np.arange(12, dtype=np.uint64)
    b.run(seeds, 20, 3, 0)
    r_on = b.results()
    b.set_count_steps(False)
    b.run(seeds, 20, 3, 0)
    r_off = b.results()
    assert [r["traj_hash"] for r in r_on] == [r["traj_hash"] for r in r_off]
    assert all(r["segments"] == 0 for r in r_off) and all(r["segments"] > 0 for r in r_on)
    b.close()
    o = oracle.vns(inst, seed=4, iters=60, kmax=3, mode=0)
    assert on["traj_hash"] == o.traj_hash
