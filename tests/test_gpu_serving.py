"""Serving with continuous batching (needs a GB300): every request's result
is the same as solving it alone (and the oracle's), admission waits for room
in the server's pools, and requests arriving while others run join them."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_05132_gb300 import build, elsr, serve
    build.build()
    return elsr, serve


def test_served_alone_equals_mixed(E):
    """Requests of every size class (one that needs a cluster of CTAs rides
    along) arrive while others run; each retires with exactly the result of
    the same run solved alone, and a sample equals the oracle's run."""
    import oracle
    elsr, serve = E
    from paper_1704_05132_gb300 import gen
    reqs = serve.poisson_requests(48, rate=4000.0, iters=25, seed=5)
    big = gen.make_instance(5, 999, K=200, T=104)
    reqs.append(serve.Request(999, big, 999, 25, reqs[10].arrival))
    stats = serve.Server(slots=64).run(reqs)
    assert len(stats.results) == len(reqs)
    assert stats.max_inflight > 3
    byid = {r.rid: r for r in stats.results}
    for q in reqs[:12] + [reqs[-1]]:
        with elsr.Solver(q.inst) as s:
            alone = s.vns(seed=q.seed, iters=q.iters, kmax=3, mode=0, traj=False, solution=False)
        got = byid[q.rid]
        assert got.status == 0
        assert (got.best_cost, got.traj_hash, got.moves_evaluated) == \
            (alone["best_cost"], alone["traj_hash"], alone["moves_evaluated"]), q.rid
    oracle.build()
    for q in reqs[:4]:
        o = oracle.vns(oracle.Instance.from_arrays(q.inst), q.seed, q.iters, 3, 0)
        got = byid[q.rid]
        assert (got.best_cost, got.traj_hash, got.moves_evaluated) == \
            (o.best_cost, o.traj_hash, o.counters["moves_evaluated"]), q.rid
    summ = stats.summary()
    assert summ["p99_ms"] >= summ["p50_ms"] > 0


def test_server_admits_by_footprint_and_keeps_solutions(E):
    """A server with room for two requests at a time: the third waits
    ("busy") until a retirement frees room; solutions are kept until
    released and equal the oracle's; steps are counted when asked."""
    import oracle
    elsr, serve = E
    from paper_1704_05132_gb300 import gen
    insts = [gen.make_instance(41, i, K=9 + i, T=20 + 3 * i) for i in range(5)]
    cells = max(g.K * g.T for g in insts) * 2
    srv = serve.NativeServer(slots=8, cells=cells, rows=10_000, count_steps=True,
                             keep_solutions=True)
    tickets, waiting, busy_seen = {}, list(range(5)), 0
    done = {}
    deadline = time.monotonic() + 60.0
    while len(done) < 5:
        assert time.monotonic() < deadline, "requests did not retire"
        while waiting:
            i = waiting[0]
            tk = srv.submit(insts[i], seed=100 + i, iters=15)
            if tk is None:
                busy_seen += 1
                break
            tickets[tk] = waiting.pop(0)
        for tk, st in srv.poll():
            i = tickets[tk]
            g = insts[i]
            # a kept solution stays readable until released, which frees room
            done[i] = (st, srv.solution(tk, g.K, g.T))
            srv.release(tk)
    assert busy_seen > 0
    oracle.build()
    for i, (st, (gm, gr)) in sorted(done.items()):
        g = insts[i]
        o = oracle.vns(oracle.Instance.from_arrays(g), 100 + i, 15, 3, 0)
        assert (st["best_cost"], st["traj_hash"]) == (o.best_cost, o.traj_hash)
        assert st["segments"] > 0
        np.testing.assert_array_equal(gm, o.gM)
        np.testing.assert_array_equal(gr, o.gR)
    assert srv.info()[0] == 0
    srv.close()


def test_batched_beats_plain_at_equal_budget(E):
    """Instances/s of the batched launch vs one plain run at a time, same
    instances and iteration budget."""
    import time
    import torch
    elsr, serve = E
    from paper_1704_05132_gb300 import gen
    insts = gen.batch_uneven(96, seed=3)
    seeds = np.arange(96, dtype=np.uint64)
    b = elsr.Batch(insts)
    b.run(seeds, 40, 3, 0)
    b.results()
    torch.cuda.synchronize()
    t = time.perf_counter()
    b.run(seeds, 40, 3, 0)
    res = b.results()
    tb = time.perf_counter() - t
    t = time.perf_counter()
    plain = []
    for i in range(16):
        with elsr.Solver(insts[i]) as s:
            plain.append(s.vns(seed=i, iters=40, kmax=3, mode=0, traj=False, solution=False))
    tp = (time.perf_counter() - t) / 16 * 96
    for i in range(16):
        assert plain[i]["best_cost"] == res[i]["best_cost"]
    assert tb < tp


def test_autotuner_picks_a_valid_shape_with_identical_results(E, tmp_path):
    elsr, serve = E
    from paper_1704_05132_gb300 import autotune, gen
    insts = gen.batch_uneven(64, seed=7)
    cache = str(tmp_path / "tune.json")
    shape = autotune.tune_batch(insts, probe_iters=3, cache_file=cache)
    assert shape in autotune.BATCH_CANDIDATES
    assert autotune.tune_batch(insts, cache_file=cache) == shape   # cached
    seeds = np.arange(64, dtype=np.uint64)
    ref = elsr.Batch(insts)
    ref.run(seeds, 15, 3, 0)
    tuned = elsr.Batch(insts, lanes=shape["lanes"], threads=shape["threads"],
                       cluster=shape["cluster"], runs_per_cta=shape["runs_per_cta"])
    looked_up = elsr.Batch(insts)       # every knob 0: the cached choice
    looked_up.run(seeds, 15, 3, 0)
    assert looked_up.launch_shape()["threads"] == shape["threads"]
    assert [r["traj_hash"] for r in looked_up.results()] == \
        [r["traj_hash"] for r in ref.results()]
    looked_up.close()
    tuned.run(seeds, 15, 3, 0)
    a, b = ref.results(), tuned.results()
    assert [(r["best_cost"], r["traj_hash"]) for r in a] == \
        [(r["best_cost"], r["traj_hash"]) for r in b]
    single = autotune.tune_single(gen.plain_small(), probe_iters=20,
                                  candidates=[dict(lanes=8, cluster=1, teams=1),
                                              dict(lanes=8, cluster=1, teams=4)])
    assert single["lanes"] == 8
