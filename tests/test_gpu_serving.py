"""Serving with continuous batching (needs a GB300): every request's result
is the same as solving it alone, admission keeps resident device memory under
the budget, and requests arriving while others run are batched as slots free
up."""
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
    elsr, serve = E
    reqs = serve.poisson_requests(48, rate=4000.0, iters=25, seed=5)
    # one oversize instance that needs a CTA cluster rides along
    from paper_1704_05132_gb300 import gen
    big = gen.make_instance(5, 999, K=200, T=104)
    reqs.append(serve.Request(999, big, 999, 25, reqs[10].arrival))
    budget = 6 * max(serve.footprint(r.inst.K, r.inst.T)[1] for r in reqs)
    srv = serve.Server(slots=3, mem_budget=budget)
    stats = srv.run(reqs)
    assert len(stats.results) == len(reqs)
    assert stats.batches > 3
    assert stats.max_resident_bytes <= budget
    byid = {r.rid: r for r in stats.results}
    for q in reqs[:12] + [reqs[-1]]:
        with elsr.Solver(q.inst) as s:
            alone = s.vns(seed=q.seed, iters=q.iters, kmax=3, mode=0, traj=False, solution=False)
        got = byid[q.rid]
        assert got.status == 0
        assert (got.best_cost, got.traj_hash, got.moves_evaluated) == \
            (alone["best_cost"], alone["traj_hash"], alone["moves_evaluated"]), q.rid
    summ = stats.summary()
    assert summ["p99_ms"] >= summ["p50_ms"] > 0


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
                       cluster=shape["cluster"])
    tuned.run(seeds, 15, 3, 0)
    a, b = ref.results(), tuned.results()
    assert [(r["best_cost"], r["traj_hash"]) for r in a] == \
        [(r["best_cost"], r["traj_hash"]) for r in b]
    single = autotune.tune_single(gen.plain_small(), probe_iters=20,
                                  candidates=[dict(lanes=8, cluster=1, teams=1),
                                              dict(lanes=8, cluster=1, teams=4)])
    assert single["lanes"] == 8
