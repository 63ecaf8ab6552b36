"""Serving-loop host logic that needs no GPU.

* A request whose device footprint alone exceeds the memory budget can never
  be admitted, so the server refuses the stream before any launch instead of
  waiting for it.
* With fake batches, events and streams in place of the CUDA launches, the
  scheduler's invariants: every request served once with its own result,
  one iteration budget and at most max_batch requests per batch, small and
  cluster-sized requests in separate launches, resident bytes within the
  budget, and batches in flight at the same time."""
import pytest

from paper_1704_05132_gb300 import build, gen, serve


def _server(budget):
    # no CUDA streams are needed: the refusal comes before any admission
    srv = object.__new__(serve.Server)
    srv.torch = None
    srv.streams = []
    srv.mem_budget = budget
    srv.max_batch = 16
    srv.kmax = 3
    srv.mode = 0
    return srv


def test_request_above_the_memory_budget_is_refused():
    build.build()
    small, big = gen.plain_small(), gen.make_instance(3, 4, K=200, T=104)
    need_small = serve.footprint(small.K, small.T)[1]
    need_big = serve.footprint(big.K, big.T)[1]
    assert need_small < need_big
    reqs = [serve.Request(0, small, 0, 10, 0.0), serve.Request(1, big, 1, 10, 0.001)]
    with pytest.raises(ValueError, match="request 1 .*more than the budget"):
        serve.Server.run(_server(need_big - 1), reqs, realtime=False)


class _FakeEvent:
    """Completes on its third poll, so batches stay in flight for a while."""

    def __init__(self):
        self.polls = 0

    def record(self, stream):
        pass

    def query(self):
        self.polls += 1
        return self.polls > 2


class _FakeStream:
    def synchronize(self):
        pass


class _FakeBatch:
    made = []
    open_now = 0
    open_max = 0

    def __init__(self, insts, stream=None):
        self.insts, self.stream, self.closed = insts, stream, False
        _FakeBatch.made.append(self)

    def run(self, seeds, iters, kmax, mode):
        self.seeds, self.iters = [int(s) for s in seeds], iters
        _FakeBatch.open_now += 1
        _FakeBatch.open_max = max(_FakeBatch.open_max, _FakeBatch.open_now)

    def results(self):
        # a result that identifies its request: cost = seed
        return [{"best_cost": s, "traj_hash": 7 * s, "moves_evaluated": 100 + s, "status": 0}
                for s in self.seeds]

    def close(self):
        self.closed = True
        _FakeBatch.open_now -= 1


class _FakeCuda:
    Event = _FakeEvent

    @staticmethod
    def stream(s):
        import contextlib
        return contextlib.nullcontext()


class _FakeTorch:
    cuda = _FakeCuda


def test_scheduler_invariants_with_fake_batches(monkeypatch):
    """Every request is served once with its own result; a batch holds one
    iteration budget, at most max_batch requests, and small and large
    (cluster) requests in separate launches; resident bytes never exceed the
    budget; several batches overlap."""
    from types import SimpleNamespace
    monkeypatch.setattr(serve, "Batch", _FakeBatch)
    big_smem = serve.SMEM_ONE_CTA + 1
    monkeypatch.setattr(serve, "footprint",
                        lambda K, T: (big_smem if K >= 150 else 1024, 1000 * K))
    _FakeBatch.made, _FakeBatch.open_now, _FakeBatch.open_max = [], 0, 0
    reqs = []
    for i in range(60):
        K = [5, 40, 160, 90, 200][i % 5]
        reqs.append(serve.Request(i, SimpleNamespace(K=K, T=20), seed=1000 + i,
                                  iters=(30 if i % 3 else 45), arrival=0.0))
    srv = _server(budget=400_000)
    srv.torch = _FakeTorch
    srv.streams = [_FakeStream() for _ in range(3)]
    srv.max_batch = 7
    stats = serve.Server.run(srv, iter(reqs), realtime=False)   # any iterable
    got = {r.rid: r for r in stats.results}
    assert sorted(got) == list(range(60))
    for q in reqs:
        assert got[q.rid].best_cost == q.seed and got[q.rid].moves_evaluated == 100 + q.seed
    byseed = {q.seed: q for q in reqs}
    for b in _FakeBatch.made:
        members = [byseed[s] for s in b.seeds]
        assert len({m.iters for m in members}) == 1 and b.iters == members[0].iters
        assert len({m.inst.K >= 150 for m in members}) == 1     # small or large, not both
        assert b.closed
    assert stats.max_resident_bytes <= 400_000
    sizes = [len(b.seeds) for b in _FakeBatch.made]
    assert max(sizes) <= 7 and sum(sizes) == 60
    assert stats.batches >= 60 // 7
    assert _FakeBatch.open_max >= 2 and _FakeBatch.open_now == 0   # overlap, then drained


def test_empty_request_stream():
    """No requests: nothing is launched and the summary reports zero
    throughput and no latency percentiles."""
    srv = _server(budget=1 << 20)
    srv.streams = [_FakeStream()]
    stats = serve.Server.run(srv, [], realtime=False)
    s = stats.summary()
    assert stats.results == [] and stats.batches == 0
    assert s["requests"] == 0 and s["p50_ms"] is None and s["instances_per_s"] == 0.0
