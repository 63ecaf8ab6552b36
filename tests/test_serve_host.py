"""Serving-loop host logic that needs no GPU, with a stand-in for the
library's server.

* A request larger than the server's pools can never be admitted, so the
  loop refuses the stream before creating a server.
* The loop's invariants with a server that admits by footprint and retires
  requests after a few polls, out of order: every request served once with
  its own result, admissions in arrival order (a request that does not fit
  waits, and none overtakes it), resident bytes within the pools, several
  requests in flight at once, latency = completion - arrival."""
import pytest

from paper_1704_05132_gb300 import gen, serve


class _FakeNative:
    """Admits while slots, cells and rows last; a request retires on the
    poll after a number of polls that depends on its seed (so out of order);
    its result identifies it: cost = seed."""
    made = []

    def __init__(self, slots, cells, rows):
        self.slots, self.cells, self.rows = slots, cells, rows
        self.live = {}      # ticket -> [polls left, seed, K, T]
        self.next = 0
        self.order = []     # seeds in admission order
        self.max_cells = 0
        self.launches = 0
        self.closed = False
        _FakeNative.made.append(self)

    def _used(self):
        return (sum(K * T for _, _, K, T in self.live.values()),
                sum(K for _, _, K, _ in self.live.values()))

    def submit(self, inst, seed, iters, kmax=3, mode=0):
        K, T = inst.D.shape
        c, r = self._used()
        if len(self.live) >= self.slots or c + K * T > self.cells or r + K > self.rows:
            return None
        tk = self.next
        self.next += 1
        self.live[tk] = [50 + seed % 7, seed, K, T]
        self.order.append(seed)
        self.max_cells = max(self.max_cells, self._used()[0])
        self.launches += 1
        return tk

    def poll(self, max_n=1024):
        out = []
        for tk in list(self.live):
            self.live[tk][0] -= 1
            if self.live[tk][0] <= 0 and len(out) < max_n:
                _, seed, _, _ = self.live.pop(tk)
                out.append((tk, {"best_cost": seed, "traj_hash": 7 * seed,
                                 "moves_evaluated": 100 + seed, "status": 0}))
        return out

    def info(self):
        return len(self.live), self.launches

    def close(self):
        self.closed = True


def test_request_larger_than_the_pools_is_refused():
    small, big = gen.plain_small(), gen.make_instance(3, 4, K=200, T=104)
    reqs = [serve.Request(0, small, 0, 10, 0.0), serve.Request(1, big, 1, 10, 0.001)]
    _FakeNative.made = []
    srv = serve.Server(cells=200 * 104 - 1, native=_FakeNative)
    with pytest.raises(ValueError, match="request 1 .*more than the server's pools"):
        srv.run(reqs, realtime=False)
    assert _FakeNative.made == []   # refused before any server was made


def test_serving_loop_invariants_with_a_fake_server():
    from types import SimpleNamespace
    import numpy as np
    _FakeNative.made = []
    reqs = []
    for i in range(60):
        K = [5, 40, 160, 90, 200][i % 5]
        inst = SimpleNamespace(D=np.zeros((K, 20), np.int32))
        reqs.append(serve.Request(i, inst, seed=1000 + i, iters=30, arrival=0.0005 * i))
    srv = serve.Server(slots=6, cells=400 * 20, rows=10_000, native=_FakeNative)
    stats = srv.run(iter(reqs), realtime=True)   # any iterable
    fake = _FakeNative.made[0]
    got = {r.rid: r for r in stats.results}
    assert sorted(got) == list(range(60))
    for q in reqs:
        r = got[q.rid]
        assert r.best_cost == q.seed and r.moves_evaluated == 100 + q.seed
        assert r.done >= r.admitted >= r.arrival and r.latency == r.done - r.arrival
    assert fake.order == [q.seed for q in reqs]          # admitted in arrival order
    assert fake.max_cells <= 400 * 20                   # within the pools
    assert stats.max_resident_bytes <= serve.footprint(400, 20) + 16 * 400
    assert stats.max_inflight >= 2                       # requests overlap
    assert fake.closed and fake.live == {}
    retire = [r.rid for r in sorted(stats.results, key=lambda r: r.done)]
    assert retire != sorted(retire) or len(set(r.done for r in stats.results)) > 1


def test_empty_request_stream():
    """No requests: no server is made and the summary reports zero
    throughput and no latency percentiles."""
    _FakeNative.made = []
    stats = serve.Server(native=_FakeNative).run([], realtime=False)
    s = stats.summary()
    assert stats.results == [] and stats.batches == 0 and _FakeNative.made == []
    assert s["requests"] == 0 and s["p50_ms"] is None and s["instances_per_s"] == 0.0
