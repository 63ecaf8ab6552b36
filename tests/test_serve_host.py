"""Serving-loop host logic that needs no GPU: a request whose device
footprint alone exceeds the memory budget can never be admitted, so the
server refuses the stream before any launch instead of waiting for it."""
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
