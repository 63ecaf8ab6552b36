"""The allocation-free neighbourhood evaluation (elsr_eval_neighbourhood_static).

Callers that cannot allocate device memory (a framework owning all device
memory through its own pool, a serving loop that must never call cudaMalloc
or cudaFree) pass their own device buffers; the library keeps intermediate
data in a fixed device array.  This test calls the entry point through the C
ABI with device buffers owned by the test and checks, on two calls in a row
each time, that it returns exactly what the allocating entry point
elsr_eval_neighbourhood returns for the same solution (integer results, so
the tolerance is zero).  It runs last so that a failure here cannot hide
failures elsewhere, and it must pass alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

from paper_1704_05132_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_05132_gb300 import _native, build, elsr
    build.build()
    return torch, _native.load(), elsr


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _static_eval(torch, lib, g, gm, gr, mask, mode):
    i32, u8, i64 = torch.int32, torch.uint8, torch.int64
    args = [_dev(torch, getattr(g, f), i32) for f in ("D", "R", "kM", "kR", "hM", "hR")]
    dgm, dgr = _dev(torch, gm, u8), _dev(torch, gr, u8)
    best = torch.full((2,), -7, dtype=i64, device="cuda")
    pc = torch.full((g.K,), -7, dtype=i64, device="cuda")
    pm = torch.full((g.K,), -7, dtype=i64, device="cuda")
    stream = torch.cuda.current_stream()
    code = lib.elsr_eval_neighbourhood_static(
        g.K, g.T, *[_ptr(a) for a in args], _ptr(dgm), _ptr(dgr), mask, mode,
        _ptr(best), _ptr(pc), _ptr(pm), ctypes.c_void_p(stream.cuda_stream))
    assert code == 0
    torch.cuda.synchronize()
    return int(best[0]), int(best[1]), pc.cpu().numpy(), pm.cpu().numpy()


def _states(g, seed):
    rng = np.random.default_rng(seed)
    yield np.ones((g.K, g.T), np.uint8), np.ones((g.K, g.T), np.uint8)
    for i in range(2):
        gm = (rng.random((g.K, g.T)) < 0.5).astype(np.uint8)
        gr = (rng.random((g.K, g.T)) < 0.4).astype(np.uint8)
        gm[:, 0] = 1
        if i:
            gr &= gm
        yield gm, gr


@pytest.mark.parametrize("shape", [(5, 12), (50, 52), (13, 100), (7, 8), (9, 20), (11, 33)])
def test_static_eval_matches_allocating_entry_point(env, shape):
    torch, lib, elsr = env
    K, T = shape
    g = gen.make_instance(77, K, K=K, T=T)
    with elsr.Solver(g) as s:
        for gm, gr in _states(g, K):
            s.set_state(gm, gr)
            for mode in (0, 1):
                for mask in (7, 1, 6, 0):
                    ref = s.eval_neighbourhood(mask, mode)
                    for _ in range(2):  # two calls in a row share the array
                        got = _static_eval(torch, lib, g, gm, gr, mask, mode)
                        assert got[0] == ref[0] and got[1] == ref[1], (mode, mask)
                        np.testing.assert_array_equal(got[2], ref[2])
                        np.testing.assert_array_equal(got[3], ref[3])


def test_static_eval_rejects_oversize(env):
    torch, lib, _ = env
    null = ctypes.c_void_p(0)
    dummy = torch.zeros(8, dtype=torch.int32, device="cuda")
    p = _ptr(dummy)
    assert lib.elsr_eval_neighbourhood_static(4097, 10, p, p, p, p, p, p, p, p, 7, 0, p,
                                              null, null, null) == -2
    assert lib.elsr_eval_neighbourhood_static(3, 129, p, p, p, p, p, p, p, p, 7, 0, p,
                                              null, null, null) == -2
