"""Instances per CTA (needs a GB300): a batched launch whose CTAs hold
several small runs at once, one per partition of their threads, gives every
run exactly the result it gets with one run per CTA and the oracle's.

The batch mixes runs that fit a partition's shared memory with runs that
need a whole CTA (those run first, one per CTA), in both table placements,
with mode P and mode G VND."""
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


def _key(r):
    return (r["status"], r["best_cost"], r["traj_hash"], r["moves_evaluated"], r["segments"],
            r["applied"], r["accepted"], r["iterations"])


def _mixed(n=60, seed=21):
    """Mostly small runs, a few that need a whole CTA (K*T near the limit)."""
    insts = [gen.make_instance(seed, i, K_range=(3, 30), T_range=(6, 40)) for i in range(n)]
    insts += [gen.make_instance(seed, 1000 + i, K=95, T=52) for i in range(3)]
    return insts


@pytest.mark.parametrize("mode", [0, 1])
def test_packed_batch_equals_unpacked_and_oracle(E, mode):
    insts = _mixed()
    seeds = np.arange(len(insts), dtype=np.uint64) + 7
    ref = None
    for threads, parts in [(1024, 1), (1024, 2), (1024, 4), (1024, 8), (512, 2), (512, 4),
                           (256, 2)]:
        b = E.Batch(insts, threads=threads, runs_per_cta=parts)
        b.run(seeds, iters=40, kmax=3, mode=mode)
        res = [_key(r) for r in b.results()]
        shape = b.launch_shape()
        if parts > 1 and threads >= 512:
            assert shape["runs_per_cta"] == parts, shape
            assert 0 < shape["whole_cta_runs"] < len(insts), shape
        elif parts > 1:  # blocks below 512 threads are not packed
            assert shape["runs_per_cta"] == 1, shape
        if ref is None:
            ref = res
            sols = [b.solution(i) for i in (0, len(insts) - 1)]
        assert res == ref, (threads, parts)
        gm, gr = b.solution(len(insts) - 1)
        np.testing.assert_array_equal(gm, sols[1][0])
        b.close()
    for i in list(range(0, len(insts), 9)) + [len(insts) - 1]:
        o = oracle.vns(oracle.Instance.from_arrays(insts[i]), int(seeds[i]), 40, 3, mode)
        assert ref[i][1:3] == (o.best_cost, o.traj_hash), i
        assert ref[i][3] == o.counters["moves_evaluated"], i


def test_packing_with_fixed_lanes_and_global_tables(E):
    """Fixed lanes per row (no per-run widening) and an instance whose prefix
    tables live in global memory, so every run of the launch does too."""
    insts = _mixed(24, seed=5) + [gen.make_instance(5, 77, K=75, T=100)]
    seeds = np.arange(len(insts), dtype=np.uint64)
    out = []
    for parts in (1, 4):
        b = E.Batch(insts, lanes=8, threads=1024, runs_per_cta=parts)
        b.run(seeds, iters=12, kmax=3, mode=0)
        out.append([_key(r) for r in b.results()])
        shape = b.launch_shape()
        assert shape["tables_in_smem"] == 0
        b.close()
    assert out[0] == out[1]
    o = oracle.vns(oracle.Instance.from_arrays(insts[3]), 3, 12, 3, 0)
    assert out[1][3][1:3] == (o.best_cost, o.traj_hash)


def test_runs_per_cta_must_be_a_power_of_two(E):
    insts = _mixed(4)
    b = E.Batch(insts)
    for bad in (-1, 3, 16):
        with pytest.raises(Exception):
            b.set_runs_per_cta(bad)
    b.close()
