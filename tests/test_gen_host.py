"""The seeded input generator (no GPU).

* Its vectorised stream is splitmix64: from a state set to the published
  seed, the draws are the published reference outputs.
* Every drawn value lies in the range the recipe states, R = floor(D * p /
  1000) with p in 200..600, and variable-size instances draw K and T in
  their ranges.
* Streams are deterministic per (seed, id), independent across ids, and
  consecutive draws continue one stream.
"""
import os

import numpy as np

from paper_1704_05132_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_vectors.txt")


def test_stream_draws_are_published_splitmix64_outputs():
    with open(GOLDEN) as f:
        expected = [int(l) for l in f if l.strip() and not l.startswith("#")]
    s = gen.Stream(0, 0)
    s.state, s.pos = 1234567, 0
    assert [int(v) for v in s.draws(len(expected))] == expected


def test_consecutive_draws_continue_the_stream():
    a, b = gen.Stream(9, 4), gen.Stream(9, 4)
    whole = a.draws(12)
    parts = np.concatenate([b.draws(5), b.draws(7)])
    np.testing.assert_array_equal(whole, parts)


def _check_ranges(g):
    assert ((g.kM >= 200) & (g.kM <= 500)).all()
    assert ((g.kR >= 100) & (g.kR <= 400)).all()
    assert ((g.hM >= 2) & (g.hM <= 6)).all()
    assert ((g.hR >= 1) & (g.hR <= g.hM - 1)).all()
    assert ((g.D >= 0) & (g.D <= 100)).all()
    D = g.D.astype(np.int64)
    R = g.R.astype(np.int64)
    assert ((R >= (D * 200) // 1000) & (R <= (D * 600) // 1000)).all()
    for a in (g.D, g.R, g.kM, g.kR, g.hM, g.hR):
        assert a.dtype == np.int32 and a.flags.c_contiguous


def test_values_in_the_stated_ranges():
    for seed, ident in [(0, 0), (1, 0), (7, 3), (2**40 + 5, 99)]:
        _check_ranges(gen.make_instance(seed, ident, K=40, T=52))
    for g in gen.batch_uneven(64, seed=2):
        _check_ranges(g)
        assert 5 <= g.K <= 100 and 12 <= g.T <= 52
    for r in range(40):
        g = gen.serving_request(r)
        _check_ranges(g)
        assert 5 <= g.K <= 200 and 12 <= g.T <= 104
    # over many instances the whole stated range of the discrete draws is hit
    many = gen.batch_uneven(200, seed=4)
    assert {int(v) for g in many for v in g.hM} == {2, 3, 4, 5, 6}
    assert min(int(g.kM.min()) for g in many) == 200 and max(int(g.kM.max()) for g in many) == 500


def test_deterministic_per_seed_and_id():
    a, b = gen.make_instance(3, 7, K=9, T=20), gen.make_instance(3, 7, K=9, T=20)
    c = gen.make_instance(3, 8, K=9, T=20)
    for f in ("D", "R", "kM", "kR", "hM", "hR"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.D, c.D)
    # the workload instances are fixed by their (seed, id) and sizes
    m = gen.plain_medium()
    assert (m.K, m.T) == (50, 52)
    np.testing.assert_array_equal(m.D, gen.make_instance(1, 0, K=50, T=52).D)


def test_production_costs_in_range_and_both_signs():
    g = gen.with_production_costs(gen.make_instance(5, 0, K=60, T=20), 8)
    assert ((g.pM >= 10) & (g.pM <= 40)).all() and ((g.pR >= 0) & (g.pR <= 60)).all()
    d = g.pR.astype(np.int64) - g.pM
    assert (d > 0).any() and (d < 0).any()
    np.testing.assert_array_equal(g.D, gen.make_instance(5, 0, K=60, T=20).D)
