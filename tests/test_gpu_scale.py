"""Parity at the sizes the workloads reach and at the limits of the move
index.

* The paper's benchmark shape (K = 300 products, T = 52 periods; its
  instances themselves are not available): a GVNS trajectory through the
  default launch, entry by entry against the oracle.
* K = 32,000 products of T = 128 periods, close to the 24-bit limit of
  the packed move index (K * 4T < 2^24): whole neighbourhoods evaluated on
  the device, checked on sampled moves that the oracle decodes one by one;
  a GVNS run of that size is refused (its rows exceed 16 CTAs of shared
  memory), and a mode-P VND at K = 1,000 is checked on sampled rows against
  the oracle's VND of that row alone (products are independent, Section 3).
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


def test_paper_shaped_trajectory(E):
    g = gen.paper_shaped()
    o = oracle.vns(oracle.Instance.from_arrays(g), seed=1, iters=60, kmax=3, mode=0)
    with E.Solver(g) as s:
        r = s.vns(seed=1, iters=60, kmax=3, mode=0)
        shape = s.launch_shape()
    assert shape["teams"] > 1 and shape["cluster"] == 16
    np.testing.assert_array_equal(r["traj"]["cost"], o.traj["cost"])
    assert r["best_cost"] == o.best_cost and r["traj_hash"] == o.traj_hash
    np.testing.assert_array_equal(r["gM"], o.gM)
    for key in ("moves_evaluated", "applied", "accepted"):
        assert r[key] == o.counters[key], key


@pytest.fixture(scope="module")
def huge():
    K, T = 32000, 128
    assert K * 4 * T < (1 << 24)
    return gen.make_instance(21, 0, K=K, T=T)


def _row_inst(g, k):
    return oracle.Instance(g.D[k:k + 1], g.R[k:k + 1], g.kM[k:k + 1], g.kR[k:k + 1],
                           g.hM[k:k + 1], g.hR[k:k + 1])


def test_index_limit_move_costs_sampled(E, huge):
    g = huge
    K, T = g.D.shape
    rng = np.random.default_rng(4)
    gm = (rng.random((K, T)) < 0.35).astype(np.uint8)
    gr = (rng.random((K, T)) < 0.35).astype(np.uint8)
    gm[:, 0] = 1
    with E.Solver(g) as s:
        s.set_state(gm, gr)
        for j in (1, 2, 3):
            c, _ = s.move_costs(j)
            per = oracle.row_moves(T, j)
            assert c.shape == (K * per,)
            for m in rng.choice(K * per, size=150, replace=False):
                k, l = divmod(int(m), per)
                inst = _row_inst(g, k)
                a, b = gm[k:k + 1].copy(), gr[k:k + 1].copy()
                oracle.apply_move(1, T, j, l, a, b)
                assert c[m] == oracle.decode_row(inst, 0, a[0], b[0])[0], (j, k, l)
        best, nimp, pc, pm = s.eval_neighbourhood(7, 0)
        for k in rng.choice(K, size=40, replace=False):
            ob = oracle.eval_neighbourhood(_row_inst(g, int(k)), gm[k:k + 1], gr[k:k + 1], 7, 0)
            assert (pc[k], pm[k]) == (ob[2][0], ob[3][0]), k


def test_index_limit_run_refused(E, huge):
    """A GVNS run keeps its rows in the shared memory of at most 16 CTAs; an
    instance beyond that is refused with an error, before any launch."""
    with E.Solver(huge) as s:
        with pytest.raises(E.nat.ElsrError) as ei:
            s.vns_run(0, 1, 3, 0)
        assert ei.value.code == E.nat.ELSR_E_RANGE


def test_large_run_vnd_rows_sampled(E):
    """Mode-P VND from every setup open at K = 1,000, T = 128 (16-CTA team,
    prefix tables in global memory): each sampled row equals the oracle's
    VND of that product alone."""
    g = gen.make_instance(21, 1, K=1000, T=128)
    K, T = g.D.shape
    with E.Solver(g) as s:
        r = s.vns(seed=0, iters=0, kmax=3, mode=0)
        shape = s.launch_shape()
    assert r["status"] == 0 and shape["cluster"] == 16 and shape["tables_in_smem"] == 0
    rng = np.random.default_rng(9)
    for k in rng.choice(K, size=12, replace=False):
        inst = _row_inst(g, int(k))
        gm0, gr0 = oracle.initial_solution(1, T)
        om, orr, _ = oracle.vnd(inst, gm0, gr0, 0)
        np.testing.assert_array_equal(r["gM"][k], om[0])
        np.testing.assert_array_equal(r["gR"][k], orr[0])
