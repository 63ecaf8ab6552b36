"""Host build of the CUDA path's row arithmetic vs the CPU oracle (no GPU).

``host_row_check.cpp`` compiles the kernels' ``elsr_row.cuh`` for the host.
These tests compare its delta re-decode (prefix tables, cached setups, the
recoverable-stock difference walk) element by element with the oracle's full
per-period decode, and its decode-step counts with the oracle's definition.  The GPU tests then check the
kernels that wrap the same header.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1704_05132_gb300 import gen

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1704_05132_gb300", "csrc")


# Set by tests/test_host_sanitized.py, which reruns this file with the
# harness built under AddressSanitizer and UBSan.
SANITIZE = os.environ.get("ELSR_HC_SANITIZE") == "1"


@pytest.fixture(scope="module")
def hc(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("hc") / "hc.so")
    opt = (["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
            "-fno-sanitize-recover=all"] if SANITIZE else ["-O2"])
    subprocess.check_call(["g++"] + opt + ["-std=c++17", "-shared", "-fPIC",
                           "-I", CSRC, os.path.join(HERE, "host_row_check.cpp"),
                           "-o", out])
    lib = ctypes.CDLL(out)
    P = ctypes.c_void_p
    lib.hc_move_costs.restype = ctypes.c_int64
    lib.hc_move_costs.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  P, P, P, P, P, ctypes.c_int32, P, P]
    lib.hc_swaps.restype = ctypes.c_int32
    lib.hc_swaps.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P]
    lib.hc_shake_draw.restype = ctypes.c_uint64
    lib.hc_shake_draw.argtypes = [ctypes.c_uint64] * 4
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _random_states(rng, T, n):
    """Mixture of structured and random setup patterns (feasible and not)."""
    for i in range(n):
        kind = i % 5
        if kind == 0:
            gm = np.ones(T, np.uint8)
            gr = np.ones(T, np.uint8)
        else:
            dm = rng.uniform(0.05, 0.8)
            dr = rng.uniform(0.05, 0.8)
            gm = (rng.random(T) < dm).astype(np.uint8)
            gr = (rng.random(T) < dr).astype(np.uint8)
            if kind in (1, 2):
                gm[0] = 1
            if kind == 2:
                gr &= gm
        yield gm, gr


@pytest.mark.parametrize("T", [1, 2, 3, 12, 52, 63, 64, 65, 104, 128])
@pytest.mark.parametrize("acc64,nw", [(0, 1), (1, 1), (0, 2), (1, 2)])
def test_delta_decode_matches_oracle(hc, T, acc64, nw):
    if nw == 1 and T > 64:
        pytest.skip("one 64-bit word holds at most 64 periods")
    rng = np.random.default_rng(T * 7 + acc64)
    g = gen.make_instance(50 + T, 1, K=1, T=T)
    if T % 3 == 0:
        g.D[0, : T // 3] = 0          # leading zero demand
    inst = oracle.Instance.from_arrays(g)
    costs = np.array([inst.kM[0], inst.kR[0], inst.hM[0], inst.hR[0], 0, 0], np.int32)
    D, R = inst.D[0].copy(), inst.R[0].copy()
    for gm, gr in _random_states(rng, T, 40):
        for j in (1, 2, 3):
            M = oracle.row_moves(T, j)
            if M <= 0:
                continue
            out = np.zeros(M, np.int64)
            segs = np.zeros(M, np.int32)
            cur = hc.hc_move_costs(acc64, nw, T, _p(D), _p(R), _p(costs), _p(gm), _p(gr),
                                   j, _p(out), _p(segs))
            assert cur == oracle.decode_row(inst, 0, gm, gr)[0]
            ref = oracle.move_costs(inst, gm[None, :], gr[None, :], j)
            np.testing.assert_array_equal(out, ref)
            win = [oracle.decode_steps(inst, 0, gm, gr, j, m) for m in range(M)]
            np.testing.assert_array_equal(segs, win)


def test_host_shake_draw_matches_oracle(hc):
    for args in [(0, 0, 1, 0), (5, 123, 3, 2), (2**63 + 11, 999, 2, 1)]:
        assert hc.hc_shake_draw(*args) == oracle.draw(*args)


def _first_shortfall(D, R, gm, gr):
    """First setup whose segment falls short (T: none, -1: demand before the
    first setup); used only to pick test cases."""
    T = len(D)
    y, seen = 0, False
    for t in range(T):
        if gm[t] or gr[t]:
            seen = True
            n = t + 1
            while n < T and not (gm[n] or gr[n]):
                n += 1
            need = int(D[t:n].sum())
            avail = y + int(R[t])
            xr = min(avail, need) if gr[t] else 0
            if not gm[t] and xr < need:
                return t
            y = avail - xr
        else:
            if not seen and D[t] > 0:
                return -1
            y += int(R[t])
    return T


@pytest.mark.parametrize("T", [16, 40, 64, 70])
def test_deficits_fixed_through_the_stock_difference(hc, T):
    """Rows that fall short at remanufacture-only setups late in the horizon.
    A move before the first shortfall fixes the row only if the extra stock
    it passes on covers every deficit after it; costs and step counts of every
    move still equal the oracle's full decode."""
    nw = 1 if T <= 64 else 2
    rng = np.random.default_rng(1000 + T)
    g = gen.make_instance(900 + T, 2, K=1, T=T)
    inst = oracle.Instance.from_arrays(g)
    costs = np.array([inst.kM[0], inst.kR[0], inst.hM[0], inst.hR[0], 0, 0], np.int32)
    D, R = inst.D[0].copy(), inst.R[0].copy()
    fixed_late = 0
    for trial in range(30):
        gm = np.ones(T, np.uint8)
        gr = (rng.random(T) < 0.6).astype(np.uint8)
        for p in rng.choice(np.arange(T // 2, T), size=int(rng.integers(1, 4)), replace=False):
            gm[p], gr[p] = 0, 1        # remanufacture-only, likely short
        bad = _first_shortfall(D, R, gm, gr)
        if bad < 0 or bad >= T:
            continue
        for j in (1, 2, 3):
            M = oracle.row_moves(T, j)
            for acc64 in (0, 1):
                out = np.zeros(M, np.int64)
                segs = np.zeros(M, np.int32)
                cur = hc.hc_move_costs(acc64, nw, T, _p(D), _p(R), _p(costs), _p(gm), _p(gr),
                                       j, _p(out), _p(segs))
                assert cur == oracle.INF
                np.testing.assert_array_equal(out, oracle.move_costs(inst, gm[None, :], gr[None, :], j))
                np.testing.assert_array_equal(
                    segs, [oracle.decode_steps(inst, 0, gm, gr, j, m) for m in range(M)])
            for m in range(M):
                nm, nr = gm[None, :].copy(), gr[None, :].copy()
                oracle.apply_move(1, T, j, m, nm, nr)
                changed = np.nonzero((nm[0] != gm) | (nr[0] != gr))[0]
                if len(changed) and changed.max() < bad and out[m] < oracle.INF:
                    fixed_late += 1
    assert fixed_late >= 3, "no move fixed a later deficit; the case is not exercised"


@pytest.mark.parametrize("T", [1, 2, 3, 31, 32, 33, 63, 64, 65, 96, 127, 128])
def test_non_null_swaps_by_rank(hc, T):
    """The N3 moves that change a row, listed by rank as the kernels take
    them: every swap of two differing neighbouring bits, gM row first, in
    index order; a null swap leaves the row (and its cost) unchanged."""
    rng = np.random.default_rng(T)
    g = gen.make_instance(70 + T, 3, K=1, T=T)
    inst = oracle.Instance.from_arrays(g)
    for nw in (1, 2):
        if nw == 1 and T > 64:
            continue
        for gm, gr in _random_states(rng, T, 12):
            out = np.zeros(max(2 * T, 1), np.int32)
            n = hc.hc_swaps(nw, T, _p(gm), _p(gr), _p(out))
            ref = [l for l in range(oracle.row_moves(T, 3))
                   if (l < T - 1 and gm[l] != gm[l + 1]) or
                   (l >= T - 1 and gr[l - T + 1] != gr[l - T + 2])]
            assert list(out[:n]) == ref
            if T > 1:
                costs = oracle.move_costs(inst, gm[None, :], gr[None, :], 3)
                cur = oracle.decode_row(inst, 0, gm, gr)[0]
                null = sorted(set(range(oracle.row_moves(T, 3))) - set(ref))
                assert all(costs[l] == cur for l in null)


@pytest.mark.parametrize("T", [3, 12, 52, 65, 104])
@pytest.mark.parametrize("acc64,nw", [(0, 1), (1, 2), (0, 2)])
def test_delta_decode_with_production_costs(hc, T, acc64, nw):
    """Unit production costs pM, pR (Algorithm 1's p_M, p_R): the delta
    re-decode against the oracle's per-period decode, with pR - pM of both
    signs and large enough to outweigh the holding saving hR*(T-t)."""
    if nw == 1 and T > 64:
        pytest.skip("one 64-bit word holds at most 64 periods")
    rng = np.random.default_rng(T * 11 + acc64 + 3 * nw)
    g = gen.make_instance(70 + T, 2, K=1, T=T)
    for pm, pr in [(10, 3), (3, 10), (0, 400), (500, 0), (37, 37)]:
        inst = oracle.Instance(g.D, g.R, g.kM, g.kR, g.hM, g.hR,
                               np.array([pm], np.int32), np.array([pr], np.int32))
        costs = np.array([inst.kM[0], inst.kR[0], inst.hM[0], inst.hR[0], pm, pr], np.int32)
        D, R = inst.D[0].copy(), inst.R[0].copy()
        for gm, gr in _random_states(rng, T, 12):
            for j in (1, 2, 3):
                M = oracle.row_moves(T, j)
                if M <= 0:
                    continue
                out = np.zeros(M, np.int64)
                segs = np.zeros(M, np.int32)
                cur = hc.hc_move_costs(acc64, nw, T, _p(D), _p(R), _p(costs), _p(gm), _p(gr),
                                       j, _p(out), _p(segs))
                assert cur == oracle.decode_row(inst, 0, gm, gr)[0]
                np.testing.assert_array_equal(out, oracle.move_costs(inst, gm[None, :],
                                                                     gr[None, :], j))


def _degenerate_rows(rng, T):
    """(name, D, R, [kM, kR, hM, hR, pM, pR]) rows of the degenerate kinds:
    no demand or returns, returns above demand, zero holding, zero setup
    costs, no cost at all, and returns above demand with pR < pM."""
    D = rng.integers(0, 101, T).astype(np.int32)
    R = (D * rng.integers(200, 601, T) // 1000).astype(np.int32)
    z = np.zeros(T, np.int32)
    more = (D + rng.integers(0, 30, T)).astype(np.int32)
    return [("empty", z, z, [310, 120, 3, 1, 0, 0]),
            ("returns_above_demand", D, more, [250, 140, 4, 2, 0, 0]),
            ("zero_holding", D, R, [260, 170, 0, 0, 0, 0]),
            ("zero_setup", D, R, [0, 0, 5, 2, 0, 0]),
            ("no_cost", D, R, [0, 0, 0, 0, 0, 0]),
            ("returns_above_demand_pR_below_pM", D, more, [250, 140, 4, 2, 90, 35])]


@pytest.mark.parametrize("T", [1, 12, 52, 64, 65, 104])
def test_degenerate_rows_match_oracle(hc, T):
    """The kernels' row arithmetic on degenerate rows (costs that tie, stock
    that only grows, rows with nothing to produce) against the oracle's full
    decode, per move, with 32- and 64-bit accumulators."""
    rng = np.random.default_rng(5000 + T)
    for name, D, R, c in _degenerate_rows(rng, T):
        inst = oracle.Instance(D[None, :], R[None, :], [c[0]], [c[1]], [c[2]], [c[3]],
                               [c[4]], [c[5]])
        costs = np.array(c, np.int32)
        for acc64, nw in [(0, 1), (1, 2)] if T <= 64 else [(0, 2), (1, 2)]:
            for gm, gr in _random_states(rng, T, 10):
                for j in (1, 2, 3):
                    M = oracle.row_moves(T, j)
                    if M <= 0:
                        continue
                    out = np.zeros(M, np.int64)
                    segs = np.zeros(M, np.int32)
                    cur = hc.hc_move_costs(acc64, nw, T, _p(D), _p(R), _p(costs), _p(gm),
                                           _p(gr), j, _p(out), _p(segs))
                    assert cur == oracle.decode_row(inst, 0, gm, gr)[0], name
                    ref = oracle.move_costs(inst, gm[None, :], gr[None, :], j)
                    np.testing.assert_array_equal(out, ref, err_msg=f"{name} j={j}")
                    win = [oracle.decode_steps(inst, 0, gm, gr, j, m) for m in range(M)]
                    np.testing.assert_array_equal(segs, win, err_msg=f"{name} j={j}")


def _golden(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([c.strip() for c in line.split("|")])
    return rows


def _golden_rows():
    """(name, D, R, [kM, kR, hM, hR, pM, pR], gM, gR, cost) of every hand-derived
    worked example, with and without unit production costs."""
    base = {r[0]: r for r in _golden("worked_examples.txt")}
    out = []
    for name, D, R, c, gm, gr, cost, *_ in base.values():
        out.append((name, D, R, c.split() + ["0", "0"], gm, gr, cost))
    for name, b, pc, _, _, cost in _golden("worked_examples_production.txt"):
        _, D, R, c, gm, gr, *_ = base[b]
        out.append((name, D, R, c.split() + pc.split(), gm, gr, cost))
    return out


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_kernel_row_cost_equals_hand_derivation(hc, row):
    """The kernels' row arithmetic gives each hand-derived example's cost
    directly (no oracle in between), with 32- and 64-bit accumulators and one
    or two words per bit row."""
    name, D, R, c, gm, gr, cost = row
    as_i32 = lambda s: np.array([int(v) for v in s.split()], np.int32)
    D, R, gm, gr = as_i32(D), as_i32(R), as_i32(gm).astype(np.uint8), as_i32(gr).astype(np.uint8)
    costs = np.array([int(v) for v in c], np.int32)
    T = len(D)
    want = oracle.INF if cost == "INF" else int(cost)
    for acc64, nw in [(0, 1), (1, 1), (0, 2), (1, 2)]:
        out = np.zeros(T, np.int64)
        segs = np.zeros(T, np.int32)
        got = hc.hc_move_costs(acc64, nw, T, _p(D), _p(R), _p(costs), _p(gm), _p(gr), 1,
                               _p(out), _p(segs))
        assert got == want, (name, acc64, nw)


def test_random_rows_property(hc):
    """Randomised rows (any T up to 128, zero or large costs, returns below
    or above demand, production costs of either sign of pR - pM, any setup
    pattern): the kernels' per-move costs and decode-step counts equal the
    oracle's.  Runs where hypothesis is installed."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=150, deadline=None, derandomize=True,
                  suppress_health_check=list(hyp.HealthCheck))
    @hyp.given(T=st.integers(1, 128), seed=st.integers(0, 2**32 - 1),
               kind=st.sampled_from(["plain", "zero_costs", "returns_above", "production",
                                     "sparse_demand"]))
    def check(T, seed, kind):
        rng = np.random.default_rng(seed)
        D = rng.integers(0, 101, T).astype(np.int32)
        if kind == "sparse_demand":
            D[rng.random(T) < 0.7] = 0
        R = (D * rng.integers(200, 601, T) // 1000).astype(np.int32)
        if kind == "returns_above":
            R = (D + rng.integers(0, 40, T)).astype(np.int32)
        c = [int(rng.integers(0, 501)), int(rng.integers(0, 401)), int(rng.integers(0, 7)),
             int(rng.integers(0, 4)), 0, 0]
        if kind == "zero_costs":
            c[int(rng.integers(0, 4))] = 0
            c[int(rng.integers(0, 4))] = 0
        if kind == "production":
            c[4], c[5] = int(rng.integers(0, 200)), int(rng.integers(0, 200))
        inst = oracle.Instance(D[None, :], R[None, :], [c[0]], [c[1]], [c[2]], [c[3]],
                               [c[4]], [c[5]])
        costs = np.array(c, np.int32)
        gm = (rng.random(T) < rng.uniform(0.05, 0.9)).astype(np.uint8)
        gr = (rng.random(T) < rng.uniform(0.05, 0.9)).astype(np.uint8)
        if rng.random() < 0.6:
            gm[0] = 1
        acc64 = int(rng.integers(0, 2))
        nw = 2 if T > 64 else int(rng.integers(1, 3))
        for j in (1, 2, 3):
            M = oracle.row_moves(T, j)
            if M <= 0:
                continue
            out = np.zeros(M, np.int64)
            segs = np.zeros(M, np.int32)
            cur = hc.hc_move_costs(acc64, nw, T, _p(D), _p(R), _p(costs), _p(gm), _p(gr), j,
                                   _p(out), _p(segs))
            assert cur == oracle.decode_row(inst, 0, gm, gr)[0]
            np.testing.assert_array_equal(out, oracle.move_costs(inst, gm[None, :], gr[None, :], j))
            win = [oracle.decode_steps(inst, 0, gm, gr, j, m) for m in range(M)]
            np.testing.assert_array_equal(segs, win)

    check()
