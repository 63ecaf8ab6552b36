"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test names what fixes the expected value: hand-derived worked examples
(tests/golden/worked_examples.txt), published splitmix64 outputs
(tests/golden/splitmix64_vectors.txt), the closed form of the all-open
initial solution, inventory invariants of Section 2's model, the
Wagner-Whitin dynamic program (Wagner & Whitin 1958) at K=1, R=0, brute force
over every setup pattern of tiny instances, and the product separability that
Section 3 states (the products do not interact).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1704_05132_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = oracle.INF


def _ints(s):
    return [int(v) for v in s.split()]


def _worked_examples():
    rows = []
    with open(os.path.join(GOLDEN, "worked_examples.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            p = [c.strip() for c in line.split("|")]
            rows.append(p)
    return rows


@pytest.mark.parametrize("row", _worked_examples(), ids=lambda r: r[0])
def test_worked_examples(row):
    name, D, R, costs, gM, gR, cost, xM, xR, yM, yR = row
    kM, kR, hM, hR = _ints(costs)
    inst = oracle.Instance(np.array([_ints(D)]), np.array([_ints(R)]),
                           [kM], [kR], [hM], [hR])
    c, plan = oracle.decode_row(inst, 0, np.array(_ints(gM)), np.array(_ints(gR)))
    if cost == "INF":
        assert c == INF
        return
    assert c == int(cost)
    assert plan[0].tolist() == _ints(xM)
    assert plan[1].tolist() == _ints(xR)
    assert plan[2].tolist() == _ints(yM)
    assert plan[3].tolist() == _ints(yR)


def test_splitmix64_published_vector():
    with open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) as f:
        expected = [int(l) for l in f if l.strip() and not l.startswith("#")]
    x = 1234567
    got = []
    for _ in expected:
        got.append(oracle.splitmix64(x))      # one step from state x
        x = (x + gen.GOLDEN) & ((1 << 64) - 1)
    assert got == expected
    # the generator module's independent splitmix64 gives the same stream
    assert [gen._mix_int((1234567 + i * gen.GOLDEN) & ((1 << 64) - 1))
            for i in range(len(expected))] == expected


def _check_plan(inst, k, gm, gr, cost, plan):
    """Invariants of Section 2's model on one decoded feasible row."""
    D, R = inst.D[k].astype(np.int64), inst.R[k].astype(np.int64)
    xM, xR, yM, yR = plan
    assert (plan >= 0).all()
    ym_prev = np.concatenate([[0], yM[:-1]])
    yr_prev = np.concatenate([[0], yR[:-1]])
    assert (yM == ym_prev + xM + xR - D).all()          # serviceable balance
    assert (yR == yr_prev + R - xR).all()               # recoverable balance
    assert ((xM == 0) | (gm == 1)).all()                # production needs a setup
    assert ((xR == 0) | (gr == 1)).all()
    assert yM[-1] == 0                                  # no stock left over
    assert xM.sum() + xR.sum() == D.sum()
    assert xR.sum() <= R.sum()
    setup = (gm | gr) == 1
    assert (ym_prev[setup] == 0).all()                  # zero-inventory ordering
    recomputed = (inst.kM[k] * gm.sum() + inst.kR[k] * gr.sum()
                  + inst.hM[k] * yM.sum() + inst.hR[k] * yR.sum())
    assert recomputed == cost


def test_invariants_random_patterns():
    rng = np.random.default_rng(7)
    inst = oracle.Instance.from_arrays(gen.make_instance(11, 0, K=6, T=20))
    n_feasible = 0
    for i in range(600):
        k = int(rng.integers(inst.K))
        dens = rng.uniform(0.1, 0.9)
        gm = (rng.random(inst.T) < dens).astype(np.uint8)
        gr = (rng.random(inst.T) < dens).astype(np.uint8)
        if i % 2:
            gr &= gm   # no remanufacture-only setups: feasible when gm[0] = 1
        gm[0] = 1 if rng.random() < 0.8 else gm[0]
        c, plan = oracle.decode_row(inst, k, gm, gr)
        if c == INF:
            continue
        n_feasible += 1
        _check_plan(inst, k, gm, gr, c, plan)
    assert n_feasible > 100


def test_infeasible_patterns_really_short():
    """A row reported infeasible has a period where the rule cannot cover
    demand: either demand before the first setup, or a remanufacture-only
    setup whose recoverable stock is below the demand it must cover."""
    rng = np.random.default_rng(3)
    inst = oracle.Instance.from_arrays(gen.make_instance(12, 0, K=1, T=10))
    D, R = inst.D[0].astype(np.int64), inst.R[0].astype(np.int64)
    for _ in range(300):
        gm = (rng.random(inst.T) < 0.3).astype(np.uint8)
        gr = (rng.random(inst.T) < 0.5).astype(np.uint8)
        c, _ = oracle.decode_row(inst, 0, gm, gr)
        setups = np.flatnonzero(gm | gr)
        first = setups[0] if len(setups) else inst.T
        pre_short = D[:first].sum() > 0
        # walk the setups by hand with stock only (no cost)
        short = pre_short
        yr = R[:first].sum() if not pre_short else 0
        if not pre_short:
            for i, s in enumerate(setups):
                n = setups[i + 1] if i + 1 < len(setups) else inst.T
                need = D[s:n].sum()
                avail = yr + R[s]
                xr = min(avail, need) if gr[s] else 0
                if not gm[s] and xr < need:
                    short = True
                    break
                yr = avail - xr + R[s + 1:n].sum()
        assert (c == INF) == short


def test_closed_form_all_open():
    """With R <= D and every setup open, no stock is ever held, so the cost of
    the initial solution is sum_k T * (kM + kR)."""
    for seed in range(5):
        g = gen.make_instance(seed, 3, K=7, T=15)
        assert (g.R <= g.D).all()
        inst = oracle.Instance.from_arrays(g)
        gm, gr = oracle.initial_solution(inst.K, inst.T)
        total, _ = oracle.total_cost(inst, gm, gr)
        assert total == int((inst.T * (inst.kM.astype(np.int64) + inst.kR)).sum())


def _wagner_whitin(D, kM, hM):
    """Textbook uncapacitated lot-sizing DP: F[t] = min cost of periods [0, t)."""
    T = len(D)
    F = [0] + [None] * T
    for t in range(1, T + 1):
        best = 0 if sum(D[:t]) == 0 else None
        for s in range(t):
            if F[s] is None:
                continue
            c = F[s] + kM + hM * sum(D[i] * (i - s) for i in range(s, t))
            best = c if best is None else min(best, c)
        F[t] = best
    return F[T]


@pytest.mark.parametrize("seed", range(4))
def test_wagner_whitin_reduction(seed):
    """K=1, R=0: the best decoded gM pattern (gR = 0) equals the Wagner-Whitin
    optimum, and so does the best over all (gM, gR) pairs for T <= 8."""
    rng = np.random.default_rng(100 + seed)
    T = 12 if seed < 2 else 8
    D = rng.integers(0, 40, T)
    if seed == 1:
        D[:3] = 0   # leading zero demand
    kM, hM = int(rng.integers(20, 200)), int(rng.integers(1, 5))
    inst = oracle.Instance(D[None, :], np.zeros((1, T), np.int64), [kM], [57], [hM], [1])
    ww = _wagner_whitin(list(D), kM, hM)
    zeros = np.zeros(T, np.uint8)
    best = min(oracle.decode_row(inst, 0, np.array(p, np.uint8), zeros)[0]
               for p in itertools.product((0, 1), repeat=T))
    assert best == ww
    if T <= 8:
        best2 = min(oracle.decode_row(inst, 0, np.array(p[:T], np.uint8),
                                      np.array(p[T:], np.uint8))[0]
                    for p in itertools.product((0, 1), repeat=2 * T))
        assert best2 == ww


def _brute_force_row(inst, k):
    T = inst.T
    best = INF
    for p in itertools.product((0, 1), repeat=2 * T):
        c, _ = oracle.decode_row(inst, k, np.array(p[:T], np.uint8), np.array(p[T:], np.uint8))
        best = min(best, c)
    return best


@pytest.mark.parametrize("seed", range(3))
def test_vns_not_below_brute_force(seed):
    g = gen.make_instance(20 + seed, 0, K=2, T=6)
    inst = oracle.Instance.from_arrays(g)
    opt = sum(_brute_force_row(inst, k) for k in range(inst.K))
    for mode in (0, 1):
        res = oracle.vns(inst, seed=seed, iters=30, kmax=3, mode=mode)
        assert res.best_cost >= opt
        # the reported cost is the cost of the returned solution
        assert oracle.total_cost(inst, res.gM, res.gR)[0] == res.best_cost


def _is_local_optimum(inst, gm, gr, mode):
    total, rc = oracle.total_cost(inst, gm, gr)
    for j in (1, 2, 3):
        c = oracle.move_costs(inst, gm, gr, j)
        per = oracle.row_moves(inst.T, j)
        if per == 0:
            continue
        c = c.reshape(inst.K, per)
        if mode == 0:
            if (c < rc[:, None]).any():
                return False
        else:
            others = total - rc[:, None]
            if ((others + c)[c != INF] < total).any():
                return False
    return True


@pytest.mark.parametrize("mode", [0, 1])
def test_vnd_reaches_local_optimum(mode):
    inst = oracle.Instance.from_arrays(gen.make_instance(4, 0, K=4, T=14))
    gm, gr = oracle.initial_solution(inst.K, inst.T)
    t0 = oracle.total_cost(inst, gm, gr)[0]
    gm2, gr2, cnt = oracle.vnd(inst, gm, gr, mode)
    t1 = oracle.total_cost(inst, gm2, gr2)[0]
    assert t1 < t0
    assert _is_local_optimum(inst, gm2, gr2, mode)
    per_cycle = sum(oracle.nb_size(inst.K, inst.T, j) for j in (1, 2, 3))
    assert cnt["moves_evaluated"] == cnt["vnd_cycles"] * per_cycle
    assert cnt["evals"] == 3 * cnt["vnd_cycles"]


def test_vnd_mode_p_separable():
    """Products are uncoupled (Section 3), so the product-parallel VND of
    Algorithm 1 gives, row by row, the VND of each product alone."""
    g = gen.make_instance(8, 0, K=6, T=18)
    inst = oracle.Instance.from_arrays(g)
    gm, gr = oracle.initial_solution(inst.K, inst.T)
    gm2, gr2, cnt = oracle.vnd(inst, gm, gr, 0)
    cycles = []
    for k in range(inst.K):
        sub = inst.row(k)
        a, b, c = oracle.vnd(sub, gm[k:k + 1], gr[k:k + 1], 0)
        assert (a[0] == gm2[k]).all() and (b[0] == gr2[k]).all()
        cycles.append(c["vnd_cycles"])
    assert cnt["vnd_cycles"] == max(cycles)


def test_move_layout_hand_cases():
    """Neighbourhood index layout on a hand-made 2 x 4 solution."""
    K, T = 2, 4
    gm = np.array([[1, 0, 0, 1], [0, 1, 1, 0]], np.uint8)
    gr = np.array([[0, 0, 1, 0], [1, 0, 0, 0]], np.uint8)
    assert oracle.nb_size(K, T, 1) == 8 and oracle.nb_size(K, T, 3) == 12
    a, b = gm.copy(), gr.copy()
    oracle.apply_move(K, T, 1, 6, a, b)            # N1: flip gM(1, 2)
    assert a[1].tolist() == [0, 1, 0, 0] and (b == gr).all()
    a, b = gm.copy(), gr.copy()
    oracle.apply_move(K, T, 2, 3, a, b)            # N2: flip gR(0, 3)
    assert b[0].tolist() == [0, 0, 1, 1] and (a == gm).all()
    a, b = gm.copy(), gr.copy()
    oracle.apply_move(K, T, 3, 6 + 0, a, b)        # N3 row 1, c=M, t=0: swap
    assert a[1].tolist() == [1, 0, 1, 0]
    a, b = gm.copy(), gr.copy()
    oracle.apply_move(K, T, 3, 0 * 6 + 3 + 1, a, b)  # N3 row 0, c=R, t=1
    assert b[0].tolist() == [0, 1, 0, 0]


def test_shake_follows_draws():
    """Shake(x, k) applies k moves of N_k indexed by the splitmix64 draws;
    the expected indices use the generator module's own splitmix64."""
    K, T = 5, 9
    mix = gen._mix_int
    for seed, it, k in [(0, 0, 1), (3, 17, 2), (99, 5, 3)]:
        gm = np.zeros((K, T), np.uint8)
        gr = np.zeros((K, T), np.uint8)
        gm[:, ::2] = 1
        gr[:, 1::3] = 1
        a, b = gm.copy(), gr.copy()
        oracle.shake(K, T, a, b, seed, it, k)
        size = oracle.nb_size(K, T, k)
        for j in range(k):
            d = mix(mix(mix(seed) ^ it) ^ ((k << 32) | j))
            assert d == oracle.draw(seed, it, k, j)
            oracle.apply_move(K, T, k, d % size, gm, gr)
        assert (a == gm).all() and (b == gr).all()


def test_gvns_trajectory_rules():
    inst = oracle.Instance.from_arrays(gen.plain_small())
    res = oracle.vns(inst, seed=0, iters=200, kmax=3, mode=0)
    gm, gr = oracle.initial_solution(inst.K, inst.T)
    gm, gr, _ = oracle.vnd(inst, gm, gr, 0)
    fx = oracle.total_cost(inst, gm, gr)[0]
    k = 1
    for e in res.traj:
        assert e["k"] == k
        acc = e["cost"] < fx
        assert bool(e["accepted"]) == acc
        if acc:
            fx, k = int(e["cost"]), 1
        else:
            k = k + 1 if k < 3 else 1
    assert fx == res.best_cost
    assert res.counters["iterations"] == 200
    assert res.counters["accepted"] == int(res.traj["accepted"].sum())


def test_eval_neighbourhood_matches_move_costs():
    inst = oracle.Instance.from_arrays(gen.make_instance(9, 0, K=3, T=7))
    rng = np.random.default_rng(1)
    gm = (rng.random((3, 7)) < 0.5).astype(np.uint8)
    gr = (rng.random((3, 7)) < 0.5).astype(np.uint8)
    gm[:, 0] = 1
    total, rc = oracle.total_cost(inst, gm, gr)
    bc, bm, pc, pm, n = oracle.eval_neighbourhood(inst, gm, gr, 0b111, 1)
    allc = []
    for j in (1, 2, 3):
        c = oracle.move_costs(inst, gm, gr, j).reshape(3, -1)
        allc.append(c)
    assert n == sum(c.size for c in allc)
    for k in range(3):
        row = np.concatenate([c[k] for c in allc])
        assert pc[k] == row.min() and pm[k] == int(np.argmin(row))


# ---------------------------------------------------------------------------
# Fork-join GVNS (Algorithm 2 with one shake + VND per worker, the minimum
# kept: the paper's two-GPU scheme of Section 3).
# ---------------------------------------------------------------------------

def test_shake_worker_follows_draws():
    """Worker p's shake applies the moves drawn with key p << 8 | j (the
    generator module's own splitmix64 recomputes them); worker 0 is the
    sequential shake."""
    K, T = 4, 11
    mix = gen._mix_int
    for seed, it, k, p in [(0, 0, 1, 0), (5, 3, 2, 1), (77, 40, 3, 6), (1, 9, 3, 255)]:
        gm = np.zeros((K, T), np.uint8)
        gr = np.zeros((K, T), np.uint8)
        gm[:, ::3] = 1
        gr[:, 1::2] = 1
        a, b = gm.copy(), gr.copy()
        oracle.shake_worker(K, T, a, b, seed, it, k, p)
        size = oracle.nb_size(K, T, k)
        for j in range(k):
            d = mix(mix(mix(seed) ^ it) ^ ((k << 32) | (p << 8) | j))
            oracle.apply_move(K, T, k, d % size, gm, gr)
        assert (a == gm).all() and (b == gr).all()
        if p == 0:
            c, d2 = a.copy(), b.copy()
            oracle.shake(K, T, a, b, seed, it, k)
            oracle.shake_worker(K, T, c, d2, seed, it, k, 0)
            assert (a == c).all() and (b == d2).all()


@pytest.mark.parametrize("mode", [0, 1])
def test_forkjoin_one_worker_is_sequential_gvns(mode):
    inst = oracle.Instance.from_arrays(gen.plain_small())
    a = oracle.vns(inst, seed=4, iters=150, kmax=3, mode=mode)
    b = oracle.vns_forkjoin(inst, seed=4, iters=150, kmax=3, mode=mode, workers=1)
    assert a.best_cost == b.best_cost and a.traj_hash == b.traj_hash
    assert a.counters == b.counters
    assert (a.gM == b.gM).all() and (a.gR == b.gR).all()
    assert (a.traj["cost"] == b.traj["cost"]).all() and (b.traj["pad"] == 0).all()


@pytest.mark.parametrize("mode,workers", [(0, 3), (1, 2), (0, 5)])
def test_forkjoin_iterations_recomposed(mode, workers):
    """Each logged iteration equals the minimum over workers of
    f(VND(Shake_p(x, k))), recomputed here from the separately pinned
    shake, VND and objective; acceptance, k and the incumbent follow the
    rules of Algorithm 2."""
    inst = oracle.Instance.from_arrays(gen.make_instance(31, 2, K=4, T=10))
    iters = 25
    res = oracle.vns_forkjoin(inst, seed=8, iters=iters, kmax=3, mode=mode, workers=workers)
    gm, gr = oracle.initial_solution(inst.K, inst.T)
    gm, gr, cnt0 = oracle.vnd(inst, gm, gr, mode)
    fx = oracle.total_cost(inst, gm, gr)[0]
    k = 1
    moves = cnt0["moves_evaluated"]
    for it in range(iters):
        cands = []
        for p in range(workers):
            a, b = gm.copy(), gr.copy()
            oracle.shake_worker(inst.K, inst.T, a, b, 8, it, k, p)
            a, b, c = oracle.vnd(inst, a, b, mode)
            moves += c["moves_evaluated"]
            cands.append((oracle.total_cost(inst, a, b)[0], p, a, b))
        f2, p, a, b = min(cands, key=lambda c: (c[0], c[1]))
        e = res.traj[it]
        assert (e["it"], e["k"], e["cost"], e["pad"]) == (it, k, f2, p)
        assert bool(e["accepted"]) == (f2 < fx)
        if f2 < fx:
            gm, gr, fx, k = a, b, f2, 1
        else:
            k = k + 1 if k < 3 else 1
    assert res.best_cost == fx
    assert (res.gM == gm).all() and (res.gR == gr).all()
    assert res.counters["moves_evaluated"] == moves
    assert res.counters["iterations"] == iters


@pytest.mark.parametrize("seed", range(2))
def test_forkjoin_not_below_brute_force(seed):
    g = gen.make_instance(40 + seed, 0, K=2, T=5)
    inst = oracle.Instance.from_arrays(g)
    opt = sum(_brute_force_row(inst, k) for k in range(inst.K))
    for mode in (0, 1):
        res = oracle.vns_forkjoin(inst, seed=seed, iters=20, kmax=3, mode=mode, workers=4)
        assert res.best_cost >= opt
        assert oracle.total_cost(inst, res.gM, res.gR)[0] == res.best_cost
        acc = res.traj["cost"][res.traj["accepted"] == 1]
        assert (np.diff(acc) < 0).all()


# ---------------------------------------------------------------------------
# Unit production costs p_M, p_R (Algorithm 1's signature).
# ---------------------------------------------------------------------------

def _worked_examples_production():
    base = {r[0]: r for r in _worked_examples()}
    rows = []
    with open(os.path.join(GOLDEN, "worked_examples_production.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            p = [c.strip() for c in line.split("|")]
            rows.append((p, base[p[1]]))
    return rows


@pytest.mark.parametrize("row", _worked_examples_production(), ids=lambda r: r[0][0])
def test_worked_examples_with_production_costs(row):
    (name, _, pc, sxm, sxr, cost), b = row
    pm, pr = _ints(pc)
    kM, kR, hM, hR = _ints(b[3])
    inst = oracle.Instance(np.array([_ints(b[1])]), np.array([_ints(b[2])]),
                           [kM], [kR], [hM], [hR], [pm], [pr])
    c, plan = oracle.decode_row(inst, 0, np.array(_ints(b[4])), np.array(_ints(b[5])))
    if cost == "INF":
        assert c == INF
        return
    assert c == int(cost)
    assert int(plan[0].sum()) == int(sxm) and int(plan[1].sum()) == int(sxr)


def test_closed_form_all_open_with_production_costs():
    """Every setup open and R <= D: xR(t) = R(t), xM(t) = D(t) - R(t) and no
    stock is held, so the cost is sum_k T(kM + kR) + pM sum D + (pR - pM) sum R."""
    for seed in range(4):
        g = gen.with_production_costs(gen.make_instance(seed, 5, K=6, T=13), seed, 9)
        inst = oracle.Instance.from_arrays(g)
        gm, gr = oracle.initial_solution(inst.K, inst.T)
        total, _ = oracle.total_cost(inst, gm, gr)
        i64 = lambda a: a.astype(np.int64)
        want = (inst.T * (i64(inst.kM) + inst.kR) + i64(inst.pM) * i64(inst.D).sum(1)
                + (i64(inst.pR) - inst.pM) * i64(inst.R).sum(1)).sum()
        assert total == int(want)


@pytest.mark.parametrize("mode", [0, 1])
def test_equal_production_costs_shift_every_feasible_cost(mode):
    """pM = pR = p adds p * sum D to every feasible row whatever its setups
    (xM + xR covers the demand), so GVNS takes the same steps and every
    feasible trajectory cost moves by p * sum D."""
    g = gen.make_instance(17, 1, K=6, T=16)
    base = oracle.vns(oracle.Instance.from_arrays(g), seed=3, iters=60, kmax=3, mode=mode)
    p = np.full(6, 23, np.int32)
    inst = oracle.Instance(g.D, g.R, g.kM, g.kR, g.hM, g.hR, p, p)
    res = oracle.vns(inst, seed=3, iters=60, kmax=3, mode=mode)
    shift = 23 * int(g.D.astype(np.int64).sum())
    assert (res.gM == base.gM).all() and (res.gR == base.gR).all()
    assert res.best_cost == base.best_cost + shift
    feas = base.traj["cost"] != INF
    assert (res.traj["cost"][feas] == base.traj["cost"][feas] + shift).all()
    assert (res.traj["cost"][~feas] == INF).all()


@pytest.mark.parametrize("seed", range(3))
def test_wagner_whitin_with_manufacturing_cost(seed):
    """K=1, R=0: every unit is manufactured, so the best gM pattern costs the
    Wagner-Whitin optimum plus pM * sum D (pR plays no part)."""
    rng = np.random.default_rng(100 + seed)
    T = 9
    D = rng.integers(0, 30, T).astype(np.int32)
    kM, hM, pm = int(rng.integers(20, 90)), int(rng.integers(1, 5)), int(rng.integers(1, 20))
    ww = _wagner_whitin(D.tolist(), kM, hM)
    inst = oracle.Instance(D[None, :], np.zeros((1, T), np.int32), [kM], [50], [hM], [1],
                           [pm], [int(rng.integers(0, 50))])
    zeros = np.zeros(T, np.uint8)
    best = min(oracle.decode_row(inst, 0, np.array(p, np.uint8), zeros)[0]
               for p in itertools.product((0, 1), repeat=T))
    assert best == ww + pm * int(D.sum())


# ---------------------------------------------------------------------------
# Degenerate instances: closed forms that hold whatever the decode's steps.
# ---------------------------------------------------------------------------

def test_closed_form_returns_exceed_demand():
    """R >= D in every period and every gR open: returns cover all demand,
    nothing is manufactured (yM = 0), and the returns stock after period t is
    sum_{i<=t} (R_i - D_i), so a row costs
    kM * |gM| + T * kR + hR * sum_i (R_i - D_i) * (T - i), whatever gM is."""
    rng = np.random.default_rng(7)
    K, T = 4, 11
    D = rng.integers(0, 60, (K, T))
    R = D + rng.integers(0, 25, (K, T))
    kM, kR = rng.integers(50, 300, K), rng.integers(50, 300, K)
    hM, hR = rng.integers(1, 6, K), rng.integers(1, 4, K)
    inst = oracle.Instance(D, R, kM, kR, hM, hR)
    gr = np.ones((K, T), np.uint8)
    w = np.arange(T, 0, -1)
    for trial in range(6):
        gm = (rng.random((K, T)) < 0.4).astype(np.uint8)
        _, rc = oracle.total_cost(inst, gm, gr)
        for k in range(K):
            want = kM[k] * gm[k].sum() + T * kR[k] + hR[k] * ((R[k] - D[k]) * w).sum()
            assert rc[k] == want, (trial, k)
            _, plan = oracle.decode_row(inst, k, gm[k], gr[k])
            assert (plan[0] == 0).all() and (plan[2] == 0).all()   # xM = yM = 0


def test_zero_demand_and_returns():
    """D = R = 0: every setup pattern is feasible and costs only its setups,
    kM * |gM| + kR * |gR|; with positive setup costs the unique local optimum
    of every neighbourhood is the empty pattern, so VND from all open and
    GVNS end there at cost 0, in both modes."""
    K, T = 3, 9
    z = np.zeros((K, T), np.int64)
    kM, kR = np.array([40, 7, 300]), np.array([1, 90, 33])
    inst = oracle.Instance(z, z, kM, kR, [3, 1, 2], [1, 1, 1])
    rng = np.random.default_rng(3)
    for _ in range(5):
        gm = (rng.random((K, T)) < 0.5).astype(np.uint8)
        gr = (rng.random((K, T)) < 0.5).astype(np.uint8)
        _, rc = oracle.total_cost(inst, gm, gr)
        assert (rc == kM * gm.sum(1) + kR * gr.sum(1)).all()
    gm0, gr0 = oracle.initial_solution(K, T)
    for mode in (0, 1):
        gm, gr, _ = oracle.vnd(inst, gm0, gr0, mode)
        assert not gm.any() and not gr.any()
        res = oracle.vns(inst, seed=5, iters=25, kmax=3, mode=mode)
        assert res.best_cost == 0 and res.counters["accepted"] == 0


def test_ties_go_to_the_lowest_index():
    """Two identical products with D = R = 0 and gM = 0110: dropping either
    open setup saves kM, every other N1 move costs more, so the per-product
    best N1 move is t = 1 (not t = 2), and the global best is product 0's
    (index 1, not product 1's index 5)."""
    T, kM = 4, 100
    z = np.zeros((2, T), np.int64)
    inst = oracle.Instance(z, z, [kM, kM], [60, 60], [1, 1], [1, 1])
    gm = np.array([[0, 1, 1, 0]] * 2, np.uint8)
    gr = np.zeros((2, T), np.uint8)
    _, _, pc, pm, _ = oracle.eval_neighbourhood(inst, gm, gr, 1, 0)
    assert pc.tolist() == [kM, kM] and pm.tolist() == [1, 1]
    bc, bm, _, _, _ = oracle.eval_neighbourhood(inst, gm, gr, 1, 1)
    assert (bc, bm) == (kM + 2 * kM, 1)
    # N3 alone: the swaps 01 -> 10 at t = 0 and 10 -> 01 at t = 2 keep the
    # cost (2 kM); the null swap at t = 1 too, so N3's first move wins.  In
    # the combined layouts it comes after N1 and N2: local index 2T, global
    # index 2KT (product 0's).
    _, _, pc3, pm3, _ = oracle.eval_neighbourhood(inst, gm, gr, 4, 0)
    assert pc3.tolist() == [2 * kM, 2 * kM] and pm3.tolist() == [2 * T, 2 * T]
    bc3, bm3, _, _, _ = oracle.eval_neighbourhood(inst, gm, gr, 4, 1)
    assert (bc3, bm3) == (4 * kM, 2 * 2 * T)


def test_multistart_best_is_lowest_start_among_ties():
    """Repeated seeds give identical starts, so costs tie exactly; the
    best-of must be the lexicographic (cost, start) minimum: never above any
    start's cost, and the first of equal starts."""
    inst = oracle.Instance.from_arrays(gen.make_instance(0, 3, K=6, T=14))
    seeds = [7, 2, 7, 2, 9]
    best, res = oracle.multistart(inst, seeds, iters=20, kmax=3, mode=0)
    costs = [r.best_cost for r in res]
    assert costs[0] == costs[2] and costs[1] == costs[3]
    assert res[0].traj_hash == res[2].traj_hash
    assert costs[best] == min(costs)
    assert best == costs.index(min(costs))       # the first start of that cost
    assert best in (0, 1, 4)


def test_move_costs_recomposed_from_apply_and_decode():
    """Each entry of move_costs is the decode of the row after that move,
    through the separately pinned apply_move and decode_row, in the layout
    k * |row moves| + local."""
    rng = np.random.default_rng(21)
    inst = oracle.Instance.from_arrays(gen.make_instance(13, 2, K=3, T=9))
    K, T = inst.K, inst.T
    for _ in range(4):
        gm = (rng.random((K, T)) < 0.5).astype(np.uint8)
        gr = (rng.random((K, T)) < 0.5).astype(np.uint8)
        gm[:, 0] = 1
        for j in (1, 2, 3):
            c = oracle.move_costs(inst, gm, gr, j)
            per = oracle.row_moves(T, j)
            assert len(c) == oracle.nb_size(K, T, j) == K * per
            for m in range(len(c)):
                a, b = gm.copy(), gr.copy()
                oracle.apply_move(K, T, j, m, a, b)
                k = m // per
                changed = np.flatnonzero((a != gm).any(1) | (b != gr).any(1))
                assert set(changed.tolist()) <= {k}
                assert c[m] == oracle.decode_row(inst, k, a[k], b[k])[0]


def _sat(*xs):
    s = 0
    for x in xs:
        s = INF if (s == INF or x == INF) else s + x
    return s


@pytest.mark.parametrize("mask", [1, 2, 4, 5, 7])
def test_eval_neighbourhood_recomposed_from_move_costs(mask):
    """Algorithm 1's best-neighbour search, recomposed: per product the
    lexicographic (cost, combined local index) minimum; mode P's objective
    after every strictly improving product applies its move, and the count
    of such products; mode G's lexicographic (objective, combined global
    index) minimum over all moves, the objective being the saturating sum of
    the other rows plus the moved row."""
    rng = np.random.default_rng(mask)
    inst = oracle.Instance.from_arrays(gen.make_instance(14, mask, K=4, T=8))
    K, T = inst.K, inst.T
    for trial in range(5):
        gm = (rng.random((K, T)) < 0.5).astype(np.uint8)
        gr = (rng.random((K, T)) < 0.5).astype(np.uint8)
        if trial % 2 == 0:
            gm[:, 0] = 1
        total, rc = oracle.total_cost(inst, gm, gr)
        blocks, offs_local, offs_global, lo, go = [], [], [], 0, 0
        for j in (1, 2, 3):
            per = oracle.row_moves(T, j)
            if mask & (1 << (j - 1)):
                blocks.append((oracle.move_costs(inst, gm, gr, j).reshape(K, per), lo, go))
            lo += per
            go += K * per
        want_pc, want_pm = [], []
        for k in range(K):
            cands = [(int(c[k, l]), off + l) for c, off, _ in blocks for l in range(c.shape[1])]
            best = min(cands)
            want_pc.append(best[0])
            want_pm.append(best[1])
        imp = [k for k in range(K) if want_pc[k] < rc[k]]
        others = [[rc[q] for q in range(K) if q != k] for k in range(K)]
        want_p = _sat(*[want_pc[k] if k in imp else rc[k] for k in range(K)])
        gcands = [(_sat(int(c[k, l]), *others[k]), goff + k * c.shape[1] + l)
                  for c, _, goff in blocks for k in range(K) for l in range(c.shape[1])]
        bc_p, bm_p, pc, pm, n = oracle.eval_neighbourhood(inst, gm, gr, mask, 0)
        assert pc.tolist() == want_pc and pm.tolist() == want_pm
        assert (bc_p, bm_p) == (want_p, len(imp))
        assert n == sum(c.size for c, _, _ in blocks)
        bc_g, bm_g, _, _, _ = oracle.eval_neighbourhood(inst, gm, gr, mask, 1)
        assert (bc_g, bm_g) == min(gcands)


def _vnd_replay(inst, gm, gr, mode):
    """Algorithm 1's pipe VND step by step from the pinned evaluation and
    apply: for j = 1..3 evaluate N_j alone; mode P applies every product's
    best move that strictly improves its row, mode G the single best move
    when it lowers the objective; stop after a sweep without improvement."""
    K, T = inst.K, inst.T
    gm, gr = gm.copy(), gr.copy()
    loff = {1: 0, 2: T, 3: 2 * T}                  # combined local offsets
    goff = {1: 0, 2: K * T, 3: 2 * K * T}          # combined global offsets
    cnt = dict(vnd_cycles=0, evals=0, moves_evaluated=0, applied=0)
    while True:
        cnt["vnd_cycles"] += 1
        improved = False
        for j in (1, 2, 3):
            per = oracle.row_moves(T, j)
            total, rc = oracle.total_cost(inst, gm, gr)
            bc, bm, pc, pm, n = oracle.eval_neighbourhood(inst, gm, gr, 1 << (j - 1), mode)
            cnt["evals"] += 1
            cnt["moves_evaluated"] += n
            if mode == 0:
                for k in range(K):
                    if pc[k] < rc[k]:
                        oracle.apply_move(K, T, j, k * per + int(pm[k]) - loff[j], gm, gr)
                        cnt["applied"] += 1
                        improved = True
            elif bc < total:
                oracle.apply_move(K, T, j, bm - goff[j], gm, gr)
                cnt["applied"] += 1
                improved = True
        if not improved:
            return gm, gr, cnt


@pytest.mark.parametrize("mode", [0, 1])
def test_vnd_replayed_from_evaluation_and_apply(mode):
    rng = np.random.default_rng(40 + mode)
    inst = oracle.Instance.from_arrays(gen.make_instance(15, mode, K=4, T=11))
    starts = [oracle.initial_solution(inst.K, inst.T)]
    for _ in range(3):
        gm = (rng.random((inst.K, inst.T)) < 0.5).astype(np.uint8)
        gr = (rng.random((inst.K, inst.T)) < 0.5).astype(np.uint8)
        gm[:, 0] = 1
        starts.append((gm, gr))
    for gm, gr in starts:
        wm, wr, wc = _vnd_replay(inst, gm, gr, mode)
        om, orr, oc = oracle.vnd(inst, gm, gr, mode)
        np.testing.assert_array_equal(om, wm)
        np.testing.assert_array_equal(orr, wr)
        for key, v in wc.items():
            assert oc[key] == v, key


@pytest.mark.parametrize("mode", [0, 1])
def test_gvns_replayed_from_shake_vnd_and_objective(mode):
    """Algorithm 2 (reading 7) step by step from the pinned Shake, VND and
    objective: every trajectory entry (k, f(x''), accepted), the final x and
    f(x) equal the oracle's run."""
    inst = oracle.Instance.from_arrays(gen.make_instance(16, mode, K=4, T=10))
    K, T, seed, iters, kmax = inst.K, inst.T, 11, 60, 3
    gm, gr = oracle.initial_solution(K, T)
    gm, gr, _ = oracle.vnd(inst, gm, gr, mode)
    fx, k = oracle.total_cost(inst, gm, gr)[0], 1
    want = []
    for it in range(iters):
        a, b = gm.copy(), gr.copy()
        oracle.shake(K, T, a, b, seed, it, k)
        a, b, _ = oracle.vnd(inst, a, b, mode)
        f = oracle.total_cost(inst, a, b)[0]
        want.append((it, k, f, int(f < fx)))
        if f < fx:
            gm, gr, fx, k = a, b, f, 1
        else:
            k = k + 1 if k < kmax else 1
    o = oracle.vns(inst, seed=seed, iters=iters, kmax=kmax, mode=mode)
    got = [(int(e["it"]), int(e["k"]), int(e["cost"]), int(e["accepted"])) for e in o.traj]
    assert got == want
    assert o.best_cost == fx
    np.testing.assert_array_equal(o.gM, gm)
    np.testing.assert_array_equal(o.gR, gr)
    assert any(w[3] for w in want) and not all(w[3] for w in want)


def test_objective_is_the_saturating_sum_of_rows():
    """Section 2's objective: the sum of the independent row costs, with any
    infeasible row making the whole solution infeasible (INT64_MAX)."""
    inst = oracle.Instance.from_arrays(gen.make_instance(17, 0, K=5, T=9))
    K, T = inst.K, inst.T
    rng = np.random.default_rng(8)
    seen_inf = seen_fin = False
    for i in range(40):
        gm = (rng.random((K, T)) < 0.5).astype(np.uint8)
        gr = (rng.random((K, T)) < 0.5).astype(np.uint8)
        gm[:, 0] = rng.random(K) < 0.85
        if i % 2:   # every row opens with manufacturing, no remanufacture-only setup
            gm[:, 0] = 1
            gr &= gm
        total, rc = oracle.total_cost(inst, gm, gr)
        rows = [oracle.decode_row(inst, k, gm[k], gr[k])[0] for k in range(K)]
        assert rc.tolist() == rows
        if INF in rows:
            assert total == INF
            seen_inf = True
        else:
            assert total == sum(rows)
            seen_fin = True
    assert seen_inf and seen_fin


# ---------------------------------------------------------------------------
# Work measure: decode steps of a move (tests/golden/decode_steps.txt).
# ---------------------------------------------------------------------------

def _decode_steps_rows():
    rows = []
    with open(os.path.join(GOLDEN, "decode_steps.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            rows.append([c.strip() for c in line.split("|")])
    return rows


@pytest.mark.parametrize("row", _decode_steps_rows(), ids=lambda r: r[0])
def test_decode_steps_hand_derived(row):
    """Every N1, N2 and N3 move of the worked-example rows, step counts
    derived by hand from the Section 2 decode (derivations in the file)."""
    name, D, R, gM, gR, n1, n2, n3 = row
    D, R = _ints(D), _ints(R)
    T = len(D)
    inst = oracle.Instance(np.array([D]), np.array([R]), [100], [50], [2], [1])
    gm, gr = np.array(_ints(gM), np.uint8), np.array(_ints(gR), np.uint8)
    for j, want in ((1, n1), (2, n2), (3, n3)):
        got = [oracle.decode_steps(inst, 0, gm, gr, j, l) for l in range(oracle.row_moves(T, j))]
        assert got == _ints(want), (name, j)


def _setups(gm, gr, a0):
    return [t for t in range(max(a0, 0), len(gm)) if gm[t] or gr[t]]


@pytest.mark.parametrize("seed", range(4))
def test_decode_steps_stop_where_the_decodes_coincide(seed):
    """What the count means, checked on the pinned decode's plans: for a
    feasible row and a feasible move, the walk covers the setups of the moved
    row from a0 and stops at the first setup after the changed periods from
    which the moved row's plan (xM, xR, yM, yR) repeats the row's plan; at every
    counted setup after the changed periods the recoverable stock entering it
    still differs.  Any move takes at most one step per setup of the moved
    row from a0, and a move that changes nothing takes none."""
    rng = np.random.default_rng(500 + seed)
    checked = 0
    for trial in range(12):
        T = int(rng.integers(2, 24))
        g = gen.make_instance(600 + seed, trial, K=1, T=T)
        inst = oracle.Instance.from_arrays(g)
        for _ in range(50):  # a feasible row, so that its plan exists
            gm = (rng.random(T) < rng.uniform(0.2, 0.9)).astype(np.uint8)
            gr = (rng.random(T) < rng.uniform(0.2, 0.9)).astype(np.uint8)
            gm[0] = 1
            c0, p0 = oracle.decode_row(inst, 0, gm, gr)
            if c0 != INF:
                break
        for j in (1, 2, 3):
            for l in range(oracle.row_moves(T, j)):
                nm, nr = gm[None, :].copy(), gr[None, :].copy()
                oracle.apply_move(1, T, j, l, nm, nr)
                nm, nr = nm[0], nr[0]
                steps = oracle.decode_steps(inst, 0, gm, gr, j, l)
                changed = np.nonzero((nm != gm) | (nr != gr))[0]
                if len(changed) == 0:
                    assert steps == 0
                    continue
                t1, t2 = int(changed[0]), int(changed[-1])
                both = [t for t in range(t1 + 1) if (gm[t] or gr[t]) and (nm[t] or nr[t])]
                s0 = both[-1] if both else -1
                su = _setups(nm, nr, s0 if s0 >= 0 else 0)
                assert 0 <= steps <= len(su)
                c1, p1 = oracle.decode_row(inst, 0, nm, nr)
                if c0 == INF or c1 == INF or steps == 0:
                    continue
                stop = su[steps] if steps < len(su) else T
                # from the stop on, the moved row's plan is the row's plan
                assert stop == T or stop > t2
                np.testing.assert_array_equal(p1[:, stop:], p0[:, stop:])
                # before it, after the change, the entering stock differed
                for s in su[:steps]:
                    if s > t2:
                        assert s > 0 and p1[3, s - 1] != p0[3, s - 1]
                # and the stop is the first such setup: stock equal there
                if stop < T:
                    assert p1[3, stop - 1] == p0[3, stop - 1]
                checked += 1
    assert checked > 200


def test_gvns_from_the_initial_vnd_output_is_the_same_run():
    """Algorithm 2 applies VND to the start before its first shake, so a run
    from the all-open start and one from that VND's output follow the same
    trajectory; their counters differ by exactly the initial descent against
    one sweep that moves nothing.  (The workload-scale GPU tests start the
    oracle there.)  Shown on the multi-start instance, K=100, T=104."""
    inst = oracle.Instance.from_arrays(gen.multistart_large())
    r0 = oracle.vns(inst, seed=0, iters=0, kmax=3, mode=0)
    a = oracle.vns(inst, seed=7, iters=3, kmax=3, mode=0)
    b = oracle.vns(inst, seed=7, iters=3, kmax=3, mode=0, gM=r0.gM, gR=r0.gR)
    assert (a.best_cost, a.traj_hash) == (b.best_cost, b.traj_hash)
    np.testing.assert_array_equal(a.traj, b.traj)
    sweep = inst.K * (2 * inst.T + 2 * (inst.T - 1))
    assert a.counters["moves_evaluated"] == \
        b.counters["moves_evaluated"] - sweep + r0.counters["moves_evaluated"]
    assert a.counters["applied"] == b.counters["applied"] + r0.counters["applied"]
    assert a.counters["accepted"] == b.counters["accepted"]
