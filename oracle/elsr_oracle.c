/*
 * elsr_oracle.c -- plain, slow, single-threaded CPU oracle for the variable
 * neighbourhood search (VNS) of Antoniadis & Sifaleras (2017) on the
 * uncapacitated multi-item economic lot-sizing problem with remanufacturing
 * (ELSR).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * It follows the paper step by step, in the paper's order and notation:
 *   - Section 2 (problem statement): products k, periods t, setup costs
 *     kM(k), kR(k), holding costs hM(k), hR(k), demand D(k,t), returns
 *     R(k,t); decisions xM, xR (manufactured / remanufactured quantities) and
 *     yM, yR (serviceable / recoverable stock); objective = setup + holding,
 *     plus unit production costs pM(k) * xM + pR(k) * xR when an instance
 *     gives them (Algorithm 1's signature names p_M, p_R; 0 otherwise).
 *   - Section 3: products are uncoupled, so the objective is a sum of
 *     per-product row costs.
 *   - Algorithm 1 (parallel VND): for each neighbourhood N_k, find each
 *     product's best neighbour, sum the improvements (diff), repeat the whole
 *     k = 1..kmax sweep until no improvement.
 *   - Algorithm 2 (GVNS): shake, VND, keep the better solution.
 *
 * The paper defers the model's exact formulation, the initial solution, the
 * neighbourhoods and the shaking operator to its reference [SK2016].  The
 * readings adopted for them are stated at each function ("Reading:").
 *
 * Every decode is a full per-period pass over the row (O(T) per candidate);
 * there are no prefix sums, no caching and no incremental evaluation here.
 *
 * Parity status: the decode, objective and neighbourhood search are pinned by
 * hand-derived worked examples, closed forms, plan invariants, a
 * Wagner-Whitin reduction and brute force.  The readings themselves (decode
 * rule, neighbourhoods, shake, acceptance) cannot be pinned against the
 * paper's unpublished [SK2016] rules: parity unpinned for those readings,
 * and likewise for the fork-join workers' draw keys (the paper gives no
 * shaking rule).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF INT64_MAX

/* Problem data of Section 2.  D and R are row-major [K][T]; costs are [K].
 * pM, pR: unit manufacturing and remanufacturing costs [K] (Algorithm 1's
 * p_M, p_R); NULL means 0. */
typedef struct {
    int32_t K, T;
    const int32_t *D, *R;
    const int32_t *kM, *kR, *hM, *hR;
    const int32_t *pM, *pR;
} orc_instance;

/* Per-run counters (Algorithm 1 / Algorithm 2 bookkeeping). */
typedef struct {
    int64_t moves_evaluated; /* sum over neighbourhood evaluations of |N_j| */
    int64_t evals;           /* neighbourhood evaluations */
    int64_t vnd_cycles;      /* full j = 1..3 sweeps of the VND repeat loop */
    int64_t applied;         /* moves applied by VND */
    int64_t iterations;      /* GVNS shaking iterations */
    int64_t accepted;        /* iterations whose VND result was kept */
} orc_counters;

/* One trajectory entry per GVNS iteration: (it, k, f(x''), accepted). */
typedef struct {
    int32_t it;
    int32_t k;
    int64_t cost;
    int32_t accepted;
    int32_t pad;
} orc_traj;

static int64_t sat_add(int64_t a, int64_t b)
{
    if (a == ORC_INF || b == ORC_INF) return ORC_INF;
    return a + b;
}

/* ------------------------------------------------------------------------ */
/* Decode and row cost (Section 2 objective; decode reading).                */
/* ------------------------------------------------------------------------ */

/*
 * Decode one product row from its setup bits and return its cost.
 *
 * Section 2: the row cost is the manufacturing and remanufacturing setup
 * costs plus the holding costs of serviceable stock yM and recoverable stock
 * yR.  Reading (the formulation is in [SK2016], not in the paper):
 *   yM(t) = yM(t-1) + xM(t) + xR(t) - D(t),  yR(t) = yR(t-1) + R(t) - xR(t),
 *   yM(-1) = yR(-1) = 0, all quantities >= 0, holding charged on end-of-period
 *   stock, setup cost charged on the setup bit, and the unit production
 *   costs p_M, p_R of Algorithm 1's signature charged per unit of xM, xR
 *   (0 unless the instance gives them).
 * Decode reading: at each period with a setup, cover the demand up to the
 * next setup; remanufacture first from the available recoverable stock when
 * gR(t) = 1, manufacture the rest when gM(t) = 1; a shortfall is infeasible.
 *
 * gM, gR: the row's T setup bits (0/1).  plan (nullable): [4][T] receives
 * xM, xR, yM, yR.  Returns ORC_INF for an infeasible row.
 */
int64_t orc_decode_row(const orc_instance *in, int32_t k,
                       const uint8_t *gM, const uint8_t *gR, int64_t *plan)
{
    const int32_t T = in->T;
    const int32_t *D = in->D + (int64_t)k * T;
    const int32_t *R = in->R + (int64_t)k * T;
    const int64_t kM = in->kM[k], kR = in->kR[k];
    const int64_t hM = in->hM[k], hR = in->hR[k];
    const int64_t pM = in->pM ? in->pM[k] : 0, pR = in->pR ? in->pR[k] : 0;
    int64_t yM_prev = 0, yR_prev = 0, cost = 0;

    for (int32_t t = 0; t < T; ++t) {
        int64_t avail = yR_prev + R[t];
        int64_t xm = 0, xr = 0;
        if (gM[t] || gR[t]) {
            int32_t n = t + 1;
            while (n < T && !(gM[n] || gR[n])) ++n;
            int64_t need = -yM_prev;
            for (int32_t i = t; i < n; ++i) need += D[i];
            if (gR[t]) xr = avail < need ? avail : need;
            if (gM[t]) {
                xm = need - xr;
            } else if (xr < need) {
                return ORC_INF; /* remanufacturing alone cannot cover demand */
            }
        }
        int64_t yM = yM_prev + xm + xr - D[t];
        if (yM < 0) return ORC_INF; /* demand not covered (e.g. before the first setup) */
        int64_t yR = avail - xr;
        cost += kM * gM[t] + kR * gR[t] + hM * yM + hR * yR + pM * xm + pR * xr;
        if (plan) {
            plan[t] = xm;
            plan[T + t] = xr;
            plan[2 * T + t] = yM;
            plan[3 * T + t] = yR;
        }
        yM_prev = yM;
        yR_prev = yR;
    }
    return cost;
}

/* Objective of Section 2: sum of the independent row costs (saturating). */
int64_t orc_total_cost(const orc_instance *in, const uint8_t *gM,
                       const uint8_t *gR, int64_t *rowcost)
{
    int64_t total = 0;
    for (int32_t k = 0; k < in->K; ++k) {
        int64_t c = orc_decode_row(in, k, gM + (int64_t)k * in->T,
                                   gR + (int64_t)k * in->T, NULL);
        if (rowcost) rowcost[k] = c;
        total = sat_add(total, c);
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Neighbourhoods (Section 3: "same as [SK2016]", omitted there; reading).   */
/* ------------------------------------------------------------------------ */

/*
 * Reading of the neighbourhood structures N_1..N_3 (sizes 2*K*T + shift
 * moves):
 *   N_1: flip gM(k,t);                     global index k*T + t
 *   N_2: flip gR(k,t);                     global index k*T + t
 *   N_3: swap g_c(k,t) <-> g_c(k,t+1), c in {M=0, R=1}, t in [0, T-2];
 *        local index c*(T-1) + t, global index k*2(T-1) + local.
 */
int64_t orc_nb_size(int32_t K, int32_t T, int32_t j)
{
    if (j == 1 || j == 2) return (int64_t)K * T;
    if (j == 3) return (int64_t)K * 2 * (T - 1);
    return 0;
}

int64_t orc_row_moves(int32_t T, int32_t j)
{
    if (j == 1 || j == 2) return T;
    if (j == 3) return 2 * (int64_t)(T - 1);
    return 0;
}

/* Apply move `local` of N_j to the bits of one row (in place). */
void orc_apply_row_move(int32_t T, int32_t j, int64_t local, uint8_t *gM,
                        uint8_t *gR)
{
    if (j == 1) {
        gM[local] ^= 1;
    } else if (j == 2) {
        gR[local] ^= 1;
    } else if (j == 3) {
        int64_t c = local / (T - 1);
        int64_t t = local % (T - 1);
        uint8_t *g = c == 0 ? gM : gR;
        uint8_t tmp = g[t];
        g[t] = g[t + 1];
        g[t + 1] = tmp;
    }
}

/* Apply global move m of N_j to the full K x T solution (in place). */
void orc_apply_move(int32_t K, int32_t T, int32_t j, int64_t m, uint8_t *gM,
                    uint8_t *gR)
{
    int64_t per_row = orc_row_moves(T, j);
    (void)K;
    if (per_row <= 0) return;
    int64_t k = m / per_row, local = m % per_row;
    orc_apply_row_move(T, j, local, gM + k * T, gR + k * T);
}

/*
 * New cost of the moved row for every move of N_j (global layout).  Each
 * candidate is a copy of the row with the move applied, decoded in full.
 */
void orc_move_costs(const orc_instance *in, const uint8_t *gM,
                    const uint8_t *gR, int32_t j, int64_t *out)
{
    const int32_t K = in->K, T = in->T;
    int64_t per_row = orc_row_moves(T, j);
    uint8_t *cm = malloc(T > 0 ? T : 1), *cr = malloc(T > 0 ? T : 1);
    for (int32_t k = 0; k < K; ++k) {
        for (int64_t l = 0; l < per_row; ++l) {
            memcpy(cm, gM + (int64_t)k * T, T);
            memcpy(cr, gR + (int64_t)k * T, T);
            orc_apply_row_move(T, j, l, cm, cr);
            out[k * per_row + l] = orc_decode_row(in, k, cm, cr, NULL);
        }
    }
    free(cm);
    free(cr);
}

/* ------------------------------------------------------------------------ */
/* Best neighbour (Algorithm 1: best-neighbour search and summed gains).    */
/* ------------------------------------------------------------------------ */

/* Offsets of N_1, N_2, N_3 in the combined (all three neighbourhoods) move
 * layout: per product [N_1 | N_2 | N_3], globally [N_1 | N_2 | N_3]. */
static int64_t comb_local_off(int32_t T, int32_t j)
{
    return j == 1 ? 0 : (j == 2 ? T : 2 * (int64_t)T);
}
static int64_t comb_global_off(int32_t K, int32_t T, int32_t j)
{
    return j == 1 ? 0 : (j == 2 ? (int64_t)K * T : 2 * (int64_t)K * T);
}

/* Total after replacing row k's cost by c (mode G): the saturating sum of
 * the other rows plus c. */
static int64_t total_with_row(const int64_t *rowcost, int32_t K, int32_t k,
                              int64_t c)
{
    int64_t s = c;
    for (int32_t i = 0; i < K; ++i)
        if (i != k) s = sat_add(s, rowcost[i]);
    return s;
}

/*
 * Evaluate the neighbourhoods in `mask` (bit j-1 selects N_j) at the current
 * solution without applying anything.
 *
 * Mode P (mode = 0, Algorithm 1): for every product k, the best move of row
 * k is the lexicographic minimum of (new row cost, combined local index);
 * pp_cost[k], pp_move[k] receive it (cost ORC_INF, move -1 when the row has
 * no moves).  *best_cost = the current objective minus the summed
 * improvements, i.e. the objective after every product applies its best
 * move when that move strictly improves its row;
 * *best_move = the number of improving products.
 *
 * Mode G (mode = 1, single argmin): the best move over the whole
 * neighbourhood is the lexicographic minimum of (new total, combined global
 * index); *best_cost, *best_move receive it.  The per-product arrays are
 * filled as in mode P.
 *
 * Output pointers may be NULL.  Returns the number of moves evaluated.
 */
int64_t orc_eval_neighbourhood(const orc_instance *in, const uint8_t *gM,
                               const uint8_t *gR, uint32_t mask, int32_t mode,
                               int64_t *best_cost, int64_t *best_move,
                               int64_t *pp_cost, int64_t *pp_move)
{
    const int32_t K = in->K, T = in->T;
    int64_t *rowcost = malloc(sizeof(int64_t) * (K > 0 ? K : 1));
    int64_t total = orc_total_cost(in, gM, gR, rowcost);
    int64_t g_cost = ORC_INF, g_move = -1, evaluated = 0;
    int64_t s_after = 0, n_improving = 0;

    for (int32_t k = 0; k < K; ++k) {
        int64_t r_cost = ORC_INF, r_move = -1;
        for (int32_t j = 1; j <= 3; ++j) {
            if (!(mask & (1u << (j - 1)))) continue;
            int64_t per_row = orc_row_moves(T, j);
            if (per_row <= 0) continue;
            int64_t *c = malloc(sizeof(int64_t) * per_row);
            uint8_t *cm = malloc(T), *cr = malloc(T);
            for (int64_t l = 0; l < per_row; ++l) {
                memcpy(cm, gM + (int64_t)k * T, T);
                memcpy(cr, gR + (int64_t)k * T, T);
                orc_apply_row_move(T, j, l, cm, cr);
                c[l] = orc_decode_row(in, k, cm, cr, NULL);
            }
            for (int64_t l = 0; l < per_row; ++l) {
                int64_t li = comb_local_off(T, j) + l;
                if (r_move < 0 || c[l] < r_cost || (c[l] == r_cost && li < r_move)) {
                    r_cost = c[l];
                    r_move = li;
                }
                int64_t nt = total_with_row(rowcost, K, k, c[l]);
                int64_t gi = comb_global_off(K, T, j) + (int64_t)k * per_row + l;
                if (g_move < 0 || nt < g_cost || (nt == g_cost && gi < g_move)) {
                    g_cost = nt;
                    g_move = gi;
                }
            }
            evaluated += per_row;
            free(c);
            free(cm);
            free(cr);
        }
        if (pp_cost) pp_cost[k] = r_cost;
        if (pp_move) pp_move[k] = r_move;
        if (r_move >= 0 && r_cost < rowcost[k]) {
            s_after = sat_add(s_after, r_cost);
            ++n_improving;
        } else {
            s_after = sat_add(s_after, rowcost[k]);
        }
    }
    if (mode == 0) {
        if (best_cost) *best_cost = s_after;
        if (best_move) *best_move = n_improving;
    } else {
        if (best_cost) *best_cost = g_move < 0 ? total : g_cost;
        if (best_move) *best_move = g_move;
    }
    free(rowcost);
    return evaluated;
}

/* ------------------------------------------------------------------------ */
/* VND (Algorithm 1, pipe form).                                             */
/* ------------------------------------------------------------------------ */

/*
 * One evaluation of N_j at the current solution followed by the update of
 * Algorithm 1.  Mode P: every product whose best row move strictly improves
 * its row takes it (all products see the same current solution; they are
 * independent).  Mode G (reading): the single best move of the whole
 * neighbourhood, by (new total, global index), is applied when its total is
 * strictly below the current total.  Returns the number of applied moves.
 */
static int64_t vnd_step(const orc_instance *in, uint8_t *gM, uint8_t *gR,
                        int32_t j, int32_t mode, orc_counters *cnt)
{
    const int32_t K = in->K, T = in->T;
    int64_t per_row = orc_row_moves(T, j);
    int64_t applied = 0;
    cnt->evals += 1;
    cnt->moves_evaluated += orc_nb_size(K, T, j);
    if (per_row <= 0) return 0;

    int64_t *rowcost = malloc(sizeof(int64_t) * K);
    int64_t total = orc_total_cost(in, gM, gR, rowcost);
    int64_t *c = malloc(sizeof(int64_t) * per_row * K);
    orc_move_costs(in, gM, gR, j, c);

    if (mode == 0) {
        for (int32_t k = 0; k < K; ++k) {
            int64_t bc = ORC_INF, bl = -1;
            for (int64_t l = 0; l < per_row; ++l) {
                int64_t v = c[k * per_row + l];
                if (bl < 0 || v < bc) { /* strict: the lowest index wins ties */
                    bc = v;
                    bl = l;
                }
            }
            if (bc < rowcost[k]) {
                orc_apply_row_move(T, j, bl, gM + (int64_t)k * T, gR + (int64_t)k * T);
                ++applied;
            }
        }
    } else {
        int64_t bt = ORC_INF, bm = -1;
        for (int32_t k = 0; k < K; ++k) {
            for (int64_t l = 0; l < per_row; ++l) {
                int64_t nt = total_with_row(rowcost, K, k, c[k * per_row + l]);
                if (bm < 0 || nt < bt) {
                    bt = nt;
                    bm = k * per_row + l;
                }
            }
        }
        if (bm >= 0 && bt < total) {
            orc_apply_move(K, T, j, bm, gM, gR);
            ++applied;
        }
    }
    free(c);
    free(rowcost);
    cnt->applied += applied;
    return applied;
}

/* VND of Algorithm 1: repeat the sweep j = 1..3 (no restart at j = 1 after
 * an improvement) until a full sweep improves nothing.  A safety cap of
 * 2^20 sweeps returns -1. */
int32_t orc_vnd(const orc_instance *in, uint8_t *gM, uint8_t *gR, int32_t mode,
                orc_counters *cnt)
{
    for (int64_t cycle = 0; cycle < (1 << 20); ++cycle) {
        int improvement = 0;
        cnt->vnd_cycles += 1;
        for (int32_t j = 1; j <= 3; ++j)
            if (vnd_step(in, gM, gR, j, mode, cnt) > 0) improvement = 1;
        if (!improvement) return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Shaking draws: splitmix64 (Steele, Lea & Flood 2014).                     */
/* ------------------------------------------------------------------------ */

/* One splitmix64 step from state z: advance by the golden-ratio increment,
 * then the published output mix. */
uint64_t orc_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Draw for move j of a shake of strength k at iteration it (reading: keyed
 * by seed, iteration and neighbourhood). */
uint64_t orc_draw(uint64_t seed, uint64_t it, uint64_t k, uint64_t j)
{
    uint64_t a = orc_splitmix64(seed);
    uint64_t b = orc_splitmix64(a ^ it);
    return orc_splitmix64(b ^ ((k << 32) | j));
}

/* Shake(x, k) of Algorithm 2 (reading): apply k successive random moves of
 * N_k, move j being draw(seed, it, k, j) mod |N_k| in N_k's global layout.
 * Moves are applied even when they make a row infeasible. */
void orc_shake(int32_t K, int32_t T, uint8_t *gM, uint8_t *gR, uint64_t seed,
               int64_t it, int32_t k)
{
    int64_t size = orc_nb_size(K, T, k);
    if (size <= 0) return;
    for (int32_t j = 0; j < k; ++j) {
        uint64_t m = orc_draw(seed, (uint64_t)it, (uint64_t)k, (uint64_t)j) % (uint64_t)size;
        orc_apply_move(K, T, k, (int64_t)m, gM, gR);
    }
}

/* Rolling trajectory hash: h <- mix(h ^ f), h <- mix(h ^ (it<<32 | k<<1 | acc)). */
static uint64_t traj_hash_step(uint64_t h, int64_t it, int32_t k, int64_t f,
                               int32_t acc)
{
    h = orc_splitmix64(h ^ (uint64_t)f);
    h = orc_splitmix64(h ^ (((uint64_t)it << 32) | ((uint64_t)k << 1) | (uint64_t)acc));
    return h;
}

/* ------------------------------------------------------------------------ */
/* GVNS (Algorithm 2, reading).                                              */
/* ------------------------------------------------------------------------ */

/*
 * Reading of Algorithm 2 (its k loop has no increment and its neighbourhood
 * change is commented out; the time limit is replaced by an iteration
 * budget):
 *   x = VND(start); k = 1
 *   for it = 0 .. iters-1:
 *       x' = Shake(x, k, it); x'' = VND(x')
 *       if f(x'') < f(x): x = x'', k = 1  else: k = k+1, back to 1 after kmax
 * gM, gR: in = start solution, out = best solution x.  log (nullable):
 * [iters] entries.  Returns 0, or -1 when a VND hit its cycle cap.
 */
int32_t orc_vns(const orc_instance *in, uint8_t *gM, uint8_t *gR, uint64_t seed,
                int32_t iters, int32_t kmax, int32_t mode, orc_counters *cnt,
                orc_traj *log, int64_t *best_cost, uint64_t *traj_hash)
{
    const int32_t K = in->K, T = in->T;
    const size_t n = (size_t)K * T;
    uint8_t *pM = malloc(n ? n : 1), *pR = malloc(n ? n : 1);
    uint64_t h = 0;
    int32_t rc = 0;

    memset(cnt, 0, sizeof(*cnt));
    if (orc_vnd(in, gM, gR, mode, cnt) != 0) rc = -1;
    int64_t fx = orc_total_cost(in, gM, gR, NULL);
    int32_t k = 1;
    for (int32_t it = 0; it < iters && rc == 0; ++it) {
        memcpy(pM, gM, n);
        memcpy(pR, gR, n);
        orc_shake(K, T, pM, pR, seed, it, k);
        if (orc_vnd(in, pM, pR, mode, cnt) != 0) rc = -1;
        int64_t f2 = orc_total_cost(in, pM, pR, NULL);
        int32_t acc = f2 < fx;
        if (log) {
            log[it].it = it;
            log[it].k = k;
            log[it].cost = f2;
            log[it].accepted = acc;
            log[it].pad = 0;
        }
        h = traj_hash_step(h, it, k, f2, acc);
        cnt->iterations += 1;
        if (acc) {
            memcpy(gM, pM, n);
            memcpy(gR, pR, n);
            fx = f2;
            k = 1;
            cnt->accepted += 1;
        } else {
            k = k + 1;
            if (k > kmax) k = 1;
        }
    }
    if (best_cost) *best_cost = fx;
    if (traj_hash) *traj_hash = h;
    free(pM);
    free(pR);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Hybrid GVNS of Algorithm 2 (fork-join over workers, reading).             */
/* ------------------------------------------------------------------------ */

/* Shake(x, k) of worker p: as orc_shake, with move j drawn as
 * draw(seed, it, k, p << 8 | j).  Worker 0 draws exactly as the sequential
 * GVNS does. */
void orc_shake_worker(int32_t K, int32_t T, uint8_t *gM, uint8_t *gR, uint64_t seed,
                      int64_t it, int32_t k, int32_t worker)
{
    int64_t size = orc_nb_size(K, T, k);
    if (size <= 0) return;
    for (int32_t j = 0; j < k; ++j) {
        uint64_t key = ((uint64_t)worker << 8) | (uint64_t)j;
        uint64_t m = orc_draw(seed, (uint64_t)it, (uint64_t)k, key) % (uint64_t)size;
        orc_apply_move(K, T, k, (int64_t)m, gM, gR);
    }
}

/*
 * Algorithm 2 as the paper runs it on two GPUs: every OpenMP thread (one per
 * GPU) shakes the same incumbent x with the same k and runs VND on its own
 * copy; the threads' objective values are compared and the minimum is kept
 * (Section 3, fork-join model).  Reading, for P workers:
 *   x = VND(start); k = 1
 *   for it = 0 .. iters-1:
 *       for p = 0 .. P-1:  x''_p = VND(Shake_p(x, k, it))
 *       p* = the p with the least (f(x''_p), p)
 *       if f(x''_p*) < f(x): x = x''_p*, k = 1
 *       else:                k = k+1, back to 1 after kmax
 * The log holds (it, k, f(x''_p*), accepted) with p* in its spare field; the
 * trajectory hash folds the same values as the sequential GVNS.  Counters
 * add up every worker's VND.  With one worker this is orc_vns.
 */
int32_t orc_vns_forkjoin(const orc_instance *in, uint8_t *gM, uint8_t *gR, uint64_t seed,
                         int32_t iters, int32_t kmax, int32_t mode, int32_t workers,
                         orc_counters *cnt, orc_traj *log, int64_t *best_cost,
                         uint64_t *traj_hash)
{
    const int32_t K = in->K, T = in->T;
    const size_t n = (size_t)K * T;
    uint8_t *pM = malloc(n ? n : 1), *pR = malloc(n ? n : 1);
    uint8_t *bM = malloc(n ? n : 1), *bR = malloc(n ? n : 1);
    uint64_t h = 0;
    int32_t rc = 0;

    memset(cnt, 0, sizeof(*cnt));
    if (orc_vnd(in, gM, gR, mode, cnt) != 0) rc = -1;
    int64_t fx = orc_total_cost(in, gM, gR, NULL);
    int32_t k = 1;
    for (int32_t it = 0; it < iters && rc == 0; ++it) {
        int64_t fbest = ORC_INF;
        int32_t pbest = -1;
        for (int32_t p = 0; p < workers; ++p) {
            memcpy(pM, gM, n);
            memcpy(pR, gR, n);
            orc_shake_worker(K, T, pM, pR, seed, it, k, p);
            if (orc_vnd(in, pM, pR, mode, cnt) != 0) rc = -1;
            int64_t f2 = orc_total_cost(in, pM, pR, NULL);
            if (pbest < 0 || f2 < fbest) { /* strict: the lowest worker wins ties */
                fbest = f2;
                pbest = p;
                memcpy(bM, pM, n);
                memcpy(bR, pR, n);
            }
        }
        int32_t acc = fbest < fx;
        if (log) {
            log[it].it = it;
            log[it].k = k;
            log[it].cost = fbest;
            log[it].accepted = acc;
            log[it].pad = pbest;
        }
        h = traj_hash_step(h, it, k, fbest, acc);
        cnt->iterations += 1;
        if (acc) {
            memcpy(gM, bM, n);
            memcpy(gR, bR, n);
            fx = fbest;
            k = 1;
            cnt->accepted += 1;
        } else {
            k = k + 1;
            if (k > kmax) k = 1;
        }
    }
    if (best_cost) *best_cost = fx;
    if (traj_hash) *traj_hash = h;
    free(pM);
    free(pR);
    free(bM);
    free(bR);
    return rc;
}

/* Initial solution (reading; the paper omits it): every setup open. */
void orc_initial_solution(int32_t K, int32_t T, uint8_t *gM, uint8_t *gR)
{
    memset(gM, 1, (size_t)K * T);
    memset(gR, 1, (size_t)K * T);
}

/* ------------------------------------------------------------------------ */
/* Work measure (not part of the method): decode steps of one move.          */
/* ------------------------------------------------------------------------ */

/*
 * Per-period decode of one row under the decode rule of orc_decode_row,
 * recording avail[t] = yR(t-1) + R(t), the recoverable stock on hand at every
 * period it reaches.  Returns the first period at which the row falls short
 * (T when none).
 *
 * With `relaxed` set, a remanufacture-only setup whose stock cannot cover its
 * need remanufactures all of it and the rest counts as manufactured, and the
 * decode goes on; demand before the first setup still ends it (there is no
 * setup to produce it).  For a feasible row both forms are the same decode.
 */
static int32_t decode_avail(const orc_instance *in, int32_t k, const uint8_t *gM,
                            const uint8_t *gR, int relaxed, int64_t *avail_at)
{
    const int32_t T = in->T;
    const int32_t *D = in->D + (int64_t)k * T, *R = in->R + (int64_t)k * T;
    int64_t yM_prev = 0, yR_prev = 0;
    for (int32_t t = 0; t < T; ++t) {
        int64_t avail = yR_prev + R[t], xm = 0, xr = 0;
        avail_at[t] = avail;
        if (gM[t] || gR[t]) {
            int32_t n = t + 1;
            while (n < T && !(gM[n] || gR[n])) ++n;
            int64_t need = -yM_prev;
            for (int32_t i = t; i < n; ++i) need += D[i];
            if (gR[t]) xr = avail < need ? avail : need;
            if (gM[t]) {
                xm = need - xr;
            } else if (xr < need) {
                if (!relaxed) return t;
                xm = need - xr;
            }
        }
        int64_t yM = yM_prev + xm + xr - D[t];
        if (yM < 0) return t;
        yM_prev = yM;
        yR_prev = avail - xr;
    }
    return T;
}

/* Next period after s holding a setup of the row (T when none). */
static int32_t next_setup(const uint8_t *gM, const uint8_t *gR, int32_t s, int32_t T)
{
    int32_t n = s + 1;
    while (n < T && !(gM[n] || gR[n])) ++n;
    return n;
}

/*
 * Decode steps of one move: the setup segments of the moved row x' that a
 * re-decode must visit before the rest of x' is known from the row x before
 * the move.  It measures work, to express throughput as integer operations
 * per second; the decode, the objective and the search do not use it.
 *
 * Let t1..t2 be the periods the move changes.  Periods before t1 carry the
 * same bits in x and x', so both decodes agree up to s0, the last period
 * <= t1 that holds a setup in both rows (the segment starting there ends
 * differently).  The re-decode starts at a0 = s0, or at the first setup of x'
 * when there is no such period, and walks x' one setup segment per step:
 *   - 0 steps when the move changes nothing, when x already falls short
 *     before s0 (that prefix is common), or when x' has demand before a0;
 *   - at a setup s > t2 (x and x' have the same setups from t2 on) the walk
 *     stops without counting s when x' enters s with the recoverable stock
 *     that x's decode has there: both rows then decode alike to the horizon;
 *   - otherwise s counts one step, and the walk stops after it when x' falls
 *     short in the segment starting at s, or at the end of the row.
 * "x's decode" in the stopping test is its relaxed decode (decode_avail):
 * it is the decode itself for a feasible x, and it also exists past the
 * first shortfall of an infeasible x, where the plain decode has stopped.
 * Once x' enters a setup with that decode's stock, x' repeats it from there
 * (x' is feasible iff the relaxed decode has no shortfall after that setup),
 * so no more decoding is needed; without the relaxed form every move of an
 * infeasible row would be charged a re-decode to the end of the row.  This
 * only lowers the count.  When x has demand before its first setup neither
 * form exists, and x' is walked to its end or its first shortfall.
 */
int64_t orc_decode_steps(const orc_instance *in, int32_t k, const uint8_t *gM,
                         const uint8_t *gR, int32_t j, int64_t local)
{
    const int32_t T = in->T;
    uint8_t *nm = malloc(T > 0 ? T : 1), *nr = malloc(T > 0 ? T : 1);
    int64_t *ax = malloc(sizeof(int64_t) * (T > 0 ? T : 1));
    int64_t *ay = malloc(sizeof(int64_t) * (T > 0 ? T : 1));
    int64_t count = 0;
    memcpy(nm, gM, T);
    memcpy(nr, gR, T);
    orc_apply_row_move(T, j, local, nm, nr);

    int32_t t1 = -1, t2 = -1;
    for (int32_t t = 0; t < T; ++t)
        if (nm[t] != gM[t] || nr[t] != gR[t]) {
            if (t1 < 0) t1 = t;
            t2 = t;
        }
    if (t1 < 0) goto done; /* nothing changes */

    int32_t f = decode_avail(in, k, gM, gR, 0, ax);           /* x, plain */
    int32_t x_alive = decode_avail(in, k, gM, gR, 1, ax) == T; /* x, relaxed */
    int32_t f2 = decode_avail(in, k, nm, nr, 0, ay);          /* x' */

    int32_t s0 = -1;
    for (int32_t t = t1; t >= 0; --t)
        if ((gM[t] || gR[t]) && (nm[t] || nr[t])) {
            s0 = t;
            break;
        }
    if (s0 >= 0 && f < s0) goto done; /* the common prefix falls short */
    int32_t a0 = s0 >= 0 ? s0 : next_setup(nm, nr, -1, T);
    if (f2 < a0) goto done; /* demand before the first setup of x' */

    for (int32_t s = a0; s < T;) {
        if (s > t2 && x_alive && ay[s] == ax[s]) break; /* x' repeats x from s */
        ++count;
        int32_t n = next_setup(nm, nr, s, T);
        if (f2 >= s && f2 < n) break; /* x' falls short in this segment */
        s = n;
    }
done:
    free(nm);
    free(nr);
    free(ax);
    free(ay);
    return count;
}
