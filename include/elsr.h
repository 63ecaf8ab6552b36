/*
 * elsr.h -- C ABI of the GB300 engine for the variable neighbourhood search
 * (VNS) of Antoniadis & Sifaleras (2017) on the uncapacitated multi-item
 * economic lot-sizing problem with remanufacturing (ELSR).
 *
 * Model (Section 2): K products, T periods; per product k setup costs
 * kM(k), kR(k), holding costs hM(k), hR(k); per (k,t) demand D(k,t) and
 * returns R(k,t).  A solution is the pair of binary setup matrices
 * gM(k,t), gR(k,t); decoding them gives manufactured / remanufactured
 * quantities xM, xR and serviceable / recoverable stocks yM, yR, and the
 * objective is setup plus holding cost.  Products are uncoupled (Section 3),
 * so the objective is a sum of row costs.
 *
 * Conventions used by every call:
 *   - integers only: quantities int32, costs int64; an infeasible row or
 *     solution costs ELSR_INF (INT64_MAX);
 *   - [K][T] arrays are row-major (product-major) and contiguous;
 *   - setup matrices cross the ABI as uint8 0/1 arrays [K][T];
 *   - every call returns ELSR_OK (0) or a negative ELSR_E_* code, and no
 *     C++ exception crosses the ABI; elsr_last_error() gives a message;
 *   - host pointers are read or written before the call returns, except
 *     where a call is documented as asynchronous; the library copies its
 *     inputs, so the caller keeps ownership of every buffer it passes;
 *   - device work is issued on the handle's CUDA stream (elsr_set_stream;
 *     default: the legacy default stream) on the device current at create;
 *   - a handle or batch is used by one host thread at a time; different
 *     handles may be used from different threads at once.
 *
 * Decode rule (the paper defers the formulation to [SK2016]; this is the
 * reading the library implements): at each period with a setup, cover the
 * demand up to the next setup; remanufacture first from the recoverable
 * stock when gR = 1, manufacture the rest when gM = 1; a shortfall, or
 * demand before the first setup, is infeasible.  Initial stocks are zero,
 * holding is charged on end-of-period stock and setup cost on the setup bit.
 *
 * Neighbourhoods (Section 3 omits them; reading): N1 flips gM(k,t), N2
 * flips gR(k,t), N3 swaps g_c(k,t) with g_c(k,t+1) for c in {M, R}.
 * Per-product (local) move index: N1 t, N2 t, N3 c*(T-1)+t.  Global index
 * within N_j: k*|row moves of N_j| + local.  When several neighbourhoods are
 * evaluated together the combined layouts are, per product,
 * [N1 | N2 | N3] (offsets 0, T, 2T) and, globally, [N1 | N2 | N3]
 * (offsets 0, K*T, 2*K*T).  Ties go to the lowest index.
 */
#ifndef ELSR_H
#define ELSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ELSR_OK 0
#define ELSR_E_ARG (-1)   /* invalid argument (null pointer, size, value) */
#define ELSR_E_RANGE (-2) /* instance exceeds the integer ranges below */
#define ELSR_E_NOMEM (-3) /* device or host allocation failed */
#define ELSR_E_CUDA (-4)  /* a CUDA runtime call or kernel failed */
#define ELSR_E_CAP (-5)   /* a VND exceeded its sweep cap (2^20 sweeps) */
#define ELSR_E_STATE (-6) /* call out of order (e.g. no result yet), or a
                             resumed state that does not match its checkpoint */
#define ELSR_E_TIMEOUT (-7) /* a device-side wait exceeded its limit */
#define ELSR_E_BUSY (-8)  /* serving: no room for a request now (retry later) */

#define ELSR_T_MAX 128 /* periods per product */
#define ELSR_MODE_P 0  /* Algorithm 1: each product takes its best move */
#define ELSR_MODE_G 1  /* one best move over the whole neighbourhood */
#define ELSR_INF INT64_MAX

typedef struct elsr_ctx elsr_t;
typedef struct elsr_batch elsr_batch_t;

/* Per-run statistics (Algorithms 1 and 2 bookkeeping). */
typedef struct {
    int64_t best_cost;       /* f(x) of the returned solution x */
    uint64_t traj_hash;      /* rolling hash of the trajectory (see below) */
    int64_t moves_evaluated; /* sum over neighbourhood evaluations of |N_j| */
    int64_t evals;           /* neighbourhood evaluations */
    int64_t vnd_cycles;      /* full j = 1..3 sweeps of VND's repeat loop */
    int64_t applied;         /* moves applied by VND (all products) */
    int64_t iterations;      /* GVNS shaking iterations run */
    int64_t accepted;        /* iterations whose VND result replaced x */
    int64_t segments;        /* decode steps of every evaluated move (work measure) */
    int32_t status;          /* ELSR_OK, ELSR_E_CAP or ELSR_E_TIMEOUT */
    int32_t reserved;
} elsr_stats_t;

/* One trajectory entry per GVNS iteration: (it, k, f(x''), accepted).
 * traj_hash folds the entries in order: h = mix(h ^ cost);
 * h = mix(h ^ (it << 32 | k << 1 | accepted)), from h = 0, mix being one
 * splitmix64 step. */
typedef struct {
    int32_t it;
    int32_t k;
    int64_t cost;
    int32_t accepted;
    int32_t reserved;
} elsr_traj_t;

/* State of a GVNS run between two iterations: Algorithm 2's loop variables
 * plus the running totals, enough to continue the run exactly where it
 * stopped (elsr_checkpoint, elsr_vns_resume).  The incumbent x itself is
 * passed beside it as two K x T 0/1 arrays.  Plain data: it may be stored
 * and loaded byte for byte. */
typedef struct {
    uint64_t seed;       /* the run's seed */
    int32_t kmax;        /* the run's kmax (1..3) */
    int32_t mode;        /* ELSR_MODE_P or ELSR_MODE_G */
    int32_t workers;     /* fork-join workers (0: the sequential GVNS) */
    int32_t next_it;     /* iterations run so far = index of the next one */
    int32_t k;           /* neighbourhood index k of the next iteration */
    int32_t status;      /* status of the run that produced it (ELSR_OK to resume) */
    int64_t cost;        /* f(x) of the incumbent */
    uint64_t traj_hash;  /* trajectory hash over iterations 0 .. next_it-1 */
    int64_t moves_evaluated, evals, vnd_cycles, applied, accepted, segments;
                         /* totals over iterations 0 .. next_it-1 and the initial VND */
} elsr_checkpoint_t;

/* Version of this ABI (major * 10000 + minor * 100 + patch). */
int elsr_version(void);

/* Resources one GVNS run of a K x T instance needs: shared memory per CTA
 * when the run uses one CTA (int32, nullable) and device memory held while
 * it is resident in a batch (int64 bytes, nullable).  For admission control
 * by callers that pack runs into batches. */
int elsr_run_footprint(int32_t K, int32_t T, int32_t *smem_one_cta,
                       int64_t *device_bytes);

/* Static text for an ELSR_* code. */
const char *elsr_strerror(int code);

/* Message of the last failed call on h (h may be NULL for create errors;
 * the text then describes the last failed create on this thread). */
const char *elsr_last_error(const elsr_t *h);

/*
 * Create a handle for one instance (Section 2 parameters).  D, R: host
 * [K][T]; kM, kR, hM, hR: host [K]; all int32, copied.  Requires 1 <= K,
 * 1 <= T <= ELSR_T_MAX, every value >= 0, sum_t D(k,t) and sum_t R(k,t)
 * below 2^31, and an objective bound
 *   sum_k T*(kM+kR) + T*(hM*sum_t D + hR*sum_t R) + hM*sum_t D*(T-t)
 *         + hR*sum_t R*(T-t)
 * below 2^40 (ELSR_E_RANGE otherwise).  The current solution starts as the
 * initial solution (every setup open).  Allocates device memory on the
 * current device.  On failure *out is NULL.
 */
int elsr_create(elsr_t **out, int32_t K, int32_t T, const int32_t *D,
                const int32_t *R, const int32_t *kM, const int32_t *kR,
                const int32_t *hM, const int32_t *hR);

/*
 * As elsr_create, with unit production costs: pM, pR host int32 [K]
 * (copied; both NULL = 0, as elsr_create).  Algorithm 1's signature carries
 * p_M and p_R beside the setup and holding costs; the row cost then adds
 * pM * xM(t) + pR * xR(t) in every period.  Each must be below 2^24, and
 * the objective bound above grows by sum_k (pM + pR) * sum_t D.  Every
 * other call works unchanged on such a handle.
 */
int elsr_create_ex(elsr_t **out, int32_t K, int32_t T, const int32_t *D,
                   const int32_t *R, const int32_t *kM, const int32_t *kR,
                   const int32_t *hM, const int32_t *hR, const int32_t *pM,
                   const int32_t *pR);

/* Free the handle and its device memory (synchronises its stream). */
void elsr_destroy(elsr_t *h);

/* Issue the handle's device work on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  Work issued afterwards on the new stream is
 * ordered after everything already issued on the previous one, which must
 * therefore still exist when the call is made.  Asynchronous. */
int elsr_set_stream(elsr_t *h, void *stream);

/* Kernel launch shape: lanes per product row (4, 8, 16 or 32 lanes of one
 * warp; 64 or 128 = a row spread over 2 or 4 warps) and threads
 * per block (multiple of 32 and of the lanes, <= 1024); 0 keeps the default. */
int elsr_set_launch(elsr_t *h, int32_t lanes_per_row, int32_t threads);

/* CTAs of one thread-block cluster that share a GVNS run of this handle
 * (1..16; 0 = automatic).  In mode G the CTAs' best keys meet through
 * distributed shared memory once per neighbourhood, so the single argmin
 * spans the whole cluster.  The cluster grows beyond the request until the
 * run's rows fit the CTAs' shared memory (K = 300 x T = 104 needs at least
 * 4 CTAs).
 * Results do not depend on it. */
int elsr_set_cluster(elsr_t *h, int32_t cluster);

/* Speculative execution of one GVNS run (mode P or G): up to `teams` clusters run
 * consecutive iterations from the same incumbent and commit them in order up
 * to the first acceptance, so trajectory, solution and counters equal the
 * sequential run's.  0 = automatic (up to 16 teams), 1 = off.  Every round
 * a team takes its position by ticket once all teams hold a ticket of the
 * previous round, and waits for the round's decision, so all teams must be
 * resident at once; their number is sized on an idle device.  When other
 * long-running work occupies the device, teams that cannot start leave the
 * others waiting, and after a few seconds the run ends with ELSR_E_TIMEOUT
 * instead of hanging; set 1 (off) for runs that share a busy device.
 * Batches and multi-start runs have no such waits. */
int elsr_set_speculation(elsr_t *h, int32_t teams);

/* Decode-step counter of the GVNS launches (elsr_stats_t.segments; a work
 * measure with no counterpart in the paper): on = 1 (the default) counts
 * the decode steps of every evaluated move, on = 0 skips that bookkeeping
 * (a few population counts per move) and reports segments = 0, e.g. while a
 * run is timed.  Results and every other counter are the same either way.
 * ELSR_E_ARG unless on is 0 or 1. */
int elsr_set_count_steps(elsr_t *h, int32_t on);

/* Launch shape of the last GVNS launch: shape[8] = {lanes per row, threads
 * per block, CTAs per run, blocks, shared bytes per block, prefix tables in
 * shared memory (0/1), 64-bit words per bit row, speculative teams}. */
int elsr_launch_shape(elsr_t *h, int32_t *shape);

/* Set the current solution from host 0/1 arrays gM, gR [K][T]; both NULL
 * restores the initial solution (every setup open). */
int elsr_set_state(elsr_t *h, const uint8_t *gM, const uint8_t *gR);

/* Copy the current solution to host gM, gR [K][T] (0/1). */
int elsr_get_state(elsr_t *h, uint8_t *gM, uint8_t *gR);

/* Row costs of the current solution to host rowcost[K]; *total (nullable)
 * receives their saturating sum (Section 2 objective). */
int elsr_cost(elsr_t *h, int64_t *rowcost, int64_t *total);

/*
 * One best-improvement evaluation of the neighbourhoods in nb_mask (bit j-1
 * selects N_j) at the current solution; nothing is applied.  This is
 * Algorithm 1's best-neighbour search over every product in one launch.
 *   mode ELSR_MODE_P: pp_cost[k], pp_move[k] = lexicographic minimum of
 *     (new row cost, combined local index) over product k's moves (cost
 *     ELSR_INF / move -1 when the row has none); *best_cost = the current
 *     objective minus the summed improvements, i.e. the objective after
 *     every product applies its best move when that move strictly improves
 *     its row; *best_move = number of such products.
 *   mode ELSR_MODE_G: *best_cost, *best_move = lexicographic minimum of
 *     (new objective, combined global index); pp_* as in mode P.
 * Outputs are host pointers and may be NULL.  Adds the moves to the
 * handle's evaluation counter.  Synchronous.  The first call for a (mode,
 * nb_mask) pair records the call's device work (reset of the reduction
 * words, the kernel, the copy of the results) as a CUDA graph owned by the
 * handle, which allocates; later calls replay it on the handle's stream.
 * Changing the lanes per row (elsr_set_launch) drops the graphs.  Callers
 * that must not allocate use elsr_eval_neighbourhood_static.
 */
int elsr_eval_neighbourhood(elsr_t *h, uint32_t nb_mask, int32_t mode,
                            int64_t *best_cost, int64_t *best_move,
                            int64_t *pp_cost, int64_t *pp_move);

/* New cost of the moved row for every move of N_nb (global layout, host
 * costs[|N_nb|]); window (nullable, host int32[|N_nb|]) receives each move's
 * decode steps: the setup segments of the moved row that a re-decode visits
 * before its stock on hand equals the row's (relaxed) decode again, up to
 * the one where it falls short (a work measure, not part of the method).
 * Synchronous. */
int elsr_move_costs(elsr_t *h, int32_t nb, int64_t *costs, int32_t *window);

/*
 * GVNS of Algorithm 2 (reading: shake with k moves of N_k drawn by
 * splitmix64 keyed by (seed, iteration, k, move), VND (Algorithm 1, pipe
 * form), keep x'' iff f(x'') < f(x), k back to 1 on improvement, else k+1
 * wrapping after kmax; an iteration budget replaces the time limit) from the
 * current solution, entirely on the device.  iters >= 0, 1 <= kmax <= 3,
 * mode ELSR_MODE_P or ELSR_MODE_G.  The current solution is not modified.
 * Asynchronous: the work is queued on the handle's stream; elsr_result()
 * waits for it.  iters = 0 runs VND alone.  A run keeps its rows in the
 * shared memory of one thread-block cluster of at most 16 CTAs (about 1,000
 * products at T = 128, 2,500 at T = 52); a larger instance is refused with
 * ELSR_E_RANGE before anything is launched.  The evaluation calls have no
 * such limit.
 */
int elsr_vns_run(elsr_t *h, uint64_t seed, int32_t iters, int32_t kmax,
                 int32_t mode);

/*
 * Algorithm 2 as the paper runs it on two GPUs (Section 3, fork-join model),
 * with `workers` workers on this GPU.  In every iteration each worker p
 * shakes the incumbent x with the iteration's k and its own draws (move j
 * of worker p is drawn as draw(seed, it, k, p << 8 | j), so worker 0 draws
 * exactly as elsr_vns_run does) and runs VND (mode P or G) on its copy; the
 * least (f(x''_p), p) replaces x when it is below f(x), and k goes back to 1,
 * else k+1, wrapping after kmax.  x starts as VND of the current solution.
 * Each worker is one team of CTAs (the handle's cluster and launch
 * settings) and all workers run at once, so `workers` may not exceed the
 * teams the device holds resident for this instance (ELSR_E_RANGE, with the
 * number in elsr_last_error) nor ELSR_FJ_WORKERS_MAX (ELSR_E_ARG).  Every
 * worker's VND counts in the statistics.  The workers meet at a grid
 * barrier every iteration, so on a device busy with other work the run may
 * end with ELSR_E_TIMEOUT (see elsr_set_speculation).  elsr_result() returns x, the
 * statistics and the trajectory; an entry's `reserved` field holds the
 * winning worker.  With one worker the run equals elsr_vns_run's.
 * Asynchronous, like elsr_vns_run.
 */
#define ELSR_FJ_WORKERS_MAX 4096
int elsr_vns_forkjoin_run(elsr_t *h, uint64_t seed, int32_t iters,
                          int32_t kmax, int32_t mode, int32_t workers);

/*
 * Wall-clock budget of the handle's next single runs (elsr_vns_run,
 * elsr_vns_forkjoin_run, elsr_vns_resume), in microseconds from the start
 * of each run on the device; 0 (the default) = none.  This is Algorithm 2's
 * stopping test on elapsed time: the run stops after the first iteration whose VND ends
 * past the budget (iters stays an upper bound), so its trajectory is a
 * prefix of the unbudgeted run's and elsr_checkpoint / elsr_vns_resume can
 * continue it.  A budgeted sequential run uses one team (no speculation).
 */
int elsr_set_time_limit(elsr_t *h, int64_t time_limit_us);

/*
 * Checkpoint of the last single run (elsr_vns_run, elsr_vns_forkjoin_run or
 * elsr_vns_resume; waits for it): *ck receives the loop state after its last
 * iteration, gM, gR (nullable together, host [K][T] 0/1) the incumbent x.
 * Returns the run's status (ELSR_OK, ELSR_E_CAP, ELSR_E_TIMEOUT,
 * ELSR_E_STATE) or an error; only an ELSR_OK checkpoint can be resumed.
 */
int elsr_checkpoint(elsr_t *h, elsr_checkpoint_t *ck, uint8_t *gM, uint8_t *gR);

/*
 * Continue a checkpointed run for `iters` more iterations (iterations
 * ck->next_it .. ck->next_it + iters - 1) from x = (gM, gR), host [K][T]
 * 0/1, with the checkpoint's seed, kmax, mode, k, trajectory hash and
 * workers (0: sequential GVNS, else fork-join).  There is no initial VND (x
 * is already VND's output), so a run of N iterations, a checkpoint and a
 * resume of M give exactly the run of N + M iterations: trajectory, x, hash
 * and totals.  x becomes the handle's current solution (as elsr_set_state;
 * this part waits for the device).  The handle may be a fresh one on the
 * same instance.  If f(x) differs from ck->cost the run stops before its
 * first iteration with status ELSR_E_STATE.  Then asynchronous, like
 * elsr_vns_run; elsr_result reports totals since iteration 0 and the
 * trajectory entries of this part.
 */
int elsr_vns_resume(elsr_t *h, const elsr_checkpoint_t *ck, const uint8_t *gM,
                    const uint8_t *gR, int32_t iters);

/*
 * Results of the last elsr_vns_run, elsr_vns_forkjoin_run or
 * elsr_vns_resume (waits for it).  stats (nullable); gM,
 * gR (nullable, host [K][T] 0/1) receive x; plan (nullable, host int32
 * [4][K][T]) receives xM, xR, yM, yR of x; traj (nullable, host
 * [traj_capacity]) receives the first min(iters, traj_capacity) entries.
 * Returns the run's status (ELSR_OK or ELSR_E_CAP) or an error.
 */
int elsr_result(elsr_t *h, elsr_stats_t *stats, uint8_t *gM, uint8_t *gR,
                int32_t *plan, elsr_traj_t *traj, int32_t traj_capacity);

/*
 * Multi-start GVNS on the handle's instance: nstarts independent runs from
 * the current solution, start s using seed seed0 + s, run concurrently in one
 * persistent launch; the best start is the lexicographic minimum of
 * (cost, s), reduced on the device.  Synchronous.  best_cost, best_start
 * (nullable) receive the winner; costs (nullable, host [nstarts]) every
 * start's cost.  elsr_result() afterwards reports the winning start.
 */
int elsr_multistart_run(elsr_t *h, uint64_t seed0, int32_t nstarts,
                        int32_t iters, int32_t kmax, int32_t mode,
                        int64_t *best_cost, int32_t *best_start,
                        int64_t *costs);

/*
 * Allocation-free neighbourhood evaluation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory,
 * such as a framework whose own pool owns all device memory, a serving loop
 * that must never call cudaMalloc or cudaFree (both can synchronise the
 * whole device), or code that records work while allocation is unavailable.
 *
 * It computes exactly what elsr_eval_neighbourhood computes (same modes,
 * masks and outputs), but every pointer is a caller-owned DEVICE pointer:
 * D, R int32 [K][T]; kM, kR, hM, hR int32 [K]; gM, gR uint8 0/1 [K][T];
 * best int64 [2] receives (best_cost, best_move); pp_cost, pp_move int64
 * [K] (nullable) receive the per-product results.  The instance must obey
 * the value ranges of elsr_create; they are not checked here (values are on
 * the device), and values outside them give unspecified results.
 *
 * Nothing is allocated: intermediate data lives in a fixed device array of
 * ELSR_STATIC_BYTES, which every GPU that loads the library holds until the
 * process exits.  Sizes beyond K <= ELSR_STATIC_K_MAX or T <= ELSR_T_MAX are
 * rejected with ELSR_E_RANGE.  The work is queued on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and the call returns without
 * waiting; outputs are valid once the stream reaches that point.  The first
 * call on each device looks up the array's device address; make that first
 * call before any stream capture.  All calls share the array and it keeps
 * the last call's contents, so calls that may overlap on the device (other
 * streams, other host threads) race on it and must be serialised.  The
 * stream and every buffer must belong to the current device (ELSR_E_ARG for
 * a stream or a device buffer of another device).  A CUDA error that an
 * earlier call of the caller left pending is reported as ELSR_E_CUDA before
 * any work is queued, and left pending.
 */
#define ELSR_STATIC_K_MAX 4096
#define ELSR_STATIC_BYTES (512 + 48 * ELSR_STATIC_K_MAX)
int elsr_eval_neighbourhood_static(int32_t K, int32_t T, const int32_t *D,
                                   const int32_t *R, const int32_t *kM,
                                   const int32_t *kR, const int32_t *hM,
                                   const int32_t *hR, const uint8_t *gM,
                                   const uint8_t *gR, uint32_t nb_mask,
                                   int32_t mode, int64_t *best,
                                   int64_t *pp_cost, int64_t *pp_move,
                                   void *stream);

/* Statistics of the first n starts of the last elsr_multistart_run (host
 * stats[n], start order). */
int elsr_multistart_stats(elsr_t *h, elsr_stats_t *stats, int32_t n);

/* Device moves evaluated since create (all calls on this handle). */
int elsr_counters(elsr_t *h, int64_t *moves_evaluated);

/*
 * Batches: n independent instances of possibly different K and T, solved by
 * one persistent launch (a CTA per run, runs taken from a device work
 * queue in descending order of size).  Ks, Ts: host [n]; D, R: host arrays
 * holding the instances' [K_i][T_i] blocks one after another; kM, kR, hM,
 * hR: host arrays holding the [K_i] blocks one after another.  Each instance
 * obeys the limits of elsr_create.  Copies everything.
 */
int elsr_batch_create(elsr_batch_t **out, int32_t n, const int32_t *Ks,
                      const int32_t *Ts, const int32_t *D, const int32_t *R,
                      const int32_t *kM, const int32_t *kR, const int32_t *hM,
                      const int32_t *hR);
/* As elsr_batch_create, with the batch's device memory allocated (stream
 * ordered) and its work issued on `stream` (a cudaStream_t) from the start;
 * elsr_batch_destroy then frees stream-ordered too, so creating and
 * destroying batches does not synchronise the device. */
int elsr_batch_create_on(elsr_batch_t **out, int32_t n, const int32_t *Ks,
                         const int32_t *Ts, const int32_t *D, const int32_t *R,
                         const int32_t *kM, const int32_t *kR,
                         const int32_t *hM, const int32_t *hR, void *stream);
/* As elsr_batch_create_on, with unit production costs pM, pR holding the
 * instances' [K_i] blocks one after another (both NULL = 0), under the
 * limits of elsr_create_ex. */
int elsr_batch_create_ex(elsr_batch_t **out, int32_t n, const int32_t *Ks,
                         const int32_t *Ts, const int32_t *D, const int32_t *R,
                         const int32_t *kM, const int32_t *kR,
                         const int32_t *hM, const int32_t *hR,
                         const int32_t *pM, const int32_t *pR, void *stream);
/* Free the batch and its device memory (stream-ordered on the batch's
 * stream, after the work already queued there).  NULL is ignored. */
void elsr_batch_destroy(elsr_batch_t *b);

/* Message of the last failed call on batch b (b NULL: last failed create on
 * this thread). */
const char *elsr_batch_last_error(const elsr_batch_t *b);
/* As elsr_set_stream, for a batch. */
int elsr_batch_set_stream(elsr_batch_t *b, void *stream);
/* As elsr_set_launch, for a batch: lanes_per_row 0 lets every run of the
 * batch pick its own row-group width (wider for runs with few products);
 * threads 0 = automatic (up to 1024 per CTA, one CTA per SM).  ELSR_E_ARG
 * outside the values elsr_set_launch accepts. */
int elsr_batch_set_launch(elsr_batch_t *b, int32_t lanes_per_row,
                          int32_t threads);

/* As elsr_set_cluster / elsr_launch_shape (shape[8]), for a batch (default:
 * 1 CTA per run). */
int elsr_batch_set_cluster(elsr_batch_t *b, int32_t cluster);
int elsr_batch_launch_shape(elsr_batch_t *b, int32_t *shape);

/* As elsr_set_count_steps, for a batch. */
int elsr_batch_set_count_steps(elsr_batch_t *b, int32_t on);

/* Instances per CTA of the next batch runs (a launch-shape choice that
 * changes no result; the paper's Algorithm 1 runs one instance per device).
 * With runs_per_cta = P > 1, every CTA of the persistent launch first takes
 * the runs whose rows need more than a P-th of its shared memory (longest
 * first, one run per CTA), then splits its threads into P partitions, each
 * running one of the remaining runs with its own barrier, so that small
 * runs do not leave row groups idle.  Applies to launches of one CTA per run
 * with at most 32 lanes per row and blocks of 512 threads or more that
 * divide into P partitions of whole warps; otherwise one run per CTA.  0 = automatic
 * (the library's choice), else a power of two <= 8; ELSR_E_ARG otherwise. */
int elsr_batch_set_runs_per_cta(elsr_batch_t *b, int32_t runs_per_cta);

/* Packing of the last launch: *runs_per_cta (1 when none) and
 * *whole_cta_runs, the runs that took a whole CTA before the partitions. */
int elsr_batch_packing(const elsr_batch_t *b, int32_t *runs_per_cta,
                       int32_t *whole_cta_runs);

/* (Re)build, on the batch's stream, the per-row prefix tables of every
 * instance in device memory: for row k of instance i, the cumulative demand
 * and returns of periods 0..t and the constant part of the row cost, the
 * quantities whose differences give the holding costs in the objective of
 * Section 2 for any setup pattern of the row.  Runs whose
 * rows do not fit shared memory read these tables; the batch builds them on
 * the first such run, and this call builds them again (to prebuild them, or
 * to time the pass: it reads D, R, hM, hR and pM once and writes
 * (cells + rows) * 8 + rows * 8 bytes).  Asynchronous; ELSR_E_ARG for a NULL
 * batch, ELSR_E_CUDA when the allocation or launch fails. */
int elsr_batch_stage_tables(elsr_batch_t *b);

/* Queue GVNS runs of every instance i with seeds[i] (host [n]), from the
 * initial solution.  Asynchronous, like elsr_vns_run. */
int elsr_batch_run(elsr_batch_t *b, const uint64_t *seeds, int32_t iters,
                   int32_t kmax, int32_t mode);

/* Wait for the batch and copy per-instance results: stats (nullable, host
 * [n]).  Returns ELSR_E_CAP when any run hit the cap. */
int elsr_batch_results(elsr_batch_t *b, elsr_stats_t *stats);

/* Solution of instance i of the last batch run: gM, gR host [K_i][T_i]. */
int elsr_batch_solution(elsr_batch_t *b, int32_t i, uint8_t *gM, uint8_t *gR);

/*
 * Serving (the paper has one instance per run; serving requests of many
 * instances as they arrive is this library's).  A server holds fixed-size
 * device pools for the instances of the requests in flight and solves each
 * request's GVNS run (Algorithm 2 with Algorithm 1's VND, mode P or G, from
 * the all-open start) exactly as elsr_vns_run would: the same statistics
 * and trajectory hash, whatever else is in flight.  Requests join the
 * kernels already running and retire one by one, in any order.
 *
 * Requests are grouped by the CTAs (1..16) their rows need and by T <= 64 or
 * not; each group has a queue in device memory.  A launch of a group runs
 * one team per CTA cluster; a team takes the next queued request, solves
 * it, writes its statistics into host memory and takes the next, and exits
 * when the queue is empty or after max_runs requests (leaving its SMs to
 * other groups).  Nothing on the device waits for the host; the host
 * launches a group again while it has requests not yet retired.  Work is
 * issued on streams the server owns; every call returns without waiting for
 * the device.  A server uses the device that is current at creation; call it
 * with that device current, from one host thread at a time.
 */
typedef struct elsr_server elsr_server_t;

typedef struct {
    int32_t slots;          /* requests in flight at most; 0: 2048 */
    int32_t threads;        /* threads per CTA, a multiple of 32 <= 1024; 0: 1024 */
    int64_t cells;          /* demand/return values the pools hold; 0: 8 Mi */
    int64_t rows;           /* product rows the pools hold; 0: 512 Ki */
    int32_t max_runs;       /* requests a team solves before it exits; 0: 1 */
    int32_t acc64;          /* 1: 64-bit row accumulators (admits any instance);
                               0: 32-bit (refuses instances that need 64) */
    int32_t count_steps;    /* 1: count decode steps (stats.segments); 0: not */
    int32_t keep_solutions; /* 1: a reported request keeps its solution until
                               elsr_server_release; 0: freed when reported */
} elsr_server_config_t;

/* Create a server (cfg NULL: every default, steps not counted, solutions
 * not kept).  Allocates its pools (device), staging buffers (pinned host)
 * and result words (host memory mapped into the device).  ELSR_E_ARG for an
 * invalid field, ELSR_E_NOMEM / ELSR_E_CUDA when an allocation fails. */
int elsr_server_create(elsr_server_t **out, const elsr_server_config_t *cfg);

/* Waits for the server's launches and copies, then frees everything. */
void elsr_server_destroy(elsr_server_t *s);

const char *elsr_server_last_error(const elsr_server_t *s);

/*
 * Submit one request: an instance as in elsr_create (host arrays D, R
 * [K][T], kM, kR, hM, hR [K], copied: the caller keeps them) and a GVNS run
 * (seed, iters, kmax <= 3, mode).  *ticket receives the request's ticket.
 * Admission by footprint: the request needs a free slot, K*T cells and K
 * rows of the pools; when they are not free now the call returns
 * ELSR_E_BUSY (retry after elsr_server_poll reports completions).
 * ELSR_E_RANGE when it can never be admitted: it exceeds the pools, its rows
 * need more than 16 CTAs, or it needs 64-bit accumulators on a 32-bit
 * server; ELSR_E_ARG / ELSR_E_RANGE as elsr_create for the instance.
 */
int elsr_server_submit(elsr_server_t *s, int32_t K, int32_t T, const int32_t *D,
                       const int32_t *R, const int32_t *kM, const int32_t *kR,
                       const int32_t *hM, const int32_t *hR, uint64_t seed,
                       int32_t iters, int32_t kmax, int32_t mode, int64_t *ticket);

/* Report up to max retired requests: tickets[i] (host) and, when stats is
 * not NULL, their statistics as elsr_result reports them (status ELSR_OK,
 * ELSR_E_CAP or ELSR_E_CUDA).  Returns how many (>= 0) or a negative error.
 * Also launches groups that still have requests to solve; a caller polls
 * until every ticket it submitted has been reported. */
int elsr_server_poll(elsr_server_t *s, int32_t max, int64_t *tickets,
                     elsr_stats_t *stats);

/* Solution of a retired request (host gM, gR [K][T] 0/1): before the poll
 * that reports it, or after it on a server that keeps solutions.
 * ELSR_E_STATE when the ticket has not retired or is no longer held. */
int elsr_server_solution(elsr_server_t *s, int64_t ticket, uint8_t *gM, uint8_t *gR);

/* Free a reported request of a server that keeps solutions. */
int elsr_server_release(elsr_server_t *s, int64_t ticket);

/* Requests in flight (submitted, not yet freed) and kernel launches so far
 * (either pointer may be NULL). */
int elsr_server_info(const elsr_server_t *s, int64_t *inflight, int64_t *launches);

/*
 * Integer-issue probe, a measurement aid with no counterpart in the paper:
 * it measures the denominator of the integer roofline that throughput
 * figures of the GVNS kernels are compared with.  Queues one launch on
 * `stream` (a cudaStream_t; NULL = legacy default stream) of `blocks` CTAs
 * of 256 threads; every thread runs `iters` x 16 steps of eight independent
 * chains, one step being one 32-bit add, minimum, exclusive-or and
 * multiply-add.  src: caller-owned device int32[36] of operands (any
 * values); sink: caller-owned device int32[blocks * 256], overwritten.
 * *ops (host) receives the integer operations the launch performs, to be
 * divided by its duration measured on the stream.  Returns without waiting;
 * ELSR_E_ARG for non-positive sizes or NULL pointers, ELSR_E_CUDA when the
 * launch fails.
 */
int elsr_int_issue_probe(void *stream, int32_t blocks, int32_t iters,
                         const int32_t *src, int32_t *sink, int64_t *ops);

#ifdef __cplusplus
}
#endif

#endif /* ELSR_H */
