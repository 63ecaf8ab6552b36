// elsr_internal.h -- device data layout and kernel launchers shared by the
// kernels (elsr_kernels.cu) and the C ABI (elsr_abi.cu).  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "elsr_row.cuh"

namespace elsr {

constexpr int kTMax = 128;
constexpr int kMaxShake = 3;        // kmax <= 3: at most 3 shaken rows
constexpr int kSmemLimit = 227 * 1024 - 1024;  // dynamic bytes; static control words (< 1 KB) take the rest
constexpr int kStatusCap = -5;      // ELSR_E_CAP
constexpr int kStatusTimeout = -7;  // ELSR_E_TIMEOUT
constexpr int kStatusState = -6;    // ELSR_E_STATE: resumed state does not match
constexpr int kStatusLaunch = -4;   // ELSR_E_CUDA: launch geometry mismatch
// Control words at the start of each partition's shared memory when a CTA
// holds several runs (the kernels check that they fit).
constexpr uint32_t kPartCtlBytes = 768;
constexpr int kMaxParts = 8;        // runs per CTA: partitions of >= 128 threads

// One instance of a batch: rows [row_off, row_off + K) of the per-row pools
// and cells [cell_off, cell_off + K*T) of the D/R pools.
struct InstDesc {
  int32_t K, T;
  int64_t cell_off;
  int64_t row_off;
  int64_t tab_off;  // into the global prefix-table pool (K*(T+1) entries)
};

// One GVNS run: instance, budget and where its outputs go.
struct RunDesc {
  int32_t inst;
  int32_t iters;
  int32_t kmax;
  int32_t mode;
  uint64_t seed;
  int32_t out;        // index into the per-run outputs
  int32_t tag;        // echoed when a served request retires (serving: its ticket)
  int64_t bits_off;   // RowBits offset of this run's solution output
  int64_t start_off;  // RowBits offset of its start solution (-1: all open)
  int64_t traj_off;   // trajectory entry offset (-1: none)
  // Continuation of a checkpointed run: iterations it0 .. it0 + iters - 1
  // from the start solution (already VND's output, so no initial VND) with
  // k = k0, trajectory hash h0, and the start's objective f0 (checked).
  int32_t it0 = 0;
  int32_t k0 = 1;
  uint64_t h0 = 0;
  int64_t f0 = 0;
  int32_t resume = 0;
  int32_t pad1 = 0;
  // Wall-clock budget (Algorithm 2's time limit), nanoseconds from the
  // run's start; 0 = none.  The run stops after the first iteration that
  // ends past it.
  int64_t time_limit_ns = 0;
};

struct RunOut {
  int64_t best_cost;
  uint64_t traj_hash;
  int64_t moves_evaluated, evals, vnd_cycles, applied, iterations, accepted;
  int64_t segments;
  int32_t status;
  int32_t reserved;
  int32_t k_next;  // k of the iteration after the last one run
  int32_t pad;
};

struct TrajEntry {
  int32_t it;
  int32_t k;
  int64_t cost;
  int32_t accepted;
  int32_t reserved;
};

// Raw instance pools (device).
struct InstPools {
  const InstDesc* insts;
  const int32_t* D;
  const int32_t* R;
  const int32_t* kM;
  const int32_t* kR;
  const int32_t* hM;
  const int32_t* hR;
  const int2* gtab;    // global prefix tables (when not staged in smem)
  const int64_t* gC0;  // per-row constants matching gtab
  const int32_t* pM;   // unit production costs per row (nullable: 0)
  const int32_t* pR;
};

// One speculative team's result for one round (spec_kernel).
struct SpecSlot {
  long long f2;
  int cycles;
  int done;  // round number whose result this slot holds
  unsigned long long applied;
  unsigned long long steps;
};

struct VnsParams {
  InstPools ip;
  const RunDesc* runs;
  int32_t nruns;
  int32_t G;  // sub-warp lanes per row
  int32_t vnd_cap;
  int32_t count_steps;  // 1: count decode steps (RunOut.segments), 0: skip (timing)
  const RowBits* start_bits;
  RowBits* out_bits;
  RunOut* out;
  TrajEntry* traj;
  int32_t* queue;  // [2] work counters (whole-CTA runs, partition runs), zero at launch
  // speculative single-run launches (spec_teams > 1)
  int32_t spec_teams;
  int32_t cluster;       // CTAs per team the launch was configured with
  SpecSlot* spec_slots;  // [2][spec_teams]
  RowBits* spec_rows;    // [2][spec_teams][3]
  int32_t* spec_bar;     // [2]: speculation: tickets taken; fork-join: arrivals, generation; zero at launch
  int32_t* spec_dec;     // [2]: per round parity, (round tag << 8) | first accepting position; zero at launch
  // fork-join launches (Algorithm 2 with one shake + VND per worker): the
  // fj_workers teams share spec_slots, spec_rows and spec_bar (0: off)
  int32_t fj_workers;
  // batched launches: choose each run's lanes per row from its row count
  // (wider groups for small instances); 0 = every run uses G
  int32_t adaptive_G;
  // instances per CTA: runs [0, n_whole) take a whole team each; with
  // parts > 1 (cluster size 1, G <= 32) the CTA then splits into `parts`
  // partitions of its threads, each a team with part_bytes of dynamic shared
  // memory, for runs [n_whole, nruns)
  int32_t parts;
  int32_t n_whole;
  uint32_t part_bytes;
  int32_t pad2;
};

// Serving queue of one request class (CTAs per team, words per bit row):
// the host appends slot numbers at slots[tail % cap] and then publishes the
// new tail; teams claim positions head .. tail - 1.  A retired request's slot
// gets done[slot] = its RunDesc tag + 1, in memory the host reads directly.
struct SrvQueue {
  const int32_t* slots;  // [cap] slot of each queue position (mod cap)
  int32_t* head;         // positions claimed
  const int32_t* tail;   // positions published
  int32_t* done;         // [slots of the server] retire words (host-mapped)
  int32_t cap;
  int32_t max_runs;      // requests a team serves before it exits (yields its SMs)
};

struct StageParams {
  InstPools ip;
  int32_t ninst;
  int2* gtab;
  int64_t* gC0;
};

// Single-instance neighbourhood evaluation (instance 0 of the pools).
struct EvalParams {
  InstPools ip;
  int32_t K, T;
  const RowBits* bits;       // current solution [K]
  const int64_t* rowcost_in; // [K] current row costs (mode G "others")
  uint32_t mask;
  int32_t mode;
  int32_t G;
  int32_t single_j;          // j of the per-move outputs (0: none)
  int64_t* rowcost_out;      // [K] nullable
  uint64_t* pp_key;          // [K] nullable: per-product best (cost, local)
  int64_t* move_cost;        // [K*row_moves(single_j)] nullable
  int32_t* move_win;         // same, nullable
  uint64_t* scratch;         // [4]: gkey, sum_after, ninf_after, n_improving
};

struct BestofParams {
  const RunOut* out;
  int32_t n;
  uint64_t* best_key;  // pack_key(cost, run)
};

struct PlanParams {
  InstPools ip;
  int32_t inst;
  const RowBits* bits;  // [K]
  int32_t* plan;        // [4][K][T]
};

// Shared-memory layout of the rows one CTA owns in the persistent GVNS
// kernel (Kc rows of T periods).
struct VnsLayout {
  uint32_t tab, rc, C0, bits, S, mark, nR, A, C, L, P, Q, save, slot, total;
};

ELSR_HD uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

ELSR_HD VnsLayout vns_layout(int Kc, int T, int acc_bytes, bool tab_smem) {
  VnsLayout L;
  uint32_t o = 0;
  const uint32_t K = (uint32_t)Kc, TT = (uint32_t)T, ab = (uint32_t)acc_bytes;
  L.tab = o;
  if (tab_smem) o = align16(o + K * (TT + 1) * 8u);
  L.rc = o;
  o = align16(o + K * (uint32_t)sizeof(RowCosts));
  L.C0 = o;
  o = align16(o + K * 8u);
  L.bits = o;
  o = align16(o + K * 32u);
  L.S = o;
  o = align16(o + K * ab);
  L.mark = o;
  o = align16(o + K * 4u);
  L.nR = o;
  o = align16(o + K * 4u);
  L.A = o;
  o = align16(o + K * TT * 4u);
  L.C = o;
  o = align16(o + K * TT * ab);
  L.L = o;
  o = align16(o + K * TT * 8u);
  L.P = o;
  o = align16(o + K * (TT + 1) * 4u);
  L.Q = o;
  o = align16(o + K * (TT + 1) * ab);
  // save slot: RowBits(32) S(8) mark(4) nR(4) | A[T] | C[T] | L[T] | P[T+1] | Q[T+1]
  L.slot = align16(48u + ((TT * 4u + 7u) & ~7u) + ((TT * ab + 7u) & ~7u) + TT * 8u +
                   (((TT + 1) * 4u + 7u) & ~7u) + (TT + 1) * ab);
  L.save = o;
  o += 2u * kMaxShake * L.slot;
  L.total = o;
  return L;
}

// Create-time checks of one instance without unit production costs (the
// ranges of elsr.h); sets *acc64 when its rows need 64-bit accumulators.
int validate_instance(int32_t K, int32_t T, const int32_t* D, const int32_t* R,
                      const int32_t* kM, const int32_t* kR, const int32_t* hM,
                      const int32_t* hR, bool* acc64, std::string& err);

// Launchers.  Each returns the launch error.
cudaError_t launch_stage(const StageParams& p, int total_rows, cudaStream_t s);
cudaError_t launch_eval(const EvalParams& p, bool acc64, int blocks,
                        int threads, size_t smem, cudaStream_t s);
cudaError_t eval_prepare(bool acc64, int T, size_t smem);
// One row of instance 0 per CTA, `threads` (a multiple of 32, <= 128) on its
// moves; grid = p.K.  Shared memory fits the default limit (T <= 128).
cudaError_t launch_eval_wide(const EvalParams& p, bool acc64, int threads, cudaStream_t s);
size_t eval_smem_bytes(int rows, int T, bool acc64);
cudaError_t launch_bestof(const BestofParams& p, cudaStream_t s);
cudaError_t launch_plan(const PlanParams& p, int K, cudaStream_t s);

// Persistent GVNS kernels (elsr_vns.cuh), one instantiation per accumulator
// width (Acc), 64-bit words per bit row (NW = 1 when T <= 64), prefix tables
// in shared memory (TS) and block size bound (MAXT = 256, 512 or 1024); each
// combination is compiled in a translation unit of its own
// (elsr_vns_inst.cu).  prepare sets the kernel attributes and returns the
// resident blocks per SM (cluster == 1) or the resident clusters on the
// device (cluster > 1).  launch starts the batched kernel, the speculative
// one (p.spec_teams > 1) or the fork-join one (p.fj_workers > 0).
template <typename Acc, int NW, bool TS, int MAXT>
cudaError_t vns_prepare_t(size_t smem, int threads, int cluster, int* active);
template <typename Acc, int NW, bool TS, int MAXT>
cudaError_t vns_launch_t(const VnsParams& p, int blocks, int threads, size_t smem,
                         int cluster, cudaStream_t s);

// Serving kernel (elsr_vns.cuh, prefix tables in shared memory, 1024-thread
// bound), instantiated per accumulator width and words per bit row.
template <typename Acc, int NW>
cudaError_t srv_prepare_t(size_t smem, int threads, int cluster, int* active);
template <typename Acc, int NW>
cudaError_t srv_launch_t(const VnsParams& p, const SrvQueue& q, int blocks, int threads,
                         size_t smem, int cluster, cudaStream_t s);
cudaError_t srv_prepare(bool acc64, int nw, size_t smem, int threads, int cluster, int* active);
cudaError_t srv_launch(bool acc64, int nw, const VnsParams& p, const SrvQueue& q, int blocks,
                       int threads, size_t smem, int cluster, cudaStream_t s);

// Run-time choice of the instantiation (elsr_vns_dispatch.cu).
cudaError_t vns_prepare(bool acc64, int nw, bool ts, int maxt, size_t smem, int threads,
                        int cluster, int* active);
cudaError_t vns_launch(bool acc64, int nw, bool ts, int maxt, const VnsParams& p,
                       int blocks, int threads, size_t smem, int cluster, cudaStream_t s);

}  // namespace elsr
