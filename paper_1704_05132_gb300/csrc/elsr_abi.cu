// elsr_abi.cu -- C ABI of include/elsr.h: validation, device memory, launch
// configuration and result marshalling around the kernels of
// elsr_kernels.cu.  No arithmetic of the method runs here; every step of the
// search runs in the kernels.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/elsr.h"
#include "elsr_internal.h"

using namespace elsr;

namespace {

thread_local std::string g_create_error;

const int kVndCap = 1 << 20;

// A failed CUDA call sets the handle's message and returns ELSR_E_NOMEM for
// a failed allocation, else ELSR_E_CUDA.
#define ELSR_TRY_CUDA(obj, call)                                               \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      (obj)->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
      return e_ == cudaErrorMemoryAllocation ? ELSR_E_NOMEM : ELSR_E_CUDA;     \
    }                                                                          \
  } while (0)

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// owner's stream), so allocating or freeing a batch never synchronises the
// device while other batches run.
template <typename T>
cudaError_t dev_alloc(T** p, size_t n, cudaStream_t s) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMallocAsync((void**)p, n * sizeof(T), s);
}

template <typename T>
void dev_free(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync((void*)p, s);
  p = nullptr;
}

// Create-time checks of one instance (ranges documented in elsr.h).  Sets
// *acc64 when a row's magnitude bound needs 64-bit accumulators.
int check_instance(int32_t K, int32_t T, const int32_t* D, const int32_t* R,
                   const int32_t* kM, const int32_t* kR, const int32_t* hM,
                   const int32_t* hR, const int32_t* pM, const int32_t* pR, bool* acc64,
                   unsigned __int128* total, std::string& err) {
  if (K < 1 || T < 1 || T > ELSR_T_MAX) {
    err = "K must be >= 1 and 1 <= T <= " + std::to_string(ELSR_T_MAX);
    return ELSR_E_ARG;
  }
  if (!D || !R || !kM || !kR || !hM || !hR) {
    err = "null instance array";
    return ELSR_E_ARG;
  }
  if ((int64_t)K * (4 * (int64_t)T) >= (1 << 24)) {
    err = "K*T too large for 24-bit move indices";
    return ELSR_E_RANGE;
  }
  for (int32_t k = 0; k < K; ++k) {
    const int64_t pm = pM ? pM[k] : 0, pr = pR ? pR[k] : 0;
    if (kM[k] < 0 || kR[k] < 0 || hM[k] < 0 || hR[k] < 0 || pm < 0 || pr < 0) {
      err = "negative cost in product " + std::to_string(k);
      return ELSR_E_ARG;
    }
    if (pm >= (1 << 24) || pr >= (1 << 24)) {
      err = "unit production cost of product " + std::to_string(k) + " exceeds 2^24";
      return ELSR_E_RANGE;
    }
    int64_t sd = 0, sr = 0, wd = 0, wr = 0;
    for (int32_t t = 0; t < T; ++t) {
      const int32_t d = D[(int64_t)k * T + t], r = R[(int64_t)k * T + t];
      if (d < 0 || r < 0) {
        err = "negative demand or return at (" + std::to_string(k) + "," +
              std::to_string(t) + ")";
        return ELSR_E_ARG;
      }
      sd += d;
      sr += r;
      wd += (int64_t)d * (T - t);
      wr += (int64_t)r * (T - t);
    }
    if (sd >= (1ll << 31) || sr >= (1ll << 31)) {
      err = "sum of demand or returns of product " + std::to_string(k) +
            " exceeds 2^31";
      return ELSR_E_RANGE;
    }
    unsigned __int128 b = (unsigned __int128)T * ((uint64_t)kM[k] + (uint64_t)kR[k]);
    b += (unsigned __int128)T * ((unsigned __int128)hM[k] * sd + (unsigned __int128)hR[k] * sr);
    b += (unsigned __int128)hM[k] * wd + (unsigned __int128)hR[k] * wr;
    b += (unsigned __int128)(pm + pr) * sd;  // pM * sum D + |pR - pM| * sum xR
    if (b >= ((unsigned __int128)1 << 30) || (int64_t)hR[k] * T + pm + pr >= (1ll << 30))
      *acc64 = true;
    *total += b;
  }
  if (*total >= ((unsigned __int128)1 << 40) - 1) {
    err = "objective bound exceeds 2^40";
    return ELSR_E_RANGE;
  }
  return ELSR_OK;
}

// Default lanes per row: single runs are latency-bound and spread each row
// over more lanes; batches are throughput-bound and keep more rows in flight.
int default_lanes(int T, bool single) {
  if (single) return T <= 8 ? 4 : (T <= 16 ? 8 : (T <= 24 ? 16 : (T <= 40 ? 32 : 64)));
  return T <= 8 ? 4 : (T <= 24 ? 8 : 16);
}

}  // namespace

namespace elsr {

int validate_instance(int32_t K, int32_t T, const int32_t* D, const int32_t* R,
                      const int32_t* kM, const int32_t* kR, const int32_t* hM,
                      const int32_t* hR, bool* acc64, std::string& err) {
  unsigned __int128 total = 0;
  *acc64 = false;
  return check_instance(K, T, D, R, kM, kR, hM, hR, nullptr, nullptr, acc64, &total, err);
}

}  // namespace elsr

// ---------------------------------------------------------------------------
// Batch (a set of instances resident on the device)
// ---------------------------------------------------------------------------
struct elsr_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int32_t n = 0;
  std::vector<InstDesc> insts;
  int64_t cells = 0, rows = 0;
  int maxK = 0, maxT = 0;
  bool acc64 = false;
  int lanes = 0, threads = 0, cluster = 0;  // 0 = defaults
  int parts = 0;                             // runs per CTA (0: automatic)
  int count_steps = 1;                       // decode-step counter on (1) or off
  int last_parts = 1, last_whole = 0;        // packing of the last launch
  int spec = 0;                              // speculative teams (0 auto, 1 off)
  int last_shape[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int sms = 0;

  InstDesc* d_insts = nullptr;
  int32_t *d_D = nullptr, *d_R = nullptr, *d_kM = nullptr, *d_kR = nullptr,
          *d_hM = nullptr, *d_hR = nullptr;
  int2* d_tab = nullptr;  // global prefix tables (staged on demand)
  int64_t* d_C0 = nullptr;
  int32_t *d_pM = nullptr, *d_pR = nullptr;  // unit production costs (none: 0)
  bool tab_ready = false;

  RunDesc* d_runs = nullptr;
  size_t runs_cap = 0;
  RunOut* d_out = nullptr;
  size_t out_cap = 0;
  RowBits* d_bits = nullptr;
  size_t bits_cap = 0;
  TrajEntry* d_traj = nullptr;
  size_t traj_cap = 0;
  int32_t* d_queue = nullptr;
  uint64_t* d_bestkey = nullptr;
  SpecSlot* d_spec_slots = nullptr;
  RowBits* d_spec_rows = nullptr;
  int32_t* d_spec_bar = nullptr;
  int32_t* d_spec_dec = nullptr;
  size_t spec_cap = 0;

  std::vector<RunDesc> h_runs;
  std::vector<int32_t> out_of_inst;  // per instance: its output index
  int32_t nruns = 0;
  bool have_result = false;

  InstPools pools() const {
    InstPools p;
    p.insts = d_insts;
    p.D = d_D;
    p.R = d_R;
    p.kM = d_kM;
    p.kR = d_kR;
    p.hM = d_hM;
    p.hR = d_hR;
    p.gtab = d_tab;
    p.gC0 = d_C0;
    p.pM = d_pM;
    p.pR = d_pR;
    return p;
  }

  ~elsr_batch() {
    if (d_insts) cudaStreamSynchronize(stream);
    dev_free(d_insts, stream);
    dev_free(d_D, stream);
    dev_free(d_R, stream);
    dev_free(d_kM, stream);
    dev_free(d_kR, stream);
    dev_free(d_hM, stream);
    dev_free(d_hR, stream);
    dev_free(d_tab, stream);
    dev_free(d_C0, stream);
    dev_free(d_pM, stream);
    dev_free(d_pR, stream);
    dev_free(d_runs, stream);
    dev_free(d_out, stream);
    dev_free(d_bits, stream);
    dev_free(d_traj, stream);
    dev_free(d_queue, stream);
    dev_free(d_bestkey, stream);
    dev_free(d_spec_slots, stream);
    dev_free(d_spec_rows, stream);
    dev_free(d_spec_bar, stream);
    dev_free(d_spec_dec, stream);
  }
};

namespace {

int default_parts(const elsr_batch* b, int threads, int G) {
  // Measured on the 1024-instance batch (K ~ U{5..100}, T ~ U{12..52}, 1024
  // threads): 2 runs per CTA 226 ms, 1 run 260 ms, 4 runs 267 ms, 8 runs
  // 326 ms.  Packing only pays when there are runs enough to keep every
  // partition busy.
  const int64_t nr = (int64_t)b->h_runs.size();
  return (threads >= 512 && G <= 32 && nr >= 4ll * std::max(1, b->sms)) ? 2 : 1;
}

int batch_init(elsr_batch* b, int32_t n, const int32_t* Ks, const int32_t* Ts,
               const int32_t* D, const int32_t* R, const int32_t* kM,
               const int32_t* kR, const int32_t* hM, const int32_t* hR,
               const int32_t* pM = nullptr, const int32_t* pR = nullptr) {
  if ((pM == nullptr) != (pR == nullptr)) {
    b->err = "pM and pR must both be given or both be NULL";
    return ELSR_E_ARG;
  }
  if (n < 1 || !Ks || !Ts) {
    b->err = "batch needs n >= 1 and K/T arrays";
    return ELSR_E_ARG;
  }
  b->n = n;
  b->insts.resize(n);
  unsigned __int128 total_all = 0;
  for (int32_t i = 0; i < n; ++i) {
    InstDesc& d = b->insts[i];
    d.K = Ks[i];
    d.T = Ts[i];
    if (d.K < 1 || d.T < 1 || d.T > ELSR_T_MAX) {
      b->err = "instance " + std::to_string(i) + ": bad K or T";
      return ELSR_E_ARG;
    }
    d.cell_off = b->cells;
    d.row_off = b->rows;
    d.tab_off = b->rows + b->cells;  // K*(T+1) = K*T + K entries
    unsigned __int128 tot = 0;
    bool a64 = false;
    int rc = check_instance(d.K, d.T, D ? D + d.cell_off : nullptr,
                            R ? R + d.cell_off : nullptr,
                            kM ? kM + d.row_off : nullptr,
                            kR ? kR + d.row_off : nullptr,
                            hM ? hM + d.row_off : nullptr,
                            hR ? hR + d.row_off : nullptr, pM ? pM + d.row_off : nullptr,
                            pR ? pR + d.row_off : nullptr, &a64, &tot, b->err);
    if (rc != ELSR_OK) {
      b->err = "instance " + std::to_string(i) + ": " + b->err;
      return rc;
    }
    b->acc64 = b->acc64 || a64;
    total_all += tot;
    b->cells += (int64_t)d.K * d.T;
    b->rows += d.K;
    b->maxK = std::max(b->maxK, d.K);
    b->maxT = std::max(b->maxT, d.T);
  }
  (void)total_all;
  ELSR_TRY_CUDA(b, cudaGetDevice(&b->device));
  ELSR_TRY_CUDA(b, cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_insts, n, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_D, b->cells, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_R, b->cells, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_kM, b->rows, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_kR, b->rows, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_hM, b->rows, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_hR, b->rows, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_queue, 2, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_bestkey, 1, b->stream));
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_insts, b->insts.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice, b->stream));
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_D, D, b->cells * 4, cudaMemcpyHostToDevice, b->stream));
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_R, R, b->cells * 4, cudaMemcpyHostToDevice, b->stream));
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_kM, kM, b->rows * 4, cudaMemcpyHostToDevice, b->stream));
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_kR, kR, b->rows * 4, cudaMemcpyHostToDevice, b->stream));
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_hM, hM, b->rows * 4, cudaMemcpyHostToDevice, b->stream));
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_hR, hR, b->rows * 4, cudaMemcpyHostToDevice, b->stream));
  if (pM) {
    ELSR_TRY_CUDA(b, dev_alloc(&b->d_pM, b->rows, b->stream));
    ELSR_TRY_CUDA(b, dev_alloc(&b->d_pR, b->rows, b->stream));
    ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_pM, pM, b->rows * 4, cudaMemcpyHostToDevice, b->stream));
    ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_pR, pR, b->rows * 4, cudaMemcpyHostToDevice, b->stream));
  }
  ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));  // host arrays may be freed on return
  return ELSR_OK;
}

template <typename T>
int ensure(elsr_batch* b, T** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return ELSR_OK;
  dev_free(*p, b->stream);
  *cap = 0;
  ELSR_TRY_CUDA(b, dev_alloc(p, need, b->stream));
  *cap = need;
  return ELSR_OK;
}

struct LaunchShape {
  int nw, maxt;
  bool ts;
  size_t smem;
  int threads, G, cluster, blocks;
  int active;  // resident blocks per SM (cluster 1) or clusters on the device
  int parts = 1;            // runs per CTA in the partitioned phase
  int n_whole = 0;          // runs [0, n_whole) take a whole CTA (or cluster)
  uint32_t part_bytes = 0;  // dynamic shared bytes per partition
};

// Runs per CTA when the caller leaves it to the library: small runs of a
// large batch share a CTA, so that few rows do not leave most of its row
// groups idle at every sweep barrier.
int default_parts(const elsr_batch* b, int threads, int G);

// Instances per CTA: split the CTA's threads into P partitions for the runs
// whose rows fit P-th of the shared memory.  Reorders b->h_runs (stably:
// runs that need the whole CTA first, each class in its longest-first
// order) and sets ls->parts, n_whole, part_bytes and the launch's dynamic
// shared memory.  Leaves one team per CTA when packing does not apply.
void pack_runs(elsr_batch* b, LaunchShape* ls, int acc, int P) {
  const int nr = (int)b->h_runs.size();
  ls->parts = 1;
  ls->n_whole = nr;
  ls->part_bytes = 0;
  if (P <= 1 || ls->cluster != 1 || nr < 2 || ls->G > 32 || ls->maxt < 512 ||
      ls->threads % (32 * P) != 0 || ls->threads / P < ls->G)
    return;
  const uint32_t lim = ((uint32_t)kSmemLimit / (uint32_t)P) & ~15u;
  std::vector<RunDesc> whole, small;
  uint32_t need_whole = 0, need_part = 0;
  for (const RunDesc& r : b->h_runs) {
    const InstDesc& d = b->insts[r.inst];
    const uint32_t lay = vns_layout(d.K, d.T, acc, ls->ts).total;
    if (lay + kPartCtlBytes <= lim) {
      small.push_back(r);
      need_part = std::max(need_part, align16(lay + kPartCtlBytes));
    } else {
      whole.push_back(r);
      need_whole = std::max(need_whole, lay);
    }
  }
  if (small.size() < 2) return;
  b->h_runs = whole;
  b->h_runs.insert(b->h_runs.end(), small.begin(), small.end());
  ls->parts = P;
  ls->n_whole = (int)whole.size();
  ls->part_bytes = need_part;
  ls->smem = std::max<size_t>(need_whole, (size_t)P * need_part);
}

// Launch shape of the persistent kernel for the runs in b->h_runs: 64-bit
// words per bit row, table placement, sub-warp width, block size, CTAs per
// run (cluster) and grid size (resident blocks).
int vns_shape(elsr_batch* b, LaunchShape* ls) {
  const int acc = b->acc64 ? 8 : 4;
  int maxK = 0, maxT = 0;
  for (const RunDesc& r : b->h_runs) {
    maxK = std::max(maxK, b->insts[r.inst].K);
    maxT = std::max(maxT, b->insts[r.inst].T);
  }
  int C = b->cluster;
  // A single run spreads its rows over a cluster: 8 CTAs keep the most
  // speculative teams resident (15 on 152 SMs); beyond ~12 rows per CTA a
  // sweep's dependent chain grows with the rows each row group walks, and
  // 16 CTAs win (K=300: 26 vs 37 ms per 1000 iterations, measured).
  if (C <= 0)
    C = b->h_runs.size() == 1 ? (maxK > 96 ? 16 : std::min(8, std::max(1, maxK / 6))) : 1;
  C = std::min(C, maxK);
  size_t need_s = 0, need_g = 0;
  // Grow the cluster until the largest run's rows fit the CTAs' shared
  // memory.
  for (;;) {
    need_s = need_g = 0;
    for (const RunDesc& r : b->h_runs) {
      const InstDesc& d = b->insts[r.inst];
      const int kc = (d.K + C - 1) / C;
      need_s = std::max<size_t>(need_s, vns_layout(kc, d.T, acc, true).total);
      need_g = std::max<size_t>(need_g, vns_layout(kc, d.T, acc, false).total);
    }
    if (need_g <= (size_t)kSmemLimit || C >= 16 || C >= maxK) break;
    ++C;
  }
  ls->nw = maxT <= 64 ? 1 : 2;
  ls->ts = need_s <= (size_t)kSmemLimit;
  ls->smem = ls->ts ? need_s : need_g;
  if (ls->smem > (size_t)kSmemLimit) {
    b->err = "instance too large for the shared memory of its CTAs (" +
             std::to_string(ls->smem) + " bytes per CTA)";
    return ELSR_E_RANGE;
  }
  const bool single = b->h_runs.size() == 1;
  ls->G = b->lanes ? b->lanes : default_lanes(maxT, single);
  const int kc = (maxK + C - 1) / C;
  int thr = b->threads;
  // Default block: one CTA per SM; a single run keeps its CTAs small (its
  // rows are few and its sweeps latency-bound), many runs fill the SM with
  // 1024 threads (more warps to hide the decode's dependent latencies).
  if (!thr)
    thr = std::min(single ? (ls->G <= 32 ? 256 : 512) : 1024,
                   std::max(64, ((kc * ls->G + 31) / 32) * 32));
  if (ls->G > 32) {
    thr = std::max(thr, ls->G);
    thr -= thr % ls->G;
    thr = std::min(thr, 15 * ls->G);  // named barriers 1..15, one per row group
  }
  ls->threads = thr;
  ls->maxt = thr <= 256 ? 256 : (thr <= 512 ? 512 : 1024);
  ls->cluster = C;
  pack_runs(b, ls, acc, b->parts > 0 ? b->parts : default_parts(b, thr, ls->G));
  int active = 0;
  cudaError_t pe = vns_prepare(b->acc64, ls->nw, ls->ts, ls->maxt, ls->smem, thr, C, &active);
  if ((pe != cudaSuccess || active < 1) && !b->threads && thr > 256) {
    cudaGetLastError();  // retry with the smaller block bound
    thr = 256;
    ls->threads = thr;
    ls->maxt = 256;
    pe = vns_prepare(b->acc64, ls->nw, ls->ts, ls->maxt, ls->smem, thr, C, &active);
  }
  if (pe != cudaSuccess || active < 1) {
    b->err = std::string("launch shape rejected (") + cudaGetErrorString(pe) +
             "): threads " + std::to_string(thr) + ", cluster " + std::to_string(C) +
             ", shared bytes " + std::to_string(ls->smem) + ", tables in shared " +
             std::to_string((int)ls->ts) + ", words " + std::to_string(ls->nw);
    cudaGetLastError();
    return pe != cudaSuccess ? ELSR_E_CUDA : ELSR_E_RANGE;
  }
  ls->active = active;
  const int64_t nr = (int64_t)b->h_runs.size();
  if (C == 1)
    ls->blocks = (int)std::min<int64_t>((int64_t)active * b->sms, nr);
  else
    ls->blocks = C * (int)std::min<int64_t>(active, nr);
  return ELSR_OK;
}

// Room for `teams` speculative teams or fork-join workers: their result
// slots and published rows (two round parities each), the grid-barrier
// words and the speculative decision words.
int ensure_spec(elsr_batch* b, int teams) {
  if (teams <= (int)b->spec_cap) return ELSR_OK;
  dev_free(b->d_spec_slots, b->stream);
  dev_free(b->d_spec_rows, b->stream);
  dev_free(b->d_spec_bar, b->stream);
  dev_free(b->d_spec_dec, b->stream);
  b->spec_cap = 0;
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_spec_slots, (size_t)2 * teams, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_spec_rows, (size_t)2 * teams * kMaxShake, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_spec_bar, 2, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&b->d_spec_dec, 2, b->stream));
  b->spec_cap = teams;
  return ELSR_OK;
}

// Prefix tables of every row of every instance in device memory (the tables
// of launches whose rows do not fit shared memory), on b->stream.
static int stage_tables(elsr_batch* b) {
  if (!b->d_tab) {
    ELSR_TRY_CUDA(b, dev_alloc(&b->d_tab, (size_t)(b->cells + b->rows), b->stream));
    ELSR_TRY_CUDA(b, dev_alloc(&b->d_C0, (size_t)b->rows, b->stream));
  }
  StageParams sp;
  sp.ip = b->pools();
  sp.ninst = b->n;
  sp.gtab = b->d_tab;
  sp.gC0 = b->d_C0;
  ELSR_TRY_CUDA(b, launch_stage(sp, (int)std::min<int64_t>(b->rows, 1 << 30), b->stream));
  b->tab_ready = true;
  return ELSR_OK;
}

// Queue the runs of b->h_runs (already ordered) on b->stream.  fj_workers > 0
// runs the single run of b->h_runs as that many fork-join workers.
int launch_runs(elsr_batch* b, const RowBits* start_bits, bool with_traj,
                int64_t traj_entries, bool allow_spec = false, int fj_workers = 0) {
  LaunchShape ls;
  int rc = vns_shape(b, &ls);
  if (rc != ELSR_OK) return rc;
  const size_t nr = b->h_runs.size();
  int64_t bits_total = 0;
  for (const RunDesc& r : b->h_runs) bits_total = std::max<int64_t>(bits_total, r.bits_off + b->insts[r.inst].K);
  if ((rc = ensure(b, &b->d_runs, &b->runs_cap, nr)) != ELSR_OK) return rc;
  if ((rc = ensure(b, &b->d_out, &b->out_cap, nr)) != ELSR_OK) return rc;
  if ((rc = ensure(b, &b->d_bits, &b->bits_cap, (size_t)bits_total)) != ELSR_OK) return rc;
  if (with_traj && (rc = ensure(b, &b->d_traj, &b->traj_cap, (size_t)std::max<int64_t>(traj_entries, 1))) != ELSR_OK)
    return rc;
  if (!ls.ts && !b->tab_ready && (rc = stage_tables(b)) != ELSR_OK) return rc;
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(b->d_runs, b->h_runs.data(), nr * sizeof(RunDesc),
                                   cudaMemcpyHostToDevice, b->stream));
  ELSR_TRY_CUDA(b, cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(int32_t), b->stream));
  VnsParams p;
  p.ip = b->pools();
  p.runs = b->d_runs;
  p.nruns = (int32_t)nr;
  p.G = ls.G;
  p.vnd_cap = kVndCap;
  p.count_steps = b->count_steps;
  p.start_bits = start_bits;
  p.out_bits = b->d_bits;
  p.out = b->d_out;
  p.traj = with_traj ? b->d_traj : nullptr;
  p.queue = b->d_queue;
  p.spec_teams = 0;
  p.cluster = ls.cluster;
  p.spec_slots = nullptr;
  p.spec_rows = nullptr;
  p.spec_bar = nullptr;
  p.spec_dec = nullptr;
  p.fj_workers = 0;
  // several runs with automatic lanes: each run picks its own row groups
  p.adaptive_G = (nr > 1 && b->lanes == 0) ? 1 : 0;
  p.parts = ls.parts;
  p.n_whole = ls.n_whole;
  p.part_bytes = ls.part_bytes;
  p.pad2 = 0;
  b->last_parts = ls.parts;
  b->last_whole = ls.n_whole;
  if (fj_workers > 0) {
    const int resident = ls.cluster == 1 ? ls.active * b->sms : ls.active;
    if (nr != 1 || fj_workers > resident) {
      b->err = "fork-join workers (" + std::to_string(fj_workers) +
               ") exceed the teams that can be resident at once (" +
               std::to_string(resident) + " with " + std::to_string(ls.cluster) +
               " CTAs per worker)";
      return ELSR_E_RANGE;
    }
    if ((rc = ensure_spec(b, fj_workers)) != ELSR_OK) return rc;
    ELSR_TRY_CUDA(b, cudaMemsetAsync(b->d_spec_bar, 0, 2 * sizeof(int32_t), b->stream));
    p.fj_workers = fj_workers;
    p.spec_slots = b->d_spec_slots;
    p.spec_rows = b->d_spec_rows;
    p.spec_bar = b->d_spec_bar;
    ls.blocks = fj_workers * ls.cluster;
    ELSR_TRY_CUDA(b, vns_launch(b->acc64, ls.nw, ls.ts, ls.maxt, p, ls.blocks, ls.threads,
                                ls.smem, ls.cluster, b->stream));
    b->last_shape[7] = fj_workers;
    b->last_shape[0] = ls.G;
    b->last_shape[1] = ls.threads;
    b->last_shape[2] = ls.cluster;
    b->last_shape[3] = ls.blocks;
    b->last_shape[4] = (int)ls.smem;
    b->last_shape[5] = ls.ts;
    b->last_shape[6] = ls.nw;
    b->nruns = 1;
    b->have_result = true;
    return ELSR_OK;
  }
  // A single run may be spread over several teams that speculate on
  // consecutive iterations (exact: the committed trajectory is the
  // sequential one).
  int teams = 1;
  if (allow_spec && nr == 1 && b->h_runs[0].iters > 1 &&
      b->spec != 1) {
    const int resident = ls.cluster == 1 ? ls.active * b->sms : ls.active;
    const int want = b->spec > 1 ? b->spec : 16;
    teams = std::max(1, std::min({want, resident, b->h_runs[0].iters}));
  }
  cudaError_t le = cudaErrorUnknown;
  if (teams > 1) {
    if ((rc = ensure_spec(b, teams)) != ELSR_OK) return rc;
    ELSR_TRY_CUDA(b, cudaMemsetAsync(b->d_spec_bar, 0, 2 * sizeof(int32_t), b->stream));
    // decision words start with no round's tag; slot round tags start at -1
    ELSR_TRY_CUDA(b, cudaMemsetAsync(b->d_spec_dec, 0, 2 * sizeof(int32_t), b->stream));
    ELSR_TRY_CUDA(b, cudaMemsetAsync(b->d_spec_slots, 0xff, 2 * teams * sizeof(SpecSlot), b->stream));
    p.spec_teams = teams;
    p.spec_slots = b->d_spec_slots;
    p.spec_rows = b->d_spec_rows;
    p.spec_bar = b->d_spec_bar;
    p.spec_dec = b->d_spec_dec;
    const int blocks = teams * ls.cluster;
    le = vns_launch(b->acc64, ls.nw, ls.ts, ls.maxt, p, blocks, ls.threads, ls.smem, ls.cluster,
                    b->stream);
    if (le != cudaSuccess) {
      cudaGetLastError();  // the speculative launch was refused: run one team
      teams = 1;
    } else {
      ls.blocks = blocks;
    }
  }
  if (teams <= 1) {
    p.spec_teams = 0;
    ELSR_TRY_CUDA(b, vns_launch(b->acc64, ls.nw, ls.ts, ls.maxt, p, ls.blocks, ls.threads,
                                ls.smem, ls.cluster, b->stream));
  }
  b->last_shape[7] = teams;
  b->last_shape[0] = ls.G;
  b->last_shape[1] = ls.threads;
  b->last_shape[2] = ls.cluster;
  b->last_shape[3] = ls.blocks;
  b->last_shape[4] = (int)ls.smem;
  b->last_shape[5] = ls.ts;
  b->last_shape[6] = ls.nw;
  b->nruns = (int32_t)nr;
  b->have_result = true;
  return ELSR_OK;
}

void to_stats(const RunOut& o, elsr_stats_t* s) {
  s->best_cost = o.best_cost;
  s->traj_hash = o.traj_hash;
  s->moves_evaluated = o.moves_evaluated;
  s->evals = o.evals;
  s->vnd_cycles = o.vnd_cycles;
  s->applied = o.applied;
  s->iterations = o.iterations;
  s->accepted = o.accepted;
  s->segments = o.segments;
  s->status = o.status;
  s->reserved = 0;
}

void unpack_bits(const std::vector<RowBits>& rb, int K, int T, uint8_t* gM, uint8_t* gR) {
  for (int k = 0; k < K; ++k)
    for (int t = 0; t < T; ++t) {
      if (gM) gM[(int64_t)k * T + t] = (uint8_t)bit_of(rb[k].m0, rb[k].m1, t);
      if (gR) gR[(int64_t)k * T + t] = (uint8_t)bit_of(rb[k].r0, rb[k].r1, t);
    }
}

int pack_bits(const uint8_t* gM, const uint8_t* gR, int K, int T, std::vector<RowBits>& rb, std::string& err) {
  rb.assign(K, RowBits{0, 0, 0, 0});
  for (int k = 0; k < K; ++k)
    for (int t = 0; t < T; ++t) {
      const uint8_t m = gM[(int64_t)k * T + t], r = gR[(int64_t)k * T + t];
      if (m > 1 || r > 1) {
        err = "setup matrices must hold 0/1";
        return ELSR_E_ARG;
      }
      if (m) flip(rb[k].m0, rb[k].m1, t);
      if (r) flip(rb[k].r0, rb[k].r1, t);
    }
  return ELSR_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Single-instance handle
// ---------------------------------------------------------------------------
struct elsr_ctx {
  elsr_batch b;
  int32_t K = 0, T = 0;
  RowBits* d_state = nullptr;
  int64_t* d_rowcost = nullptr;
  // one device buffer for the evaluation's reduction words [4] and
  // per-product keys [K], mirrored by a pinned host buffer, so that an
  // evaluation needs one asynchronous copy each way
  uint64_t* d_evalbuf = nullptr;
  uint64_t* h_evalbuf = nullptr;  // pinned, [4 + K] results + [4] initial words
  uint64_t* d_ppkey = nullptr;    // d_evalbuf + 4
  uint64_t* d_scratch = nullptr;  // d_evalbuf
  // elsr_eval_neighbourhood as one CUDA graph per (mode, mask): reset of the
  // reduction words, the evaluation kernel and the copy of its results,
  // captured on a private stream and replayed on the handle's stream; made
  // again when the lanes per row change
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t eval_exec[2][8] = {};
  int32_t eval_exec_lanes = 0;
  int64_t* d_movecost = nullptr;
  int32_t* d_movewin = nullptr;
  int32_t* d_plan = nullptr;
  int64_t moves_total = 0;
  int last_kind = 0;  // 1: vns_run / forkjoin / resume, 2: multistart
  int32_t last_iters = 0;
  int32_t best_out = 0;
  bool counted = true;
  int64_t time_limit_ns = 0;  // wall-clock budget of the next runs (0: none)
  // the last single run (for checkpoints): its parameters and, for a resumed
  // run, the checkpoint it continued (iterations and counters before it)
  uint64_t run_seed = 0;
  int32_t run_kmax = 0, run_mode = 0, run_workers = 0;
  elsr_checkpoint_t base = {};

  ~elsr_ctx() {
    if (b.d_insts) cudaStreamSynchronize(b.stream);
    const cudaStream_t stream = b.stream;
    dev_free(d_state, stream);
    dev_free(d_rowcost, stream);
    dev_free(d_evalbuf, stream);
    if (h_evalbuf) cudaFreeHost(h_evalbuf);
    drop_eval_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    dev_free(d_movecost, stream);
    dev_free(d_movewin, stream);
    dev_free(d_plan, stream);
  }

  void drop_eval_graphs() {
    for (auto& row : eval_exec)
      for (auto& ex : row)
        if (ex) {
          cudaGraphExecDestroy(ex);
          ex = nullptr;
        }
  }
};

namespace {

// Launch geometry and parameters of one full-neighbourhood evaluation.
struct EvalPlan {
  EvalParams p;
  int blocks = 0;
  int threads = 128;
  size_t smem = 0;
  bool wide = false;  // one row per 128-thread CTA (eval_wide_kernel)
};

int eval_plan(elsr_ctx* h, uint32_t mask, int32_t mode, int single_j, bool write_rowcost,
              EvalPlan& pl) {
  elsr_batch* b = &h->b;
  // the evaluation kernel reduces within a warp: at most 32 lanes per row
  const int G = std::min(32, b->lanes ? b->lanes : default_lanes(h->T, true));
  const int nsub = pl.threads / G;
  pl.smem = eval_smem_bytes(nsub, h->T, b->acc64);
  ELSR_TRY_CUDA(b, eval_prepare(b->acc64, h->T, pl.smem));
  EvalParams& p = pl.p;
  p.ip = b->pools();
  p.K = h->K;
  p.T = h->T;
  p.bits = h->d_state;
  p.rowcost_in = h->d_rowcost;
  p.mask = mask;
  p.mode = mode;
  p.G = G;
  p.single_j = single_j;
  p.rowcost_out = write_rowcost ? h->d_rowcost : nullptr;
  p.pp_key = h->d_ppkey;
  p.move_cost = single_j ? h->d_movecost : nullptr;
  p.move_win = single_j ? h->d_movewin : nullptr;
  p.scratch = h->d_scratch;
  // Few rows: one row per CTA with 128 threads on its moves (the default
  // for a single run spreads a row over more than a warp); many rows: rows
  // of G lanes packed four to a CTA.
  pl.wide = G >= 32 && !b->lanes && (int64_t)h->K <= 2 * (int64_t)b->sms;
  pl.blocks = (h->K + nsub - 1) / nsub;
  return ELSR_OK;
}

// The evaluation's stream work: the reduction words {gkey, sum after,
// infeasible after, improving} set to {~0, 0, 0, 0} from the fixed pinned
// block after the results, then the kernel.
cudaError_t eval_issue(elsr_ctx* h, const EvalPlan& pl, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(h->d_scratch, h->h_evalbuf + 4 + h->K, 4 * sizeof(uint64_t),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return pl.wide ? launch_eval_wide(pl.p, h->b.acc64, pl.threads, s)
                 : launch_eval(pl.p, h->b.acc64, pl.blocks, pl.threads, pl.smem, s);
}

int eval_launch(elsr_ctx* h, uint32_t mask, int32_t mode, int single_j,
                bool write_rowcost) {
  EvalPlan pl;
  const int rc = eval_plan(h, mask, mode, single_j, write_rowcost, pl);
  if (rc != ELSR_OK) return rc;
  ELSR_TRY_CUDA(&h->b, eval_issue(h, pl, h->b.stream));
  return ELSR_OK;
}

// Graph of one elsr_eval_neighbourhood call (initial words, kernel, copy of
// the reduction words and per-product keys into the pinned buffer), made on
// first use of a (mode, mask) and kept until the lanes per row change.
int eval_graph(elsr_ctx* h, uint32_t mask, int32_t mode, cudaGraphExec_t* out) {
  elsr_batch* b = &h->b;
  if (h->eval_exec_lanes != b->lanes) {
    h->drop_eval_graphs();
    h->eval_exec_lanes = b->lanes;
  }
  cudaGraphExec_t& ex = h->eval_exec[mode][mask];
  if (!ex) {
    EvalPlan pl;
    const int rc = eval_plan(h, mask, mode, 0, false, pl);
    if (rc != ELSR_OK) return rc;
    if (!h->cap_stream)
      ELSR_TRY_CUDA(b, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    ELSR_TRY_CUDA(b, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = eval_issue(h, pl, h->cap_stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->h_evalbuf, h->d_evalbuf, ((size_t)h->K + 4) * sizeof(uint64_t),
                          cudaMemcpyDeviceToHost, h->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(h->cap_stream, &g);
    if (e == cudaSuccess) e = e_end;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ex = nullptr;
      b->err = std::string("evaluation graph: ") + cudaGetErrorString(e);
      return ELSR_E_CUDA;
    }
  }
  *out = ex;
  return ELSR_OK;
}

int refresh_rowcost(elsr_ctx* h) { return eval_launch(h, 0u, 0, 0, true); }

}  // namespace

extern "C" {

int elsr_version(void) { return 10300; }

int elsr_run_footprint(int32_t K, int32_t T, int32_t* smem_one_cta, int64_t* device_bytes) {
  if (K < 1 || T < 1 || T > ELSR_T_MAX) return ELSR_E_ARG;
  if (smem_one_cta) {
    const uint32_t with_tab = vns_layout(K, T, 4, true).total;
    const uint32_t without = vns_layout(K, T, 4, false).total;
    *smem_one_cta = (int32_t)(with_tab <= (uint32_t)kSmemLimit ? with_tab : without);
  }
  if (device_bytes) {
    // instance pools, prefix tables, descriptors, solution and statistics
    *device_bytes = (int64_t)K * T * 8 + (int64_t)K * (T + 1) * 8 + (int64_t)K * (16 + 8 + 32) +
                    (int64_t)(sizeof(InstDesc) + sizeof(RunDesc) + sizeof(RunOut));
  }
  return ELSR_OK;
}

const char* elsr_strerror(int code) {
  switch (code) {
    case ELSR_OK: return "ok";
    case ELSR_E_ARG: return "invalid argument";
    case ELSR_E_RANGE: return "instance exceeds the supported integer ranges";
    case ELSR_E_NOMEM: return "out of memory";
    case ELSR_E_CUDA: return "CUDA error";
    case ELSR_E_CAP: return "VND sweep cap reached";
    case ELSR_E_STATE: return "call out of order";
    case ELSR_E_TIMEOUT: return "a device-side wait exceeded its limit";
    case ELSR_E_BUSY: return "no room for the request now; retry after a completion";
    default: return "unknown error";
  }
}

const char* elsr_last_error(const elsr_t* h) {
  return h ? h->b.err.c_str() : g_create_error.c_str();
}

int elsr_create(elsr_t** out, int32_t K, int32_t T, const int32_t* D,
                const int32_t* R, const int32_t* kM, const int32_t* kR,
                const int32_t* hM, const int32_t* hR) {
  return elsr_create_ex(out, K, T, D, R, kM, kR, hM, hR, nullptr, nullptr);
}

int elsr_create_ex(elsr_t** out, int32_t K, int32_t T, const int32_t* D,
                   const int32_t* R, const int32_t* kM, const int32_t* kR,
                   const int32_t* hM, const int32_t* hR, const int32_t* pM,
                   const int32_t* pR) {
  if (!out) {
    g_create_error = "out is NULL";
    return ELSR_E_ARG;
  }
  *out = nullptr;
  elsr_ctx* h = new (std::nothrow) elsr_ctx();
  if (!h) {
    g_create_error = "host allocation failed";
    return ELSR_E_NOMEM;
  }
  const int32_t Ks[1] = {K}, Ts[1] = {T};
  int rc = batch_init(&h->b, 1, Ks, Ts, D, R, kM, kR, hM, hR, pM, pR);
  if (rc == ELSR_OK) {
    h->K = K;
    h->T = T;
    elsr_batch* b = &h->b;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dev_alloc(&h->d_state, K, b->stream);
    if (e == cudaSuccess) e = dev_alloc(&h->d_rowcost, K, b->stream);
    if (e == cudaSuccess) e = dev_alloc(&h->d_evalbuf, (size_t)K + 4, b->stream);
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_evalbuf, ((size_t)K + 8) * sizeof(uint64_t));
    if (e == cudaSuccess) {
      uint64_t* init = h->h_evalbuf + 4 + K;
      init[0] = ~0ull;
      init[1] = init[2] = init[3] = 0ull;
    }
    if (e == cudaSuccess) {
      h->d_scratch = h->d_evalbuf;
      h->d_ppkey = h->d_evalbuf + 4;
    }
    if (e == cudaSuccess) e = dev_alloc(&h->d_plan, (size_t)4 * K * T, b->stream);
    if (e != cudaSuccess) {
      b->err = std::string("device allocation: ") + cudaGetErrorString(e);
      rc = ELSR_E_NOMEM;
    } else {
      rc = elsr_set_state(h, nullptr, nullptr);
    }
  }
  if (rc != ELSR_OK) {
    g_create_error = h->b.err;
    delete h;
    return rc;
  }
  *out = h;
  return ELSR_OK;
}

void elsr_destroy(elsr_t* h) { delete h; }

int elsr_set_stream(elsr_t* h, void* stream) {
  if (!h) return ELSR_E_ARG;
  return elsr_batch_set_stream(&h->b, stream);
}

int elsr_set_launch(elsr_t* h, int32_t lanes, int32_t threads) {
  if (!h) return ELSR_E_ARG;
  return elsr_batch_set_launch(&h->b, lanes, threads);
}

int elsr_set_speculation(elsr_t* h, int32_t teams) {
  if (!h) return ELSR_E_ARG;
  if (teams < 0 || teams > 1024) {
    h->b.err = "teams must be 0 (automatic), 1 (off) or 2..1024";
    return ELSR_E_ARG;
  }
  h->b.spec = teams;
  return ELSR_OK;
}

int elsr_set_cluster(elsr_t* h, int32_t cluster) {
  if (!h) return ELSR_E_ARG;
  return elsr_batch_set_cluster(&h->b, cluster);
}

int elsr_launch_shape(elsr_t* h, int32_t* shape) {
  if (!h || !shape) return ELSR_E_ARG;
  return elsr_batch_launch_shape(&h->b, shape);
}

int elsr_set_state(elsr_t* h, const uint8_t* gM, const uint8_t* gR) {
  if (!h) return ELSR_E_ARG;
  if ((gM == nullptr) != (gR == nullptr)) {
    h->b.err = "gM and gR must both be given or both be NULL";
    return ELSR_E_ARG;
  }
  std::vector<uint8_t> ones;
  if (!gM) {
    ones.assign((size_t)h->K * h->T, 1);
    gM = gR = ones.data();
  }
  std::vector<RowBits> rb;
  int rc = pack_bits(gM, gR, h->K, h->T, rb, h->b.err);
  if (rc != ELSR_OK) return rc;
  ELSR_TRY_CUDA(&h->b, cudaMemcpyAsync(h->d_state, rb.data(), h->K * sizeof(RowBits),
                                       cudaMemcpyHostToDevice, h->b.stream));
  rc = refresh_rowcost(h);
  if (rc != ELSR_OK) return rc;
  ELSR_TRY_CUDA(&h->b, cudaStreamSynchronize(h->b.stream));
  return ELSR_OK;
}

int elsr_get_state(elsr_t* h, uint8_t* gM, uint8_t* gR) {
  if (!h || !gM || !gR) return ELSR_E_ARG;
  std::vector<RowBits> rb(h->K);
  ELSR_TRY_CUDA(&h->b, cudaMemcpyAsync(rb.data(), h->d_state, h->K * sizeof(RowBits),
                                       cudaMemcpyDeviceToHost, h->b.stream));
  ELSR_TRY_CUDA(&h->b, cudaStreamSynchronize(h->b.stream));
  unpack_bits(rb, h->K, h->T, gM, gR);
  return ELSR_OK;
}

int elsr_cost(elsr_t* h, int64_t* rowcost, int64_t* total) {
  if (!h) return ELSR_E_ARG;
  std::vector<int64_t> rc(h->K);
  ELSR_TRY_CUDA(&h->b, cudaMemcpyAsync(rc.data(), h->d_rowcost, h->K * sizeof(int64_t),
                                       cudaMemcpyDeviceToHost, h->b.stream));
  ELSR_TRY_CUDA(&h->b, cudaStreamSynchronize(h->b.stream));
  if (rowcost) memcpy(rowcost, rc.data(), h->K * sizeof(int64_t));
  if (total) {
    int64_t s = 0;
    for (int64_t c : rc) s = (c == INT64_MAX || s == INT64_MAX) ? INT64_MAX : s + c;
    *total = s;
  }
  return ELSR_OK;
}

int elsr_eval_neighbourhood(elsr_t* h, uint32_t nb_mask, int32_t mode,
                            int64_t* best_cost, int64_t* best_move,
                            int64_t* pp_cost, int64_t* pp_move) {
  if (!h) return ELSR_E_ARG;
  if ((nb_mask & ~7u) || (mode != ELSR_MODE_P && mode != ELSR_MODE_G)) {
    h->b.err = "nb_mask must be within 0..7 and mode P or G";
    return ELSR_E_ARG;
  }
  cudaGraphExec_t ex = nullptr;
  int rc = eval_graph(h, nb_mask, mode, &ex);
  if (rc != ELSR_OK) return rc;
  ELSR_TRY_CUDA(&h->b, cudaGraphLaunch(ex, h->b.stream));
  ELSR_TRY_CUDA(&h->b, cudaStreamSynchronize(h->b.stream));
  const uint64_t* sc = h->h_evalbuf;
  const uint64_t* keys = h->h_evalbuf + 4;
  for (int k = 0; k < h->K; ++k) {
    if (pp_cost) pp_cost[k] = keys[k] == ~0ull ? INT64_MAX : key_cost(keys[k]);
    if (pp_move) pp_move[k] = keys[k] == ~0ull ? -1 : key_index(keys[k]);
  }
  int64_t moves = 0;
  for (int j = 1; j <= 3; ++j)
    if (nb_mask & (1u << (j - 1))) moves += (int64_t)h->K * row_moves(h->T, j);
  h->moves_total += moves;
  if (mode == ELSR_MODE_P) {
    if (best_cost) *best_cost = sc[2] ? INT64_MAX : (int64_t)sc[1];
    if (best_move) *best_move = (int64_t)sc[3];
  } else {
    if (sc[0] == ~0ull) {
      int64_t tot = 0;
      rc = elsr_cost(h, nullptr, &tot);
      if (rc != ELSR_OK) return rc;
      if (best_cost) *best_cost = tot;
      if (best_move) *best_move = -1;
    } else {
      if (best_cost) *best_cost = key_cost(sc[0]);
      if (best_move) *best_move = key_index(sc[0]);
    }
  }
  return ELSR_OK;
}

int elsr_move_costs(elsr_t* h, int32_t nb, int64_t* costs, int32_t* window) {
  if (!h || nb < 1 || nb > 3 || !costs) return ELSR_E_ARG;
  const int64_t n = (int64_t)h->K * row_moves(h->T, nb);
  if (n <= 0) return ELSR_OK;
  elsr_batch* b = &h->b;
  dev_free(h->d_movecost, b->stream);
  dev_free(h->d_movewin, b->stream);
  ELSR_TRY_CUDA(b, dev_alloc(&h->d_movecost, n, b->stream));
  ELSR_TRY_CUDA(b, dev_alloc(&h->d_movewin, n, b->stream));
  int rc = eval_launch(h, 1u << (nb - 1), ELSR_MODE_P, nb, false);
  if (rc != ELSR_OK) return rc;
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(costs, h->d_movecost, n * sizeof(int64_t), cudaMemcpyDeviceToHost, b->stream));
  if (window)
    ELSR_TRY_CUDA(b, cudaMemcpyAsync(window, h->d_movewin, n * sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream));
  ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  h->moves_total += n;
  return ELSR_OK;
}

int elsr_set_time_limit(elsr_t* h, int64_t time_limit_us) {
  if (!h) return ELSR_E_ARG;
  if (time_limit_us < 0 || time_limit_us > (int64_t)1e12) {
    h->b.err = "time_limit_us must be 0 (none) or a positive budget below 10^12";
    return ELSR_E_ARG;
  }
  h->time_limit_ns = time_limit_us * 1000;
  return ELSR_OK;
}

namespace {

// Bookkeeping of a queued single run for elsr_result / elsr_checkpoint.
void note_single_run(elsr_t* h, const RunDesc& r, int32_t workers, const elsr_checkpoint_t* from) {
  h->last_kind = 1;
  h->last_iters = r.iters;
  h->best_out = 0;
  h->counted = false;
  h->run_seed = r.seed;
  h->run_kmax = r.kmax;
  h->run_mode = r.mode;
  h->run_workers = workers;
  if (from) {
    h->base = *from;
  } else {
    h->base = elsr_checkpoint_t{};
  }
}

RunDesc single_run(uint64_t seed, int32_t iters, int32_t kmax, int32_t mode) {
  RunDesc r;
  r.inst = 0;
  r.iters = iters;
  r.kmax = kmax;
  r.mode = mode;
  r.seed = seed;
  r.out = 0;
  r.tag = 0;
  r.bits_off = 0;
  r.start_off = 0;
  r.traj_off = 0;
  return r;
}

}  // namespace

int elsr_vns_run(elsr_t* h, uint64_t seed, int32_t iters, int32_t kmax, int32_t mode) {
  if (!h) return ELSR_E_ARG;
  if (iters < 0 || kmax < 1 || kmax > 3 || (mode != ELSR_MODE_P && mode != ELSR_MODE_G)) {
    h->b.err = "need iters >= 0, 1 <= kmax <= 3, mode P or G";
    return ELSR_E_ARG;
  }
  elsr_batch* b = &h->b;
  RunDesc r = single_run(seed, iters, kmax, mode);
  r.time_limit_ns = h->time_limit_ns;
  b->h_runs.assign(1, r);
  // a budgeted run is one team: speculative rounds cannot stop mid-way
  int rc = launch_runs(b, h->d_state, true, iters, h->time_limit_ns == 0);
  if (rc != ELSR_OK) return rc;
  note_single_run(h, r, 0, nullptr);
  return ELSR_OK;
}

int elsr_vns_forkjoin_run(elsr_t* h, uint64_t seed, int32_t iters, int32_t kmax,
                          int32_t mode, int32_t workers) {
  if (!h) return ELSR_E_ARG;
  if (iters < 0 || kmax < 1 || kmax > 3 || (mode != ELSR_MODE_P && mode != ELSR_MODE_G) ||
      workers < 1 || workers > ELSR_FJ_WORKERS_MAX) {
    h->b.err = "need iters >= 0, 1 <= kmax <= 3, mode P or G, 1 <= workers <= " +
               std::to_string(ELSR_FJ_WORKERS_MAX);
    return ELSR_E_ARG;
  }
  elsr_batch* b = &h->b;
  RunDesc r = single_run(seed, iters, kmax, mode);
  r.time_limit_ns = h->time_limit_ns;
  b->h_runs.assign(1, r);
  int rc = launch_runs(b, h->d_state, true, iters, false, workers);
  if (rc != ELSR_OK) return rc;
  note_single_run(h, r, workers, nullptr);
  return ELSR_OK;
}

int elsr_checkpoint(elsr_t* h, elsr_checkpoint_t* ck, uint8_t* gM, uint8_t* gR) {
  if (!h || !ck || ((gM == nullptr) != (gR == nullptr))) return ELSR_E_ARG;
  elsr_batch* b = &h->b;
  if (h->last_kind != 1) {
    b->err = "no single GVNS run (elsr_vns_run, elsr_vns_forkjoin_run, elsr_vns_resume) to checkpoint";
    return ELSR_E_STATE;
  }
  ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  RunOut o;
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(&o, b->d_out, sizeof(RunOut), cudaMemcpyDeviceToHost,
                                   b->stream));
  ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  elsr_checkpoint_t c = h->base;
  c.seed = h->run_seed;
  c.kmax = h->run_kmax;
  c.mode = h->run_mode;
  c.workers = h->run_workers;
  c.next_it = h->base.next_it + (int32_t)o.iterations;
  c.k = o.k_next;
  c.status = o.status;
  c.cost = o.best_cost;
  c.traj_hash = o.traj_hash;
  c.moves_evaluated += o.moves_evaluated;
  c.evals += o.evals;
  c.vnd_cycles += o.vnd_cycles;
  c.applied += o.applied;
  c.accepted += o.accepted;
  c.segments += o.segments;
  *ck = c;
  if (gM) {
    std::vector<RowBits> rb(h->K);
    ELSR_TRY_CUDA(b, cudaMemcpyAsync(rb.data(), b->d_bits, h->K * sizeof(RowBits),
                                     cudaMemcpyDeviceToHost, b->stream));
    ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
    unpack_bits(rb, h->K, h->T, gM, gR);
  }
  return o.status;
}

int elsr_vns_resume(elsr_t* h, const elsr_checkpoint_t* ck, const uint8_t* gM,
                    const uint8_t* gR, int32_t iters) {
  if (!h || !ck || !gM || !gR) return ELSR_E_ARG;
  elsr_batch* b = &h->b;
  if (iters < 0 || ck->kmax < 1 || ck->kmax > 3 ||
      (ck->mode != ELSR_MODE_P && ck->mode != ELSR_MODE_G) || ck->workers < 0 ||
      ck->workers > ELSR_FJ_WORKERS_MAX || ck->next_it < 0 || ck->k < 1 || ck->k > ck->kmax ||
      (int64_t)ck->next_it + iters > INT32_MAX || ck->status != ELSR_OK) {
    b->err = "invalid checkpoint (kmax, mode, workers, next_it, k or status) or iters";
    return ELSR_E_ARG;
  }
  int rc = elsr_set_state(h, gM, gR);  // x becomes the handle's current solution
  if (rc != ELSR_OK) return rc;
  RunDesc r = single_run(ck->seed, iters, ck->kmax, ck->mode);
  r.it0 = ck->next_it;
  r.k0 = ck->k;
  r.h0 = ck->traj_hash;
  r.f0 = ck->cost;
  r.resume = 1;
  r.time_limit_ns = h->time_limit_ns;
  b->h_runs.assign(1, r);
  rc = launch_runs(b, h->d_state, true, iters, h->time_limit_ns == 0 && ck->workers == 0,
                   ck->workers);
  if (rc != ELSR_OK) return rc;
  note_single_run(h, r, ck->workers, ck);
  return ELSR_OK;
}

int elsr_result(elsr_t* h, elsr_stats_t* stats, uint8_t* gM, uint8_t* gR,
                int32_t* plan, elsr_traj_t* traj, int32_t traj_capacity) {
  if (!h) return ELSR_E_ARG;
  elsr_batch* b = &h->b;
  if (!h->last_kind) {
    b->err = "no run has been queued";
    return ELSR_E_STATE;
  }
  ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  ELSR_TRY_CUDA(b, cudaGetLastError());
  RunOut o;
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(&o, b->d_out + h->best_out, sizeof(RunOut), cudaMemcpyDeviceToHost,
                                   b->stream));
  ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  if (!h->counted) {
    h->moves_total += o.moves_evaluated;
    h->counted = true;
  }
  if (stats) {
    to_stats(o, stats);
    if (h->last_kind == 1) {  // a resumed run reports totals since its first iteration
      stats->moves_evaluated += h->base.moves_evaluated;
      stats->evals += h->base.evals;
      stats->vnd_cycles += h->base.vnd_cycles;
      stats->applied += h->base.applied;
      stats->iterations += h->base.next_it;
      stats->accepted += h->base.accepted;
      stats->segments += h->base.segments;
    }
  }
  const RowBits* sol = b->d_bits + (int64_t)h->best_out * h->K;
  if (gM || gR) {
    std::vector<RowBits> rb(h->K);
    ELSR_TRY_CUDA(b, cudaMemcpyAsync(rb.data(), sol, h->K * sizeof(RowBits), cudaMemcpyDeviceToHost,
                                     b->stream));
    ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
    unpack_bits(rb, h->K, h->T, gM, gR);
  }
  if (plan) {
    PlanParams pp;
    pp.ip = b->pools();
    pp.inst = 0;
    pp.bits = sol;
    pp.plan = h->d_plan;
    ELSR_TRY_CUDA(b, launch_plan(pp, h->K, b->stream));
    ELSR_TRY_CUDA(b, cudaMemcpyAsync(plan, h->d_plan, (size_t)4 * h->K * h->T * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, b->stream));
    ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  }
  if (traj && traj_capacity > 0 && h->last_kind == 1) {
    const int32_t n = std::min(traj_capacity, h->last_iters);
    if (n > 0)
      ELSR_TRY_CUDA(b, cudaMemcpyAsync(traj, b->d_traj, n * sizeof(TrajEntry), cudaMemcpyDeviceToHost,
                                       b->stream));
    ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  }
  return o.status;
}

int elsr_multistart_run(elsr_t* h, uint64_t seed0, int32_t nstarts, int32_t iters,
                        int32_t kmax, int32_t mode, int64_t* best_cost,
                        int32_t* best_start, int64_t* costs) {
  if (!h) return ELSR_E_ARG;
  if (nstarts < 1 || nstarts >= (1 << 24) || iters < 0 || kmax < 1 || kmax > 3 ||
      (mode != ELSR_MODE_P && mode != ELSR_MODE_G)) {
    h->b.err = "need 1 <= nstarts < 2^24, iters >= 0, 1 <= kmax <= 3, mode P or G";
    return ELSR_E_ARG;
  }
  elsr_batch* b = &h->b;
  b->h_runs.assign(nstarts, RunDesc{});  // fresh descriptors: no resume, no budget
  for (int32_t s = 0; s < nstarts; ++s) {
    RunDesc& r = b->h_runs[s];
    r.inst = 0;
    r.iters = iters;
    r.kmax = kmax;
    r.mode = mode;
    r.seed = seed0 + (uint64_t)s;
    r.out = s;
    r.tag = 0;
    r.bits_off = (int64_t)s * h->K;
    r.start_off = 0;
    r.traj_off = -1;
  }
  int rc = launch_runs(b, h->d_state, false, 0);
  if (rc != ELSR_OK) return rc;
  BestofParams bp;
  bp.out = b->d_out;
  bp.n = nstarts;
  bp.best_key = b->d_bestkey;
  ELSR_TRY_CUDA(b, launch_bestof(bp, b->stream));
  uint64_t key = 0;
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(&key, b->d_bestkey, sizeof(key), cudaMemcpyDeviceToHost, b->stream));
  std::vector<RunOut> outs;
  if (costs) {
    outs.resize(nstarts);
    ELSR_TRY_CUDA(b, cudaMemcpyAsync(outs.data(), b->d_out, nstarts * sizeof(RunOut),
                                     cudaMemcpyDeviceToHost, b->stream));
  }
  ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  if (costs)
    for (int32_t s = 0; s < nstarts; ++s) costs[s] = outs[s].best_cost;
  h->last_kind = 2;
  h->last_iters = iters;
  h->best_out = key_index(key);
  if (best_cost) *best_cost = key_cost(key);
  if (best_start) *best_start = h->best_out;
  h->counted = true;
  return ELSR_OK;
}

int elsr_multistart_stats(elsr_t* h, elsr_stats_t* stats, int32_t n) {
  if (!h || !stats || n < 0) return ELSR_E_ARG;
  elsr_batch* b = &h->b;
  if (h->last_kind != 2) {
    b->err = "no multi-start run has been queued";
    return ELSR_E_STATE;
  }
  const int32_t m = std::min(n, b->nruns);
  std::vector<RunOut> outs(m > 0 ? m : 1);
  if (m > 0) {
    ELSR_TRY_CUDA(b, cudaMemcpyAsync(outs.data(), b->d_out, m * sizeof(RunOut),
                                     cudaMemcpyDeviceToHost, b->stream));
    ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  }
  for (int32_t i = 0; i < m; ++i) to_stats(outs[i], &stats[i]);
  return ELSR_OK;
}

int elsr_counters(elsr_t* h, int64_t* moves) {
  if (!h || !moves) return ELSR_E_ARG;
  *moves = h->moves_total;
  return ELSR_OK;
}

// ---------------------------------------------------------------------------
// Batch ABI
// ---------------------------------------------------------------------------
int elsr_batch_create(elsr_batch_t** out, int32_t n, const int32_t* Ks,
                      const int32_t* Ts, const int32_t* D, const int32_t* R,
                      const int32_t* kM, const int32_t* kR, const int32_t* hM,
                      const int32_t* hR) {
  return elsr_batch_create_on(out, n, Ks, Ts, D, R, kM, kR, hM, hR, nullptr);
}

int elsr_batch_create_on(elsr_batch_t** out, int32_t n, const int32_t* Ks,
                         const int32_t* Ts, const int32_t* D, const int32_t* R,
                         const int32_t* kM, const int32_t* kR, const int32_t* hM,
                         const int32_t* hR, void* stream) {
  return elsr_batch_create_ex(out, n, Ks, Ts, D, R, kM, kR, hM, hR, nullptr, nullptr, stream);
}

int elsr_batch_create_ex(elsr_batch_t** out, int32_t n, const int32_t* Ks,
                         const int32_t* Ts, const int32_t* D, const int32_t* R,
                         const int32_t* kM, const int32_t* kR, const int32_t* hM,
                         const int32_t* hR, const int32_t* pM, const int32_t* pR,
                         void* stream) {
  if (!out) {
    g_create_error = "out is NULL";
    return ELSR_E_ARG;
  }
  *out = nullptr;
  elsr_batch* b = new (std::nothrow) elsr_batch();
  if (!b) {
    g_create_error = "host allocation failed";
    return ELSR_E_NOMEM;
  }
  b->stream = (cudaStream_t)stream;
  int rc = batch_init(b, n, Ks, Ts, D, R, kM, kR, hM, hR, pM, pR);
  if (rc != ELSR_OK) {
    g_create_error = b->err;
    delete b;
    return rc;
  }
  *out = b;
  return ELSR_OK;
}

void elsr_batch_destroy(elsr_batch_t* b) { delete b; }

const char* elsr_batch_last_error(const elsr_batch_t* b) {
  return b ? b->err.c_str() : g_create_error.c_str();
}

int elsr_batch_set_stream(elsr_batch_t* b, void* stream) {
  if (!b) return ELSR_E_ARG;
  const cudaStream_t to = (cudaStream_t)stream;
  if (to != b->stream) {
    // work issued later on the new stream runs after everything issued so
    // far on the old one (a run still in flight writes the same buffers)
    cudaEvent_t ev = nullptr;
    ELSR_TRY_CUDA(b, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
    cudaEventDestroy(ev);  // released once the recorded work completes
    ELSR_TRY_CUDA(b, e);
    b->stream = to;
  }
  return ELSR_OK;
}

int elsr_batch_set_launch(elsr_batch_t* b, int32_t lanes, int32_t threads) {
  if (!b) return ELSR_E_ARG;
  if (lanes && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32 && lanes != 64 &&
      lanes != 128) {
    b->err = "lanes_per_row must be 4, 8, 16, 32, 64 or 128";
    return ELSR_E_ARG;
  }
  if (threads && (threads % 32 || threads < 32 || threads > 1024)) {
    b->err = "threads must be a multiple of 32 in [32, 1024]";
    return ELSR_E_ARG;
  }
  b->lanes = lanes;
  b->threads = threads;
  return ELSR_OK;
}

int elsr_batch_set_cluster(elsr_batch_t* b, int32_t cluster) {
  if (!b) return ELSR_E_ARG;
  if (cluster < 0 || cluster > 16) {
    b->err = "cluster must be 0 (automatic) or 1..16 CTAs";
    return ELSR_E_ARG;
  }
  b->cluster = cluster;
  return ELSR_OK;
}

int elsr_batch_set_count_steps(elsr_batch_t* b, int32_t on) {
  if (!b || (on != 0 && on != 1)) return ELSR_E_ARG;
  b->count_steps = on;
  return ELSR_OK;
}

int elsr_set_count_steps(elsr_t* h, int32_t on) {
  if (!h) return ELSR_E_ARG;
  return elsr_batch_set_count_steps(&h->b, on);
}

int elsr_batch_set_runs_per_cta(elsr_batch_t* b, int32_t runs_per_cta) {
  if (!b) return ELSR_E_ARG;
  if (runs_per_cta < 0 || runs_per_cta > kMaxParts ||
      (runs_per_cta & (runs_per_cta - 1)) != 0) {
    b->err = "runs per CTA must be 0 (automatic) or a power of two up to " +
             std::to_string(kMaxParts);
    return ELSR_E_ARG;
  }
  b->parts = runs_per_cta;
  return ELSR_OK;
}

int elsr_batch_packing(const elsr_batch_t* b, int32_t* runs_per_cta, int32_t* whole_cta_runs) {
  if (!b || !runs_per_cta || !whole_cta_runs) return ELSR_E_ARG;
  *runs_per_cta = b->last_parts;
  *whole_cta_runs = b->last_whole;
  return ELSR_OK;
}

int elsr_batch_launch_shape(elsr_batch_t* b, int32_t* shape) {
  if (!b || !shape) return ELSR_E_ARG;
  for (int i = 0; i < 8; ++i) shape[i] = b->last_shape[i];
  return ELSR_OK;
}

int elsr_batch_stage_tables(elsr_batch_t* b) {
  if (!b) return ELSR_E_ARG;
  return stage_tables(b);
}

int elsr_batch_run(elsr_batch_t* b, const uint64_t* seeds, int32_t iters, int32_t kmax,
                   int32_t mode) {
  if (!b || !seeds) return ELSR_E_ARG;
  if (iters < 0 || kmax < 1 || kmax > 3 || (mode != ELSR_MODE_P && mode != ELSR_MODE_G)) {
    b->err = "need iters >= 0, 1 <= kmax <= 3, mode P or G";
    return ELSR_E_ARG;
  }
  // Longest-first order of the work queue (cost ~ K*T per sweep).
  std::vector<int32_t> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) {
    return (int64_t)b->insts[a].K * b->insts[a].T > (int64_t)b->insts[c].K * b->insts[c].T;
  });
  b->h_runs.assign(b->n, RunDesc{});  // fresh descriptors: no resume, no budget
  b->out_of_inst.assign(b->n, 0);
  for (int32_t q = 0; q < b->n; ++q) {
    const int32_t i = order[q];
    RunDesc& r = b->h_runs[q];
    r.inst = i;
    r.iters = iters;
    r.kmax = kmax;
    r.mode = mode;
    r.seed = seeds[i];
    r.out = i;
    r.tag = 0;
    r.bits_off = b->insts[i].row_off;
    r.start_off = -1;
    r.traj_off = -1;
    b->out_of_inst[i] = i;
  }
  return launch_runs(b, nullptr, false, 0);
}

int elsr_batch_results(elsr_batch_t* b, elsr_stats_t* stats) {
  if (!b) return ELSR_E_ARG;
  if (!b->have_result) {
    b->err = "no batch run has been queued";
    return ELSR_E_STATE;
  }
  std::vector<RunOut> outs(b->n);
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(outs.data(), b->d_out, b->n * sizeof(RunOut),
                                   cudaMemcpyDeviceToHost, b->stream));
  ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  int status = ELSR_OK;
  for (int32_t i = 0; i < b->n; ++i) {
    if (stats) to_stats(outs[i], &stats[i]);
    if (outs[i].status != ELSR_OK) status = outs[i].status;
  }
  return status;
}

int elsr_batch_solution(elsr_batch_t* b, int32_t i, uint8_t* gM, uint8_t* gR) {
  if (!b || i < 0 || i >= b->n || !gM || !gR) return ELSR_E_ARG;
  if (!b->have_result) {
    b->err = "no batch run has been queued";
    return ELSR_E_STATE;
  }
  const InstDesc& d = b->insts[i];
  std::vector<RowBits> rb(d.K);
  ELSR_TRY_CUDA(b, cudaMemcpyAsync(rb.data(), b->d_bits + d.row_off, d.K * sizeof(RowBits),
                                   cudaMemcpyDeviceToHost, b->stream));
  ELSR_TRY_CUDA(b, cudaStreamSynchronize(b->stream));
  unpack_bits(rb, d.K, d.T, gM, gR);
  return ELSR_OK;
}

}  // extern "C"
