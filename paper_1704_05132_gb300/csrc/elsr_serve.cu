// elsr_serve.cu -- serving runtime of include/elsr.h (elsr_server_*): GVNS
// requests are admitted as they arrive, join the kernels already running and
// retire one by one.
//
// Device side (srv_kernel in elsr_vns.cuh): requests are grouped in classes
// by the CTAs a team needs for the request's rows (1..16, a thread-block
// cluster) and the words of its setup-bit rows (1 or 2).  Each class has a
// queue of request slots in device memory.  A launch of a class runs one team
// per cluster; a team claims the next queued request, solves it and writes
// its statistics and solution into host-mapped memory, then its retire word,
// and claims again.  Nothing in the kernel waits for the host: a team whose
// claim finds the queue empty exits, and so does one that has served
// max_runs requests, which leaves its SMs to the launches of other classes.
//
// Host side (this file): admission by footprint -- a request needs one slot
// and K*T cells and K rows of the fixed-capacity device pools, found by
// first fit, else the call answers ELSR_E_BUSY and the caller retries after
// a completion.  Its instance is copied into pinned staging memory and from
// there into the pools on a copy stream, followed in stream order by its
// descriptors, its queue entry and the queue's new tail.  A class with
// requests not yet retired and no launch in flight is launched again (on its
// own stream, after the copies); polling reads the retire words, which are
// in host memory, without synchronising any stream.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "../../include/elsr.h"
#include "elsr_internal.h"

using namespace elsr;

namespace {

constexpr int kClasses = 32;  // CTAs per team 1..16 x words per bit row 1..2
constexpr int kDefaultSlots = 2048;
constexpr int64_t kDefaultCells = 8ll << 20;
constexpr int64_t kDefaultRows = 512ll << 10;
constexpr int kVndCapSrv = 1 << 20;

// First-fit allocator of ranges of [0, cap): the host's record of which pool
// space holds a request.
class RangeAlloc {
 public:
  void reset(int64_t cap) {
    free_.clear();
    if (cap > 0) free_[0] = cap;
  }
  int64_t alloc(int64_t n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const int64_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > n) free_[off + n] = len - n;
      return off;
    }
    return -1;
  }
  void release(int64_t off, int64_t n) {
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<int64_t, int64_t> free_;
};

struct Live {
  int64_t ticket = -1;  // -1: slot free
  bool reported = false;  // retired and reported, kept for its solution
  int cls = 0;
  int64_t cell_off = 0, row_off = 0;
  int32_t K = 0, T = 0;
};

template <typename T>
cudaError_t host_alloc(T** p, size_t n, unsigned flags) {
  *p = nullptr;
  return cudaHostAlloc((void**)p, (n ? n : 1) * sizeof(T), flags);
}

}  // namespace

struct elsr_server {
  int device = 0, sms = 0;
  int32_t cap = 0;
  int64_t cells_cap = 0, rows_cap = 0;
  bool acc64 = false;
  int threads = 1024, max_runs = 1, count_steps = 1, keep = 0;
  std::string err;

  cudaStream_t cstream = nullptr;
  cudaEvent_t staged = nullptr;
  cudaStream_t kstream[kClasses] = {};
  cudaEvent_t kdone[kClasses] = {};
  bool launched[kClasses] = {};
  int active[kClasses] = {};
  int64_t launches = 0;

  // device pools and queues
  InstDesc* d_insts = nullptr;
  RunDesc* d_runs = nullptr;
  int32_t *d_D = nullptr, *d_R = nullptr, *d_kM = nullptr, *d_kR = nullptr, *d_hM = nullptr,
          *d_hR = nullptr;
  int32_t* d_q = nullptr;    // [kClasses][cap]
  int32_t* d_ctr = nullptr;  // [kClasses][2]: head, tail
  // pinned staging (each request's data stays put until it retires)
  int32_t *h_D = nullptr, *h_R = nullptr, *h_kM = nullptr, *h_kR = nullptr, *h_hM = nullptr,
          *h_hR = nullptr;
  InstDesc* h_insts = nullptr;
  RunDesc* h_runs = nullptr;
  int32_t* h_qslot = nullptr;  // [cap] the queue entry a slot's request wrote
  int32_t* h_tail = nullptr;   // [cap] the tail its request published
  // host-mapped results (host and device views)
  RunOut *m_out = nullptr, *dm_out = nullptr;
  int32_t *m_done = nullptr, *dm_done = nullptr;
  RowBits *m_bits = nullptr, *dm_bits = nullptr;

  RangeAlloc cells, rows;
  std::vector<int32_t> free_slots;
  std::vector<Live> live;
  int32_t tail[kClasses] = {};
  int64_t unfinished[kClasses] = {};
  int64_t inflight = 0;
  int64_t next_ticket = 0;

  ~elsr_server() {
    for (int c = 0; c < kClasses; ++c)
      if (kstream[c]) cudaStreamSynchronize(kstream[c]);
    if (cstream) cudaStreamSynchronize(cstream);
    for (int c = 0; c < kClasses; ++c) {
      if (kdone[c]) cudaEventDestroy(kdone[c]);
      if (kstream[c]) cudaStreamDestroy(kstream[c]);
    }
    if (staged) cudaEventDestroy(staged);
    void* dev[] = {d_insts, d_runs, d_D, d_R, d_kM, d_kR, d_hM, d_hR, d_q, d_ctr};
    for (void* p : dev)
      if (p) cudaFree(p);
    void* host[] = {h_D, h_R, h_kM, h_kR, h_hM, h_hR, h_insts, h_runs, h_qslot, h_tail,
                    m_out, m_done, m_bits};
    for (void* p : host)
      if (p) cudaFreeHost(p);
    if (cstream) cudaStreamDestroy(cstream);
  }
};

namespace {

#define SRV_TRY(s, call)                                                       \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      (s)->err = std::string(#call) + ": " + cudaGetErrorString(e_);           \
      return e_ == cudaErrorMemoryAllocation ? ELSR_E_NOMEM : ELSR_E_CUDA;     \
    }                                                                          \
  } while (0)

// CTAs per team and class of a request of K rows and T periods (prefix tables
// in shared memory, one CTA per SM); -1 when even 16 CTAs are too few.
int request_class(const elsr_server* s, int32_t K, int32_t T, int* C_out, int* nw_out) {
  const int acc = s->acc64 ? 8 : 4;
  for (int C = 1; C <= 16 && C <= K; ++C) {
    const int kc = (K + C - 1) / C;
    if (vns_layout(kc, T, acc, true).total <= (uint32_t)kSmemLimit) {
      *C_out = C;
      *nw_out = T <= 64 ? 1 : 2;
      return (C - 1) * 2 + (*nw_out - 1);
    }
  }
  return -1;
}

// Launch class c again when it has requests not yet retired and no launch in
// flight.  One team per resident cluster, at most one per unfinished request.
int maybe_launch(elsr_server* s, int c) {
  if (s->unfinished[c] == 0) return ELSR_OK;
  if (s->launched[c]) {
    const cudaError_t q = cudaEventQuery(s->kdone[c]);
    if (q == cudaErrorNotReady) return ELSR_OK;
    if (q != cudaSuccess) SRV_TRY(s, q);
  }
  const int C = c / 2 + 1, nw = c % 2 + 1;
  if (!s->kstream[c]) {
    SRV_TRY(s, cudaStreamCreateWithFlags(&s->kstream[c], cudaStreamNonBlocking));
    SRV_TRY(s, cudaEventCreateWithFlags(&s->kdone[c], cudaEventDisableTiming));
  }
  if (!s->active[c]) {
    int a = 0;
    SRV_TRY(s, srv_prepare(s->acc64, nw, (size_t)kSmemLimit, s->threads, C, &a));
    if (a < 1) {
      s->err = "serving launch of " + std::to_string(C) + " CTAs per team cannot be resident";
      return ELSR_E_RANGE;
    }
    s->active[c] = C == 1 ? a * s->sms : a;
  }
  const int teams = (int)std::min<int64_t>(s->unfinished[c], s->active[c]);
  VnsParams p = {};
  p.ip.insts = s->d_insts;
  p.ip.D = s->d_D;
  p.ip.R = s->d_R;
  p.ip.kM = s->d_kM;
  p.ip.kR = s->d_kR;
  p.ip.hM = s->d_hM;
  p.ip.hR = s->d_hR;
  p.runs = s->d_runs;
  p.nruns = s->cap;
  p.G = 16;
  p.vnd_cap = kVndCapSrv;
  p.count_steps = s->count_steps;
  p.out_bits = s->dm_bits;
  p.out = s->dm_out;
  p.cluster = C;
  p.parts = 1;
  SrvQueue q;
  q.slots = s->d_q + (int64_t)c * s->cap;
  q.head = s->d_ctr + 2 * c;
  q.tail = s->d_ctr + 2 * c + 1;
  q.done = s->dm_done;
  q.cap = s->cap;
  q.max_runs = s->max_runs;
  SRV_TRY(s, cudaStreamWaitEvent(s->kstream[c], s->staged, 0));
  SRV_TRY(s, srv_launch(s->acc64, nw, p, q, teams * C, s->threads, (size_t)kSmemLimit, C,
                        s->kstream[c]));
  SRV_TRY(s, cudaEventRecord(s->kdone[c], s->kstream[c]));
  s->launched[c] = true;
  ++s->launches;
  return ELSR_OK;
}

void release_slot(elsr_server* s, int32_t slot) {
  Live& L = s->live[slot];
  s->cells.release(L.cell_off, (int64_t)L.K * L.T);
  s->rows.release(L.row_off, L.K);
  --s->inflight;
  L.ticket = -1;
  L.reported = false;
  s->free_slots.push_back(slot);
}

}  // namespace

extern "C" {

int elsr_server_create(elsr_server_t** out, const elsr_server_config_t* cfg) {
  if (!out) return ELSR_E_ARG;
  *out = nullptr;
  elsr_server_config_t c = {};
  if (cfg) c = *cfg;
  if (c.slots < 0 || c.cells < 0 || c.rows < 0 || c.threads < 0 || c.max_runs < 0 ||
      (c.acc64 != 0 && c.acc64 != 1) || (c.count_steps != 0 && c.count_steps != 1) ||
      (c.keep_solutions != 0 && c.keep_solutions != 1))
    return ELSR_E_ARG;
  if (c.threads && (c.threads % 32 || c.threads > 1024)) return ELSR_E_ARG;
  elsr_server* s = new elsr_server();
  s->cap = c.slots ? c.slots : kDefaultSlots;
  s->cells_cap = c.cells ? c.cells : kDefaultCells;
  s->rows_cap = c.rows ? c.rows : kDefaultRows;
  s->threads = c.threads ? c.threads : 1024;
  s->max_runs = c.max_runs ? c.max_runs : 1;
  s->acc64 = c.acc64 == 1;
  s->count_steps = c.count_steps;
  s->keep = c.keep_solutions;
  int rc = ELSR_OK;
  auto fail = [&](int code) {
    rc = code;
    delete s;
    return code;
  };
#define SRV_INIT(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return fail(e_ == cudaErrorMemoryAllocation ? ELSR_E_NOMEM \
                                                                       : ELSR_E_CUDA); \
  } while (0)
  SRV_INIT(cudaGetDevice(&s->device));
  SRV_INIT(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device));
  SRV_INIT(cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking));
  SRV_INIT(cudaEventCreateWithFlags(&s->staged, cudaEventDisableTiming));
  const size_t cap = (size_t)s->cap, cells = (size_t)s->cells_cap, rows = (size_t)s->rows_cap;
  SRV_INIT(cudaMalloc((void**)&s->d_insts, cap * sizeof(InstDesc)));
  SRV_INIT(cudaMalloc((void**)&s->d_runs, cap * sizeof(RunDesc)));
  SRV_INIT(cudaMalloc((void**)&s->d_D, cells * 4));
  SRV_INIT(cudaMalloc((void**)&s->d_R, cells * 4));
  SRV_INIT(cudaMalloc((void**)&s->d_kM, rows * 4));
  SRV_INIT(cudaMalloc((void**)&s->d_kR, rows * 4));
  SRV_INIT(cudaMalloc((void**)&s->d_hM, rows * 4));
  SRV_INIT(cudaMalloc((void**)&s->d_hR, rows * 4));
  SRV_INIT(cudaMalloc((void**)&s->d_q, (size_t)kClasses * cap * 4));
  SRV_INIT(cudaMalloc((void**)&s->d_ctr, (size_t)kClasses * 2 * 4));
  SRV_INIT(cudaMemset(s->d_ctr, 0, (size_t)kClasses * 2 * 4));
  SRV_INIT(host_alloc(&s->h_D, cells, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->h_R, cells, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->h_kM, rows, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->h_kR, rows, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->h_hM, rows, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->h_hR, rows, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->h_insts, cap, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->h_runs, cap, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->h_qslot, cap, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->h_tail, cap, cudaHostAllocDefault));
  SRV_INIT(host_alloc(&s->m_out, cap, cudaHostAllocMapped));
  SRV_INIT(host_alloc(&s->m_done, cap, cudaHostAllocMapped));
  SRV_INIT(host_alloc(&s->m_bits, rows, cudaHostAllocMapped));
  SRV_INIT(cudaHostGetDevicePointer((void**)&s->dm_out, s->m_out, 0));
  SRV_INIT(cudaHostGetDevicePointer((void**)&s->dm_done, s->m_done, 0));
  SRV_INIT(cudaHostGetDevicePointer((void**)&s->dm_bits, s->m_bits, 0));
#undef SRV_INIT
  memset(s->m_done, 0, cap * sizeof(int32_t));
  s->cells.reset(s->cells_cap);
  s->rows.reset(s->rows_cap);
  s->live.assign(cap, Live{});
  s->free_slots.resize(cap);
  for (int32_t i = 0; i < s->cap; ++i) s->free_slots[i] = s->cap - 1 - i;
  (void)rc;
  *out = s;
  return ELSR_OK;
}

void elsr_server_destroy(elsr_server_t* s) { delete s; }

const char* elsr_server_last_error(const elsr_server_t* s) { return s ? s->err.c_str() : ""; }

int elsr_server_submit(elsr_server_t* s, int32_t K, int32_t T, const int32_t* D,
                       const int32_t* R, const int32_t* kM, const int32_t* kR,
                       const int32_t* hM, const int32_t* hR, uint64_t seed, int32_t iters,
                       int32_t kmax, int32_t mode, int64_t* ticket) {
  if (!s || !ticket) return ELSR_E_ARG;
  if (iters < 0 || kmax < 1 || kmax > 3 || (mode != ELSR_MODE_P && mode != ELSR_MODE_G)) {
    s->err = "need iters >= 0, 1 <= kmax <= 3, mode P or G";
    return ELSR_E_ARG;
  }
  bool a64 = false;
  int rc = validate_instance(K, T, D, R, kM, kR, hM, hR, &a64, s->err);
  if (rc != ELSR_OK) return rc;
  if (a64 && !s->acc64) {
    s->err = "instance needs 64-bit row accumulators; create the server with acc64 = 1";
    return ELSR_E_RANGE;
  }
  int C = 0, nw = 0;
  const int c = request_class(s, K, T, &C, &nw);
  if (c < 0) {
    s->err = "instance rows exceed the shared memory of 16 CTAs";
    return ELSR_E_RANGE;
  }
  const int64_t ncell = (int64_t)K * T;
  if (ncell > s->cells_cap || K > s->rows_cap) {
    s->err = "instance larger than the server's pools";
    return ELSR_E_RANGE;
  }
  if (s->free_slots.empty()) {
    s->err = "every request slot is in use";
    return ELSR_E_BUSY;
  }
  const int64_t cell = s->cells.alloc(ncell);
  if (cell < 0) {
    s->err = "no room in the demand/return pools";
    return ELSR_E_BUSY;
  }
  const int64_t row = s->rows.alloc(K);
  if (row < 0) {
    s->cells.release(cell, ncell);
    s->err = "no room in the per-product pools";
    return ELSR_E_BUSY;
  }
  const int32_t slot = s->free_slots.back();
  s->free_slots.pop_back();
  const int64_t tk = s->next_ticket++;

  memcpy(s->h_D + cell, D, ncell * 4);
  memcpy(s->h_R + cell, R, ncell * 4);
  memcpy(s->h_kM + row, kM, (size_t)K * 4);
  memcpy(s->h_kR + row, kR, (size_t)K * 4);
  memcpy(s->h_hM + row, hM, (size_t)K * 4);
  memcpy(s->h_hR + row, hR, (size_t)K * 4);
  InstDesc d;
  d.K = K;
  d.T = T;
  d.cell_off = cell;
  d.row_off = row;
  d.tab_off = 0;
  s->h_insts[slot] = d;
  RunDesc r{};
  r.inst = slot;
  r.iters = iters;
  r.kmax = kmax;
  r.mode = mode;
  r.seed = seed;
  r.out = slot;
  r.tag = (int32_t)(tk & 0x3fffffff);
  r.bits_off = row;
  r.start_off = -1;
  r.traj_off = -1;
  s->h_runs[slot] = r;
  const int32_t pos = s->tail[c];
  s->h_qslot[slot] = slot;
  s->h_tail[slot] = pos + 1;
  ((volatile int32_t*)s->m_done)[slot] = 0;

  cudaStream_t cs = s->cstream;
  SRV_TRY(s, cudaMemcpyAsync(s->d_D + cell, s->h_D + cell, ncell * 4, cudaMemcpyHostToDevice, cs));
  SRV_TRY(s, cudaMemcpyAsync(s->d_R + cell, s->h_R + cell, ncell * 4, cudaMemcpyHostToDevice, cs));
  SRV_TRY(s, cudaMemcpyAsync(s->d_kM + row, s->h_kM + row, (size_t)K * 4, cudaMemcpyHostToDevice, cs));
  SRV_TRY(s, cudaMemcpyAsync(s->d_kR + row, s->h_kR + row, (size_t)K * 4, cudaMemcpyHostToDevice, cs));
  SRV_TRY(s, cudaMemcpyAsync(s->d_hM + row, s->h_hM + row, (size_t)K * 4, cudaMemcpyHostToDevice, cs));
  SRV_TRY(s, cudaMemcpyAsync(s->d_hR + row, s->h_hR + row, (size_t)K * 4, cudaMemcpyHostToDevice, cs));
  SRV_TRY(s, cudaMemcpyAsync(s->d_insts + slot, s->h_insts + slot, sizeof(InstDesc),
                             cudaMemcpyHostToDevice, cs));
  SRV_TRY(s, cudaMemcpyAsync(s->d_runs + slot, s->h_runs + slot, sizeof(RunDesc),
                             cudaMemcpyHostToDevice, cs));
  SRV_TRY(s, cudaMemcpyAsync(s->d_q + (int64_t)c * s->cap + pos % s->cap, s->h_qslot + slot, 4,
                             cudaMemcpyHostToDevice, cs));
  // the new tail last: a team that sees it finds everything above in place
  SRV_TRY(s, cudaMemcpyAsync(s->d_ctr + 2 * c + 1, s->h_tail + slot, 4, cudaMemcpyHostToDevice, cs));
  SRV_TRY(s, cudaEventRecord(s->staged, cs));

  s->tail[c] = pos + 1;
  Live& L = s->live[slot];
  L.ticket = tk;
  L.cls = c;
  L.cell_off = cell;
  L.row_off = row;
  L.K = K;
  L.T = T;
  ++s->unfinished[c];
  ++s->inflight;
  *ticket = tk;
  return maybe_launch(s, c);
}

int elsr_server_poll(elsr_server_t* s, int32_t max, int64_t* tickets, elsr_stats_t* stats) {
  if (!s || max < 0 || (max > 0 && !tickets)) return ELSR_E_ARG;
  int32_t n = 0;
  const volatile int32_t* done = s->m_done;
  for (int32_t slot = 0; slot < s->cap && n < max; ++slot) {
    Live& L = s->live[slot];
    if (L.ticket < 0 || L.reported || done[slot] != (int32_t)(L.ticket & 0x3fffffff) + 1)
      continue;
    std::atomic_thread_fence(std::memory_order_acquire);
    tickets[n] = L.ticket;
    if (stats) {
      RunOut o;
      memcpy(&o, (const void*)(s->m_out + slot), sizeof(RunOut));
      elsr_stats_t& st = stats[n];
      st.best_cost = o.best_cost;
      st.traj_hash = o.traj_hash;
      st.moves_evaluated = o.moves_evaluated;
      st.evals = o.evals;
      st.vnd_cycles = o.vnd_cycles;
      st.applied = o.applied;
      st.iterations = o.iterations;
      st.accepted = o.accepted;
      st.segments = o.segments;
      st.status = o.status;
      st.reserved = 0;
    }
    ++n;
    --s->unfinished[L.cls];
    if (s->keep) {
      L.reported = true;  // freed by elsr_server_release
    } else {
      release_slot(s, slot);
    }
  }
  for (int c = kClasses - 1; c >= 0; --c) {  // the largest requests first
    const int rc = maybe_launch(s, c);
    if (rc != ELSR_OK) return rc;
  }
  return n;
}

int elsr_server_solution(elsr_server_t* s, int64_t ticket, uint8_t* gM, uint8_t* gR) {
  if (!s || !gM || !gR) return ELSR_E_ARG;
  for (int32_t slot = 0; slot < s->cap; ++slot) {
    const Live& L = s->live[slot];
    if (L.ticket != ticket) continue;
    if (s->m_done[slot] != (int32_t)(ticket & 0x3fffffff) + 1) {
      s->err = "request has not retired yet";
      return ELSR_E_STATE;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    for (int32_t k = 0; k < L.K; ++k) {
      RowBits b;
      memcpy(&b, (const void*)(s->m_bits + L.row_off + k), sizeof(RowBits));
      for (int32_t t = 0; t < L.T; ++t) {
        gM[(int64_t)k * L.T + t] = (uint8_t)bit_of(b.m0, b.m1, t);
        gR[(int64_t)k * L.T + t] = (uint8_t)bit_of(b.r0, b.r1, t);
      }
    }
    return ELSR_OK;
  }
  s->err = "no request with this ticket in flight";
  return ELSR_E_STATE;
}

int elsr_server_release(elsr_server_t* s, int64_t ticket) {
  if (!s) return ELSR_E_ARG;
  for (int32_t slot = 0; slot < s->cap; ++slot) {
    if (s->live[slot].ticket == ticket && s->live[slot].reported) {
      release_slot(s, slot);
      return ELSR_OK;
    }
  }
  s->err = "no reported request with this ticket is kept";
  return ELSR_E_STATE;
}

int elsr_server_info(const elsr_server_t* s, int64_t* inflight, int64_t* launches) {
  if (!s) return ELSR_E_ARG;
  if (inflight) *inflight = s->inflight;
  if (launches) *launches = s->launches;
  return ELSR_OK;
}

}  // extern "C"
