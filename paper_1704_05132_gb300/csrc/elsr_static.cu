// elsr_static.cu -- allocation-free variant of the neighbourhood evaluation
// (elsr_eval_neighbourhood_static in include/elsr.h).
//
// Some callers cannot allocate device memory: a framework that owns every
// byte of device memory through its own pool and forbids libraries from
// calling cudaMalloc, a serving loop that must never hit cudaMalloc /
// cudaFree (they can synchronise the whole device), or code that records
// its work while the allocator is unavailable.  This entry point takes its
// inputs and outputs as device pointers owned by the caller and keeps the
// evaluation's intermediate data in the fixed array below, so it never
// allocates.
//
// The array is a file-scope __device__ variable: every device that loads the
// library holds its ELSR_STATIC_BYTES until the process exits.  All calls on
// a device share it and it keeps the last call's contents (each call
// re-initialises what it needs), so calls that may overlap on the device --
// on different streams, or from several host threads -- race on it and must
// be serialised by the caller.
//
// Host code cannot use the array's name as a device address; it gets the
// address from cudaGetSymbolAddress once per device, on that device's first
// call (which should therefore come before any stream capture).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/elsr.h"
#include "elsr_internal.h"

namespace elsr {

namespace {

// Scratch layout (bytes): InstDesc | 4 reduction words | row costs [K] |
// per-product keys [K] | packed setup bits [K].
constexpr size_t kRedOff = 256;
constexpr size_t kCostOff = 512;
constexpr size_t kKeyOff = kCostOff + 8ull * ELSR_STATIC_K_MAX;
constexpr size_t kBitsOff = kKeyOff + 8ull * ELSR_STATIC_K_MAX;
constexpr size_t kScratchBytes = kBitsOff + 32ull * ELSR_STATIC_K_MAX;
static_assert(kScratchBytes == ELSR_STATIC_BYTES, "scratch size must match elsr.h");
static_assert(sizeof(InstDesc) <= kRedOff, "the instance descriptor overlaps the reduction words");
static_assert(kRedOff + 4 * sizeof(uint64_t) <= kCostOff, "reduction words overlap the row costs");
static_assert(sizeof(RowBits) == 32, "packed setup bits are 32 bytes per row");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_addr[64] = {nullptr};

// Pack the caller's 0/1 setup matrices into per-row bit words, describe the
// instance and reset the reduction words.
__global__ void static_pack_kernel(int K, int T, const uint8_t* __restrict__ gM,
                                   const uint8_t* __restrict__ gR, unsigned char* scratch) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    InstDesc d;
    d.K = K;
    d.T = T;
    d.cell_off = 0;
    d.row_off = 0;
    d.tab_off = 0;
    *(InstDesc*)scratch = d;
    uint64_t* red = (uint64_t*)(scratch + kRedOff);
    red[0] = ~0ull;
    red[1] = red[2] = red[3] = 0ull;
  }
  if (k >= K) return;
  RowBits b{0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    if (gM[(int64_t)k * T + t]) flip(b.m0, b.m1, t);
    if (gR[(int64_t)k * T + t]) flip(b.r0, b.r1, t);
  }
  ((RowBits*)(scratch + kBitsOff))[k] = b;
}

// Reset the reduction words between the row-cost pass and the evaluation.
__global__ void static_reset_kernel(unsigned char* scratch) {
  uint64_t* red = (uint64_t*)(scratch + kRedOff);
  red[0] = ~0ull;
  red[1] = red[2] = red[3] = 0ull;
}

// Turn the packed keys and reductions into the caller's outputs (one block).
__global__ void __launch_bounds__(1024) static_finish_kernel(
    int K, int mode, const unsigned char* scratch, int64_t* best, int64_t* pp_cost,
    int64_t* pp_move) {
  __shared__ unsigned long long sh_sum;
  __shared__ int sh_inf;
  const int64_t* rowcost = (const int64_t*)(scratch + kCostOff);
  const uint64_t* keys = (const uint64_t*)(scratch + kKeyOff);
  const uint64_t* red = (const uint64_t*)(scratch + kRedOff);
  if (threadIdx.x == 0) {
    sh_sum = 0ull;
    sh_inf = 0;
  }
  __syncthreads();
  unsigned long long s = 0;
  int ninf = 0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const uint64_t key = keys[k];
    if (pp_cost) pp_cost[k] = key == ~0ull ? INT64_MAX : key_cost(key);
    if (pp_move) pp_move[k] = key == ~0ull ? -1 : key_index(key);
    if (rowcost[k] == INT64_MAX) ++ninf; else s += (unsigned long long)rowcost[k];
  }
  if (s) atomicAdd(&sh_sum, s);
  if (ninf) atomicAdd(&sh_inf, ninf);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (mode == ELSR_MODE_P) {
      best[0] = red[2] ? INT64_MAX : (int64_t)red[1];
      best[1] = (int64_t)red[3];
    } else if (red[0] == ~0ull) {
      best[0] = sh_inf ? INT64_MAX : (int64_t)sh_sum;
      best[1] = -1;
    } else {
      best[0] = key_cost(red[0]);
      best[1] = key_index(red[0]);
    }
  }
}

// Device address of the scratch array for the current device (first call on
// a device looks it up).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = (unsigned char*)p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace elsr

using namespace elsr;

extern "C" int elsr_eval_neighbourhood_static(
    int32_t K, int32_t T, const int32_t* D, const int32_t* R, const int32_t* kM,
    const int32_t* kR, const int32_t* hM, const int32_t* hR, const uint8_t* gM,
    const uint8_t* gR, uint32_t nb_mask, int32_t mode, int64_t* best, int64_t* pp_cost,
    int64_t* pp_move, void* stream) {
  if (K < 1 || K > ELSR_STATIC_K_MAX || T < 1 || T > ELSR_T_MAX) return ELSR_E_RANGE;
  if (!D || !R || !kM || !kR || !hM || !hR || !gM || !gR || !best) return ELSR_E_ARG;
  if ((nb_mask & ~7u) || (mode != ELSR_MODE_P && mode != ELSR_MODE_G)) return ELSR_E_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  // An error an earlier call of the caller left pending is reported, and left
  // pending: the launch checks below would otherwise clear it as their own.
  if (cudaPeekAtLastError() != cudaSuccess) return ELSR_E_CUDA;
  // The array's address is per device: the stream and the caller's buffers
  // must belong to the current device.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ELSR_E_CUDA;
  if (s) {
    int sdev = -1;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return ELSR_E_CUDA;
    if (sdev != dev) return ELSR_E_ARG;
  }
  const void* bufs[] = {D, R, kM, kR, hM, hR, gM, gR, best, pp_cost, pp_move};
  for (const void* b : bufs) {
    if (!b) continue;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, b) != cudaSuccess) return ELSR_E_CUDA;
    if (a.type == cudaMemoryTypeDevice && a.device != dev) return ELSR_E_ARG;
  }
  unsigned char* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return ELSR_E_CUDA;

  static_pack_kernel<<<(K + 127) / 128, 128, 0, s>>>(K, T, gM, gR, scratch);
  if (cudaGetLastError() != cudaSuccess) return ELSR_E_CUDA;

  const int G = T <= 8 ? 4 : (T <= 16 ? 8 : (T <= 40 ? 16 : 32));
  const int threads = 128, nsub = threads / G;
  const size_t smem = eval_smem_bytes(nsub, T, true);
  if (eval_prepare(true, T, smem) != cudaSuccess) return ELSR_E_CUDA;
  EvalParams p;
  p.ip.insts = (const InstDesc*)scratch;
  p.ip.D = D;
  p.ip.R = R;
  p.ip.kM = kM;
  p.ip.kR = kR;
  p.ip.hM = hM;
  p.ip.hR = hR;
  p.ip.gtab = nullptr;
  p.ip.gC0 = nullptr;
  p.ip.pM = nullptr;  // no unit production costs
  p.ip.pR = nullptr;
  p.K = K;
  p.T = T;
  p.bits = (const RowBits*)(scratch + kBitsOff);
  p.rowcost_in = (const int64_t*)(scratch + kCostOff);
  p.G = G;
  p.single_j = 0;
  p.move_cost = nullptr;
  p.move_win = nullptr;
  p.scratch = (uint64_t*)(scratch + kRedOff);
  const int blocks = (K + nsub - 1) / nsub;
  // pass 1: row costs of the current solution (the "other rows" of mode G)
  p.mask = 0u;
  p.mode = ELSR_MODE_P;
  p.rowcost_out = (int64_t*)(scratch + kCostOff);
  p.pp_key = nullptr;
  if (launch_eval(p, true, blocks, threads, smem, s) != cudaSuccess) return ELSR_E_CUDA;
  static_reset_kernel<<<1, 1, 0, s>>>(scratch);
  if (cudaGetLastError() != cudaSuccess) return ELSR_E_CUDA;
  // pass 2: the evaluation itself
  p.mask = nb_mask;
  p.mode = mode;
  p.rowcost_out = nullptr;
  p.pp_key = (uint64_t*)(scratch + kKeyOff);
  if (launch_eval(p, true, blocks, threads, smem, s) != cudaSuccess) return ELSR_E_CUDA;
  static_finish_kernel<<<1, 1024, 0, s>>>(K, mode, scratch, best, pp_cost, pp_move);
  if (cudaGetLastError() != cudaSuccess) return ELSR_E_CUDA;
  return ELSR_OK;
}
