// elsr_kernels.cu -- sm_103a kernels of the ELSR VNS hot path other than the
// persistent GVNS kernel (elsr_vns.cuh):
//
//   stage_kernel  prefix tables of every instance row into global memory
//                 (warp-shuffle scans), for instances too large to stage in
//                 shared memory.
//   eval_kernel   one best-improvement evaluation of whole neighbourhoods of
//                 one instance (Algorithm 1's best-neighbour search for every
//                 product at once): stage rows in shared memory, build each
//                 row's cache, delta re-decode every candidate, sub-warp
//                 argmin per product, global argmin for mode G.
//   bestof_kernel lexicographic (cost, run) minimum over runs (multi-start
//                 best-of: the minimum objective is selected, Section 3).
//   plan_kernel   decode a solution into xM, xR, yM, yR.
//
// Integer arithmetic only; no tensor cores: this is combinatorial search,
// not a dense contraction.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "elsr_vns.cuh"

namespace elsr {

namespace {

using vns::kFull;
using vns::stage_row_warp;
using vns::subwarp_min;
using vns::umin64;

// ---------------------------------------------------------------------------
// stage_kernel: every warp stages a contiguous chunk of rows (rows numbered
// across the instances in order).  The warp finds the instance of its first
// row with a 32-way search over the instances' first rows (one coalesced
// probe per level: two levels for 1024 instances) and then walks forward.
// ---------------------------------------------------------------------------
__global__ void stage_kernel(const StageParams p, int64_t total_rows) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const InstDesc* insts = p.ip.insts;
  if (p.ninst <= 0) return;
  const int64_t chunk = (total_rows + nw - 1) / nw;
  const int64_t row0 = gw * chunk;
  const int64_t row1 = row0 + chunk < total_rows ? row0 + chunk : total_rows;
  if (row0 >= row1) return;
  // the last instance whose rows start at or before row0: insts[lo] always
  // qualifies, and each level narrows [lo, lo + n) to one of 32 slices
  int lo = 0, n = p.ninst;
  while (n > 1) {
    const int step = (n + 31) >> 5;
    const int i = lo + lane * step;
    const unsigned le = __ballot_sync(kFull, i < lo + n && insts[i].row_off <= row0);
    const int s = 31 - __clz(le);  // lane 0 (i = lo) always qualifies
    lo += s * step;
    n = (s + 1) * step <= n ? step : n - s * step;
  }
  InstDesc id = insts[lo];
  for (int64_t row = row0; row < row1; ++row) {
    while (row >= id.row_off + id.K) id = insts[++lo];  // next non-empty instance
    const int k = (int)(row - id.row_off);
    const int T = id.T;
    stage_row_warp(p.ip.D + id.cell_off + (int64_t)k * T,
                   p.ip.R + id.cell_off + (int64_t)k * T, T, lane,
                   p.gtab + id.tab_off + (int64_t)k * (T + 1),
                   p.ip.hM[row], p.ip.hR[row], p.ip.pM ? p.ip.pM[row] : 0, p.gC0 + row);
  }
}

// ---------------------------------------------------------------------------
// eval_kernel: rows [blockIdx.x * nsub, +nsub) of instance 0, one per
// sub-warp.  Shared memory: tab[nsub][T+1] | C0[nsub] | A | C | L [nsub][T].
// ---------------------------------------------------------------------------
template <typename Acc>
struct EvalLayout {
  uint32_t C0, A, C, L, P, Q, total;
  __host__ __device__ EvalLayout(int rows, int T) {
    uint32_t o = align16((uint32_t)rows * (T + 1) * 8u);
    C0 = o;
    o = align16(o + rows * 8u);
    A = o;
    o = align16(o + (uint32_t)rows * T * 4u);
    C = o;
    o = align16(o + (uint32_t)rows * T * (uint32_t)sizeof(Acc));
    L = o;
    o = align16(o + (uint32_t)rows * T * 8u);
    P = o;
    o = align16(o + (uint32_t)rows * (T + 1) * 4u);
    Q = o;
    o += (uint32_t)rows * (T + 1) * (uint32_t)sizeof(Acc);
    total = o;
  }
};

template <typename Acc, int NW>
__global__ void __launch_bounds__(1024) eval_kernel(const EvalParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long sh_F;
  __shared__ int sh_Finf;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = p.G, lane = tid & (G - 1), sub = tid / G, nsub = nthr / G;
  const int wlane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int K = p.K, T = p.T;
  const InstDesc id = p.ip.insts[0];
  const int row0 = blockIdx.x * nsub;
  const EvalLayout<Acc> lay(nsub, T);
  int2* tab = (int2*)smem;
  int64_t* C0 = (int64_t*)(smem + lay.C0);
  int32_t* A = (int32_t*)(smem + lay.A);
  Acc* C = (Acc*)(smem + lay.C);
  int2* Lst = (int2*)(smem + lay.L);
  int32_t* Pst = (int32_t*)(smem + lay.P);
  Acc* Qst = (Acc*)(smem + lay.Q);

  for (int i = warp; i < nsub; i += nwarps) {
    const int k = row0 + i;
    if (k < K) {
      stage_row_warp(p.ip.D + id.cell_off + (int64_t)k * T,
                     p.ip.R + id.cell_off + (int64_t)k * T, T, wlane,
                     tab + (int64_t)i * (T + 1), p.ip.hM[id.row_off + k],
                     p.ip.hR[id.row_off + k], p.ip.pM ? p.ip.pM[id.row_off + k] : 0, &C0[i]);
    }
  }
  if (tid == 0) {
    sh_F = 0;
    sh_Finf = 0;
  }
  __syncthreads();
  if (p.mode == 1 && p.rowcost_in) {
    long long s = 0;
    int ni = 0;
    for (int k = tid; k < K; k += nthr) {
      const int64_t c = p.rowcost_in[k];
      if (c == INT64_MAX) ++ni; else s += c;
    }
    if (s) atomicAdd((unsigned long long*)&sh_F, (unsigned long long)s);
    if (ni) atomicAdd(&sh_Finf, ni);
    __syncthreads();
  }
  const int64_t F = sh_F;
  const int Finf = sh_Finf;

  const int k = row0 + sub;
  const bool valid = k < K;
  RowState<Acc> cur;
  RowCosts rc{0, 0, 0, 0, 0};
  int64_t c0 = 0;
  const int2* tk = tab + (int64_t)sub * (T + 1);
  int32_t* Ak = A + sub * T;
  Acc* Ck = C + sub * T;
  int2* Lk = Lst + sub * T;
  int32_t* Pk = Pst + sub * (T + 1);
  Acc* Qk = Qst + sub * (T + 1);
  cur.S = 0;
  cur.bad = T;
  cur.nR = 0;
  cur.ld = -1;
  if (valid) {
    const int64_t ro = id.row_off + k;
    rc = vns::row_costs(p.ip, ro);
    c0 = C0[sub];
    cur.b = p.bits[k];
    if (lane == 0) {
      int dummy = 0;
      cur.S = build_row<Acc, NW>(tk, T, rc, cur.b, Ak, Ck, Lk, Pk, Qk, cur.bad, cur.nR, cur.ld,
                                 dummy);
    }
  }
  __syncwarp();
  {
    const int leader = wlane & ~(G - 1);
    cur.S = __shfl_sync(kFull, cur.S, leader);
    cur.bad = __shfl_sync(kFull, cur.bad, leader);
    cur.nR = __shfl_sync(kFull, cur.nR, leader);
    cur.ld = __shfl_sync(kFull, cur.ld, leader);
  }
  const int64_t rck = valid ? state_cost<Acc>(cur.S, cur.bad, T, c0) : 0;
  if (valid && lane == 0 && p.rowcost_out) p.rowcost_out[k] = rck;

  const int infk = rck == INT64_MAX;
  const int64_t others = (Finf - infk > 0) ? INT64_MAX : F - (infk ? 0 : rck);
  uint64_t bestP = ~0ull, bestG = ~0ull;
  for (int j = 1; j <= 3; ++j) {
    if (!(p.mask & (1u << (j - 1)))) continue;
    const int M = row_moves(T, j);
    if (M <= 0 || !valid) continue;
    const uint32_t loff = j == 1 ? 0u : (j == 2 ? (uint32_t)T : 2u * T);
    const uint32_t goff = j == 1 ? 0u : (j == 2 ? (uint32_t)(K * T) : 2u * K * T);
    for (int l = lane; l < M; l += G) {
      int st = 0;
      const Acc S = eval_move<Acc, NW>(tk, T, rc, cur, Ak, Ck, Lk, Pk, Qk, j, l, st);
      const int64_t nc = row_cost<Acc>(S, c0);
      bestP = umin64(bestP, pack_key(nc, loff + (uint32_t)l));
      if (p.mode == 1) {
        const int64_t nt = (others == INT64_MAX || nc == INT64_MAX) ? INT64_MAX : others + nc;
        bestG = umin64(bestG, pack_key(nt, goff + (uint32_t)(k * M + l)));
      }
      if (j == p.single_j) {
        if (p.move_cost) p.move_cost[(int64_t)k * M + l] = nc;
        if (p.move_win) p.move_win[(int64_t)k * M + l] = st;
      }
    }
  }
  bestP = subwarp_min(bestP, G);
  bestG = subwarp_min(bestG, G);
  if (valid && lane == 0) {
    if (p.pp_key) p.pp_key[k] = bestP;
    if (p.scratch) {
      if (p.mode == 1 && bestG != ~0ull)
        atomicMin((unsigned long long*)&p.scratch[0], (unsigned long long)bestG);
      const bool imp = bestP != ~0ull && key_cost(bestP) < rck;
      const int64_t after = imp ? key_cost(bestP) : rck;
      if (after == INT64_MAX) {
        atomicAdd((unsigned long long*)&p.scratch[2], 1ull);
      } else {
        atomicAdd((unsigned long long*)&p.scratch[1], (unsigned long long)after);
      }
      if (imp) atomicAdd((unsigned long long*)&p.scratch[3], 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// eval_wide_kernel: one row of instance 0 per CTA, every thread of the block
// on its moves (a neighbourhood of one row is 2T or 2(T-1) moves, so about
// one or two per thread).  Warp 0 stages the row and builds its cache with
// the lane-parallel rebuild; the block's minimum goes through shared memory.
// Same outputs as eval_kernel.  Shared memory: the single-row layout of the
// GVNS kernels without their save slots.
// ---------------------------------------------------------------------------
template <typename Acc, int NW>
__global__ void __launch_bounds__(128, 1) eval_wide_kernel(const EvalParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long sh_F;
  __shared__ int sh_Finf;
  __shared__ unsigned long long sh_key[2][4];
  const int tid = threadIdx.x, nthr = blockDim.x, wlane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const int K = p.K, T = p.T, k = blockIdx.x;
  const InstDesc id = p.ip.insts[0];
  const VnsLayout lay = vns_layout(1, T, (int)sizeof(Acc), true);
  vns::Rows<Acc> m;
  m.tab = (const int2*)(smem + lay.tab);
  m.place(smem, lay.rc, lay.C0, lay.bits, lay.S, lay.mark, lay.nR, lay.A, lay.C, lay.L, lay.P,
          lay.Q, 0);  // no save slots
  m.slot = 0;
  m.T = T;
  m.C_ = 1;
  m.crank = 0;
  m.ts = true;
  const int64_t ro = id.row_off + k;
  if (warp == 0) {
    stage_row_warp(p.ip.D + id.cell_off + (int64_t)k * T, p.ip.R + id.cell_off + (int64_t)k * T,
                   T, wlane, (int2*)(smem + lay.tab), p.ip.hM[ro], p.ip.hR[ro],
                   p.ip.pM ? p.ip.pM[ro] : 0, &m.C0()[0]);
    if (wlane == 0) {
      m.rc()[0] = vns::row_costs(p.ip, ro);
      m.bits()[0] = p.bits[k];
    }
  }
  if (tid == 0) {
    sh_F = 0;
    sh_Finf = 0;
  }
  __syncthreads();
  if (p.mode == 1 && p.rowcost_in) {
    long long sf = 0;
    int ni = 0;
    for (int r = tid; r < K; r += nthr) {
      const int64_t c = p.rowcost_in[r];
      if (c == INT64_MAX) ++ni; else sf += c;
    }
    if (sf) atomicAdd((unsigned long long*)&sh_F, (unsigned long long)sf);
    if (ni) atomicAdd(&sh_Finf, ni);
  }
  if (warp == 0) vns::rebuild_any<Acc, NW>(m, 0, wlane, 32, kFull);
  __syncthreads();
  const int64_t F = sh_F;
  const int Finf = sh_Finf;
  const RowState<Acc> cur = m.state(0);
  const RowCosts rc = m.rc()[0];
  const int64_t c0 = m.C0()[0];
  const int64_t rck = m.cost(0);
  if (tid == 0 && p.rowcost_out) p.rowcost_out[k] = rck;
  const int infk = rck == INT64_MAX;
  const int64_t others = (Finf - infk > 0) ? INT64_MAX : F - (infk ? 0 : rck);
  uint64_t bestP = ~0ull, bestG = ~0ull;
  for (int j = 1; j <= 3; ++j) {
    if (!(p.mask & (1u << (j - 1)))) continue;
    const int M = row_moves(T, j);
    if (M <= 0) continue;
    const uint32_t loff = j == 1 ? 0u : (j == 2 ? (uint32_t)T : 2u * T);
    const uint32_t goff = j == 1 ? 0u : (j == 2 ? (uint32_t)(K * T) : 2u * K * T);
    for (int l = tid; l < M; l += nthr) {
      int st = 0;
      const Acc S = eval_move<Acc, NW>(m.tab, T, rc, cur, m.A(), m.C(), m.L(), m.P(), m.Q(), j, l, st);
      const int64_t nc = row_cost<Acc>(S, c0);
      bestP = umin64(bestP, pack_key(nc, loff + (uint32_t)l));
      if (p.mode == 1) {
        const int64_t nt = (others == INT64_MAX || nc == INT64_MAX) ? INT64_MAX : others + nc;
        bestG = umin64(bestG, pack_key(nt, goff + (uint32_t)(k * M + l)));
      }
      if (j == p.single_j) {
        if (p.move_cost) p.move_cost[(int64_t)k * M + l] = nc;
        if (p.move_win) p.move_win[(int64_t)k * M + l] = st;
      }
    }
  }
  bestP = subwarp_min(bestP, 32);
  bestG = subwarp_min(bestG, 32);
  if (wlane == 0) {
    sh_key[0][warp] = bestP;
    sh_key[1][warp] = bestG;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < nwarps; ++w) {
      bestP = umin64(bestP, sh_key[0][w]);
      bestG = umin64(bestG, sh_key[1][w]);
    }
    if (p.pp_key) p.pp_key[k] = bestP;
    if (p.scratch) {
      if (p.mode == 1 && bestG != ~0ull)
        atomicMin((unsigned long long*)&p.scratch[0], (unsigned long long)bestG);
      const bool imp = bestP != ~0ull && key_cost(bestP) < rck;
      const int64_t after = imp ? key_cost(bestP) : rck;
      if (after == INT64_MAX) {
        atomicAdd((unsigned long long*)&p.scratch[2], 1ull);
      } else {
        atomicAdd((unsigned long long*)&p.scratch[1], (unsigned long long)after);
      }
      if (imp) atomicAdd((unsigned long long*)&p.scratch[3], 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// bestof_kernel: one block, lexicographic (cost, run) minimum.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) bestof_kernel(const BestofParams p) {
  __shared__ unsigned long long sh[32];
  uint64_t best = ~0ull;
  for (int i = threadIdx.x; i < p.n; i += blockDim.x)
    best = umin64(best, pack_key(p.out[i].best_cost, (uint32_t)i));
  for (int o = 16; o > 0; o >>= 1) best = umin64(best, __shfl_xor_sync(kFull, best, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : ~0ull;
    for (int o = 16; o > 0; o >>= 1) best = umin64(best, __shfl_xor_sync(kFull, best, o));
    if (threadIdx.x == 0) *p.best_key = best;
  }
}

// ---------------------------------------------------------------------------
// plan_kernel: one thread per row; xM, xR, yM, yR by the decode rule (-1
// everywhere after a shortfall).
// ---------------------------------------------------------------------------
__global__ void plan_kernel(const PlanParams p) {
  const InstDesc id = p.ip.insts[p.inst];
  const int K = id.K, T = id.T;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int32_t* D = p.ip.D + id.cell_off + (int64_t)k * T;
  const int32_t* R = p.ip.R + id.cell_off + (int64_t)k * T;
  const RowBits b = p.bits[k];
  const uint64_t u0 = b.m0 | b.r0, u1 = b.m1 | b.r1;
  const int64_t KT = (int64_t)K * T;
  int32_t* xM = p.plan + (int64_t)k * T;
  int32_t* xR = xM + KT;
  int32_t* yM = xM + 2 * KT;
  int32_t* yR = xM + 3 * KT;
  int32_t ym = 0, yr = 0;
  bool ok = true;
  for (int t = 0; t < T; ++t) {
    const int32_t avail = yr + R[t];
    int32_t xm = 0, xr = 0;
    if (ok && bit_of(u0, u1, t)) {
      const int n = next_set(u0, u1, t, T);
      int32_t need = -ym;
      for (int i = t; i < n; ++i) need += D[i];
      if (bit_of(b.r0, b.r1, t)) xr = avail < need ? avail : need;
      if (bit_of(b.m0, b.m1, t)) xm = need - xr;
      else if (xr < need) ok = false;
    }
    ym = ym + xm + xr - D[t];
    if (ym < 0) ok = false;
    yr = avail - xr;
    xM[t] = ok ? xm : -1;
    xR[t] = ok ? xr : -1;
    yM[t] = ok ? ym : -1;
    yR[t] = ok ? yr : -1;
  }
}

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than it was last given on this device (the attribute call is not free).
template <typename Acc>
cudaError_t eval_prepare_t(int T, size_t smem) {
  constexpr int kDevices = 64;
  // per word count and device, the largest size granted so far (0: none);
  // handles on several host threads may race here, which at worst repeats
  // the attribute call
  static std::atomic<int> granted[2][kDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int w = T <= 64 ? 0 : 1;
  const bool cached = dev >= 0 && dev < kDevices;
  if (cached && granted[w][dev].load(std::memory_order_relaxed) >= (int)smem) return cudaSuccess;
  e = w == 0 ? cudaFuncSetAttribute(eval_kernel<Acc, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem)
             : cudaFuncSetAttribute(eval_kernel<Acc, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
  if (e == cudaSuccess && cached) {
    int cur = granted[w][dev].load(std::memory_order_relaxed);
    while (cur < (int)smem &&
           !granted[w][dev].compare_exchange_weak(cur, (int)smem, std::memory_order_relaxed)) {
    }
  }
  return e;
}

template <typename Acc>
void eval_launch_t(const EvalParams& p, int blocks, int threads, size_t smem, cudaStream_t s) {
  if (p.T <= 64)
    eval_kernel<Acc, 1><<<blocks, threads, smem, s>>>(p);
  else
    eval_kernel<Acc, 2><<<blocks, threads, smem, s>>>(p);
}

template <typename Acc>
cudaError_t eval_wide_launch_t(const EvalParams& p, int threads, cudaStream_t s) {
  const size_t smem = vns_layout(1, p.T, (int)sizeof(Acc), true).save;
  if (p.T <= 64)
    eval_wide_kernel<Acc, 1><<<p.K, threads, smem, s>>>(p);
  else
    eval_wide_kernel<Acc, 2><<<p.K, threads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_eval_wide(const EvalParams& p, bool acc64, int threads, cudaStream_t s) {
  return acc64 ? eval_wide_launch_t<int64_t>(p, threads, s) : eval_wide_launch_t<int32_t>(p, threads, s);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_stage(const StageParams& p, int total_rows, cudaStream_t s) {
  if (total_rows <= 0) return cudaSuccess;
  const int threads = 256;
  int blocks = (total_rows * 32 + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  stage_kernel<<<blocks, threads, 0, s>>>(p, total_rows);
  return cudaGetLastError();
}

size_t eval_smem_bytes(int rows, int T, bool acc64) {
  return acc64 ? EvalLayout<int64_t>(rows, T).total : EvalLayout<int32_t>(rows, T).total;
}

cudaError_t eval_prepare(bool acc64, int T, size_t smem) {
  return acc64 ? eval_prepare_t<int64_t>(T, smem) : eval_prepare_t<int32_t>(T, smem);
}

cudaError_t launch_eval(const EvalParams& p, bool acc64, int blocks, int threads,
                        size_t smem, cudaStream_t s) {
  if (acc64)
    eval_launch_t<int64_t>(p, blocks, threads, smem, s);
  else
    eval_launch_t<int32_t>(p, blocks, threads, smem, s);
  return cudaGetLastError();
}

cudaError_t launch_bestof(const BestofParams& p, cudaStream_t s) {
  bestof_kernel<<<1, 1024, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_plan(const PlanParams& p, int K, cudaStream_t s) {
  const int threads = 128;
  plan_kernel<<<(K + threads - 1) / threads, threads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace elsr
