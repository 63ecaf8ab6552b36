// elsr_kernels.cu -- sm_103a kernels of the ELSR VNS hot path.
//
//   stage_kernel  prefix tables of every instance row into global memory
//                 (warp-shuffle scans), for instances too large to stage in
//                 shared memory.
//   eval_kernel   one best-improvement evaluation of whole neighbourhoods of
//                 one instance (Algorithm 1's "find best neighbour" for every
//                 product at once): stage rows in shared memory, build each
//                 row's cache, delta re-decode every candidate, sub-warp
//                 argmin per product, block/global argmin for mode G.
//   vns_kernel    persistent GVNS (Algorithm 2) with VND (Algorithm 1): one
//                 CTA per run, runs taken from a device work queue; instance
//                 rows, setup bits and row caches live in shared memory for
//                 the whole run.
//   bestof_kernel lexicographic (cost, run) minimum over runs (multi-start
//                 best-of, the "minimum one is selected" of Section 3).
//   plan_kernel   decode a solution into xM, xR, yM, yR.
//
// Integer arithmetic only; no tensor cores: this is combinatorial search,
// not a dense contraction.  Row ownership: product k belongs to sub-warp
// k mod nsub (G lanes); that sub-warp evaluates, applies and shakes row k,
// so Algorithm 1's product loop needs no barrier between neighbourhoods.
#include <cuda_runtime.h>
#include <stdint.h>

#include "elsr_internal.h"

namespace elsr {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) {
  return a < b ? a : b;
}

__device__ __forceinline__ uint64_t subwarp_min(uint64_t v, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) v = umin64(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ RowBits all_open(int T) {
  RowBits b;
  b.m0 = T >= 64 ? ~0ull : ((1ull << T) - 1ull);
  b.m1 = T > 64 ? (T >= 128 ? ~0ull : ((1ull << (T - 64)) - 1ull)) : 0ull;
  b.r0 = b.m0;
  b.r1 = b.m1;
  return b;
}

// Stage one row with a full warp: tab[0..T] = {CD[j], CR1[j]} by warp
// inclusive scans over 32-period chunks (coalesced int32 loads), and the row
// constant C0 = hR * sum R(t)(T-t) - hM * sum D(t)(T-t).
__device__ void stage_row_warp(const int32_t* __restrict__ D,
                               const int32_t* __restrict__ R, int T, int lane,
                               int2* tab, int32_t hM, int32_t hR,
                               int64_t* C0) {
  int32_t carryD = 0, carryR = 0;
  int64_t wd = 0, wr = 0;
  for (int base = 0; base < T; base += 32) {
    const int t = base + lane;
    const int32_t d = t < T ? __ldg(D + t) : 0;
    const int32_t r = t < T ? __ldg(R + t) : 0;
    wd += (int64_t)d * (T - t);
    wr += (int64_t)r * (T - t);
    int32_t sd = d, sr = r;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t a = __shfl_up_sync(kFull, sd, o);
      const int32_t b = __shfl_up_sync(kFull, sr, o);
      if (lane >= o) {
        sd += a;
        sr += b;
      }
    }
    if (t < T) {
      tab[t + 1].x = carryD + sd;  // CD[t+1]
      tab[t].y = carryR + sr;      // CR1[t]
    }
    carryD += __shfl_sync(kFull, sd, 31);
    carryR += __shfl_sync(kFull, sr, 31);
  }
  wd = warp_sum64(wd);
  wr = warp_sum64(wr);
  if (lane == 0) {
    tab[0].x = 0;
    tab[T].y = carryR;
    *C0 = (int64_t)hR * wr - (int64_t)hM * wd;
  }
}

// ---------------------------------------------------------------------------
// stage_kernel: one warp per row of every instance.
// ---------------------------------------------------------------------------
__global__ void stage_kernel(const StageParams p) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  // rows are enumerated instance by instance
  int inst = 0;
  int64_t row_base = 0;
  for (int64_t row = gw;; row += nw) {
    while (inst < p.ninst && row >= row_base + p.ip.insts[inst].K) {
      row_base += p.ip.insts[inst].K;
      ++inst;
    }
    if (inst >= p.ninst) return;
    const InstDesc id = p.ip.insts[inst];
    const int k = (int)(row - row_base);
    const int T = id.T;
    stage_row_warp(p.ip.D + id.cell_off + (int64_t)k * T,
                   p.ip.R + id.cell_off + (int64_t)k * T, T, lane,
                   p.gtab + id.tab_off + (int64_t)k * (T + 1),
                   p.ip.hM[id.row_off + k], p.ip.hR[id.row_off + k],
                   p.gC0 + id.row_off + k);
  }
}

// ---------------------------------------------------------------------------
// Shared helpers of the VNS kernel.
// ---------------------------------------------------------------------------
template <typename Acc>
struct RunSmem {
  const int2* tab;  // [K][T+1] (shared or global)
  RowCosts* rc;     // [K]
  int64_t* C0;      // [K]
  RowBits* bits;    // [K]
  Acc* S;           // [K]
  int32_t* bad;     // [K]
  int32_t* A;       // [K][T]
  Acc* C;           // [K][T]
  unsigned char* save;
  uint32_t slot;
  int K, T;

  __device__ __forceinline__ RowState<Acc> state(int k) const {
    RowState<Acc> st;
    st.b = bits[k];
    st.S = S[k];
    st.bad = bad[k];
    return st;
  }
  __device__ __forceinline__ int64_t cost(int k) const {
    return row_cost<Acc>(S[k], C0[k]);
  }
  __device__ __forceinline__ unsigned char* slot_ptr(int par, int j) const {
    return save + (uint32_t)(par * kMaxShake + j) * slot;
  }
};

// Copy row k of the cache to / from a save slot (sub-warp collective).
template <typename Acc>
__device__ void save_row(const RunSmem<Acc>& m, int k, unsigned char* sl,
                         int lane, int G) {
  const int T = m.T;
  int32_t* sA = (int32_t*)(sl + 48);
  Acc* sC = (Acc*)(sl + 48 + (((uint32_t)T * 4u + 7u) & ~7u));
  for (int s = lane; s < T; s += G) {
    sA[s] = m.A[k * T + s];
    sC[s] = m.C[k * T + s];
  }
  if (lane == 0) {
    *(RowBits*)sl = m.bits[k];
    *(int64_t*)(sl + 32) = (int64_t)m.S[k];
    *(int32_t*)(sl + 40) = m.bad[k];
  }
}

template <typename Acc>
__device__ void restore_row(const RunSmem<Acc>& m, int k,
                            const unsigned char* sl, int lane, int G) {
  const int T = m.T;
  const int32_t* sA = (const int32_t*)(sl + 48);
  const Acc* sC = (const Acc*)(sl + 48 + (((uint32_t)T * 4u + 7u) & ~7u));
  for (int s = lane; s < T; s += G) {
    m.A[k * T + s] = sA[s];
    m.C[k * T + s] = sC[s];
  }
  if (lane == 0) {
    m.bits[k] = *(const RowBits*)sl;
    m.S[k] = (Acc)(*(const int64_t*)(sl + 32));
    m.bad[k] = *(const int32_t*)(sl + 40);
  }
}

// Apply move (j, local) to row k and patch its cache (sub-warp collective;
// every lane of the warp must call it, `imp` says whether this sub-warp
// applies).  A feasible row is patched over the walked window and shifted
// after the merge point; an infeasible one is rebuilt.
template <typename Acc>
__device__ void apply_move_row(const RunSmem<Acc>& m, bool imp, int k, int j,
                               int local, int lane, int G, int leader) {
  const int T = m.T;
  int merge = T;
  Acc delta = 0;
  if (imp && lane == 0) {
    const RowState<Acc> cur = m.state(k);
    RowBits nb = cur.b;
    apply_row_move(nb, T, j, local);
    const int2* tk = m.tab + (int64_t)k * (T + 1);
    int32_t* Ak = m.A + k * T;
    Acc* Ck = m.C + k * T;
    int dummy = 0;
    if (cur.bad == T) {
      const DeltaOut<Acc> d =
          eval_move<Acc, true>(tk, T, m.rc[k], cur, Ak, Ck, j, local, dummy);
      m.S[k] = d.S;
      merge = d.merge;
      delta = d.delta;
      m.bad[k] = T;
    } else {
      int b2 = T;
      m.S[k] = build_row<Acc>(tk, T, m.rc[k], nb, Ak, Ck, b2, dummy);
      m.bad[k] = b2;
    }
    m.bits[k] = nb;
  }
  __syncwarp();
  merge = __shfl_sync(kFull, merge, leader);
  delta = __shfl_sync(kFull, delta, leader);
  if (imp && merge < T) {
    const RowBits nb = m.bits[k];
    const uint64_t u0 = nb.m0 | nb.r0, u1 = nb.m1 | nb.r1;
    Acc* Ck = m.C + k * T;
    for (int s = merge + lane; s < T; s += G)
      if (bit_of(u0, u1, s)) Ck[s] += delta;
  }
  __syncwarp();
}

// Best move of row k in N_j over this lane's share of the candidates.
template <typename Acc>
__device__ __forceinline__ uint64_t row_best_p(const RunSmem<Acc>& m, int k,
                                               const RowState<Acc>& cur, int j,
                                               int M, int lane, int G,
                                               uint32_t& segs) {
  const int T = m.T;
  const int2* tk = m.tab + (int64_t)k * (T + 1);
  int32_t* Ak = m.A + k * T;
  Acc* Ck = m.C + k * T;
  const RowCosts rc = m.rc[k];
  const int64_t c0 = m.C0[k];
  uint64_t best = ~0ull;
  int sg = 0;
  for (int l = lane; l < M; l += G) {
    const DeltaOut<Acc> d = eval_move<Acc, false>(tk, T, rc, cur, Ak, Ck, j, l, sg);
    best = umin64(best, pack_key(row_cost<Acc>(d.S, c0), (uint32_t)l));
  }
  segs += (uint32_t)sg;
  return best;
}

// ---------------------------------------------------------------------------
// vns_kernel
// ---------------------------------------------------------------------------
template <typename Acc, bool TS>
__global__ void __launch_bounds__(1024, 1) vns_kernel(const VnsParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int sh_run;
  __shared__ unsigned long long sh_acc[2];
  __shared__ int sh_ninf[2];
  __shared__ unsigned long long sh_gkey[2];
  __shared__ long long sh_F;
  __shared__ int sh_Finf;
  __shared__ unsigned long long sh_applied, sh_segs;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = p.G;
  const int lane = tid & (G - 1), sub = tid / G, nsub = nthr / G;
  const int wlane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int leader = wlane & ~(G - 1);

  for (;;) {
    if (tid == 0) sh_run = atomicAdd(p.queue, 1);
    __syncthreads();
    const int r = sh_run;
    __syncthreads();
    if (r >= p.nruns) return;
    const RunDesc rd = p.runs[r];
    const InstDesc id = p.ip.insts[rd.inst];
    const int K = id.K, T = id.T;
    const VnsLayout L = vns_layout(K, T, (int)sizeof(Acc), TS);
    RunSmem<Acc> m;
    m.tab = TS ? (const int2*)(smem + L.tab) : (p.ip.gtab + id.tab_off);
    m.rc = (RowCosts*)(smem + L.rc);
    m.C0 = (int64_t*)(smem + L.C0);
    m.bits = (RowBits*)(smem + L.bits);
    m.S = (Acc*)(smem + L.S);
    m.bad = (int32_t*)(smem + L.bad);
    m.A = (int32_t*)(smem + L.A);
    m.C = (Acc*)(smem + L.C);
    m.save = smem + L.save;
    m.slot = L.slot;
    m.K = K;
    m.T = T;

    // ---- A1: stage the instance (one warp per row) ----
    for (int k = warp; k < K; k += nwarps) {
      const int64_t ro = id.row_off + k;
      if (TS) {
        stage_row_warp(p.ip.D + id.cell_off + (int64_t)k * T,
                       p.ip.R + id.cell_off + (int64_t)k * T, T, wlane,
                       (int2*)(smem + L.tab) + (int64_t)k * (T + 1),
                       p.ip.hM[ro], p.ip.hR[ro], &m.C0[k]);
      } else if (wlane == 0) {
        m.C0[k] = p.ip.gC0[ro];
      }
      if (wlane == 0) {
        m.rc[k] = RowCosts{p.ip.kM[ro], p.ip.kR[ro], p.ip.hM[ro], p.ip.hR[ro]};
        m.bits[k] = rd.start_off >= 0 ? p.start_bits[rd.start_off + k] : all_open(T);
      }
    }
    if (tid == 0) {
      sh_acc[0] = sh_acc[1] = 0ull;
      sh_ninf[0] = sh_ninf[1] = 0;
      sh_gkey[0] = sh_gkey[1] = ~0ull;
      sh_applied = 0ull;
      sh_segs = 0ull;
    }
    __syncthreads();

    uint32_t my_segs = 0;
    uint32_t my_applied = 0;
    // row caches of the start solution (row owner's leader lane)
    if (lane == 0) {
      for (int k = sub; k < K; k += nsub) {
        int b = T, dummy = 0;
        m.S[k] = build_row<Acc>(m.tab + (int64_t)k * (T + 1), T, m.rc[k],
                                m.bits[k], m.A + k * T, m.C + k * T, b, dummy);
        m.bad[k] = b;
      }
    }
    __syncwarp();

    const int Kr = ((K + nsub - 1) / nsub) * nsub;  // uniform row-loop bound
    const int64_t moves_per_cycle =
        (int64_t)K * (2 * T + (T > 1 ? 2 * (T - 1) : 0));
    int status = 0;
    int64_t cycles_total = 0;
    int tp = 0;  // parity of the total accumulators

    // Saturating team-wide objective (sum of row costs).  Precondition: the
    // accumulators of parity `tp` are zero and a barrier separates their
    // reset from this call.
    auto team_total = [&]() -> int64_t {
      if (lane == 0) {
        int64_t s = 0;
        int ni = 0;
        for (int k = sub; k < K; k += nsub) {
          const int64_t c = m.cost(k);
          if (c == INT64_MAX) ++ni; else s += c;
        }
        if (s) atomicAdd(&sh_acc[tp], (unsigned long long)s);
        if (ni) atomicAdd(&sh_ninf[tp], ni);
      }
      __syncthreads();
      const int64_t tot = sh_ninf[tp] ? INT64_MAX : (int64_t)sh_acc[tp];
      if (tid == 0) {
        sh_acc[tp ^ 1] = 0ull;
        sh_ninf[tp ^ 1] = 0;
      }
      tp ^= 1;
      return tot;
    };

    // VND of Algorithm 1 (pipe form), mode P: every product takes its best
    // strictly improving move of N_j; repeat the j = 1..3 sweep until no
    // product improves.  Returns the sweeps run, or -1 at the cap.
    auto vnd_p = [&]() -> int {
      int cycles = 0;
      for (;;) {
        int improved = 0;
        for (int j = 1; j <= 3; ++j) {
          const int M = row_moves(T, j);
          if (M <= 0) continue;
          for (int kk = sub; kk < Kr; kk += nsub) {
            const bool valid = kk < K;
            const int k = valid ? kk : 0;
            uint64_t best = ~0ull;
            RowState<Acc> cur;
            if (valid) {
              cur = m.state(k);
              best = row_best_p<Acc>(m, k, cur, j, M, lane, G, my_segs);
            }
            best = subwarp_min(best, G);
            const bool imp = valid && key_cost(best) < m.cost(k);
            apply_move_row<Acc>(m, imp, k, j, key_index(best), lane, G, leader);
            if (imp) {
              improved = 1;
              if (lane == 0) ++my_applied;
            }
          }
        }
        ++cycles;
        if (!__syncthreads_or(improved)) break;
        if (cycles >= p.vnd_cap) return -1;
      }
      return cycles;
    };

    // VND, mode G: one best move of the whole neighbourhood, by
    // (new objective, global index), applied when it lowers the objective.
    auto vnd_g = [&]() -> int {
      if (tid == 0) {
        sh_F = 0;
        sh_Finf = 0;
      }
      __syncthreads();
      if (lane == 0) {
        long long s = 0;
        int ni = 0;
        for (int k = sub; k < K; k += nsub) {
          const int64_t c = m.cost(k);
          if (c == INT64_MAX) ++ni; else s += c;
        }
        if (s) atomicAdd((unsigned long long*)&sh_F, (unsigned long long)s);
        if (ni) atomicAdd(&sh_Finf, ni);
      }
      __syncthreads();
      int cycles = 0, e = 0;
      for (;;) {
        bool improved = false;
        for (int j = 1; j <= 3; ++j) {
          const int M = row_moves(T, j);
          if (M <= 0) continue;
          const int64_t F = sh_F;
          const int Finf = sh_Finf;
          const int64_t total = Finf ? INT64_MAX : F;
          for (int kk = sub; kk < Kr; kk += nsub) {
            const bool valid = kk < K;
            const int k = valid ? kk : 0;
            uint64_t best = ~0ull;
            if (valid) {
              const RowState<Acc> cur = m.state(k);
              const int64_t rck = m.cost(k);
              const int infk = rck == INT64_MAX;
              const int64_t others =
                  (Finf - infk > 0) ? INT64_MAX : F - (infk ? 0 : rck);
              const int2* tk = m.tab + (int64_t)k * (T + 1);
              const RowCosts rc = m.rc[k];
              const int64_t c0 = m.C0[k];
              int sg = 0;
              for (int l = lane; l < M; l += G) {
                const DeltaOut<Acc> d = eval_move<Acc, false>(
                    tk, T, rc, cur, m.A + k * T, m.C + k * T, j, l, sg);
                const int64_t nc = row_cost<Acc>(d.S, c0);
                const int64_t nt =
                    (others == INT64_MAX || nc == INT64_MAX) ? INT64_MAX : others + nc;
                best = umin64(best, pack_key(nt, (uint32_t)(k * M + l)));
              }
              my_segs += (uint32_t)sg;
            }
            best = subwarp_min(best, G);
            if (valid && lane == 0 && best != ~0ull) atomicMin(&sh_gkey[e], best);
          }
          __syncthreads();
          const uint64_t gk = sh_gkey[e];
          if (tid == 0) sh_gkey[e ^ 1] = ~0ull;
          const bool imp = gk != ~0ull && key_cost(gk) < total;
          if (imp) {
            const int gi = key_index(gk);
            const int kw = gi / M, lw = gi - kw * M;
            const bool mine = (kw % nsub) == sub;
            const int64_t old = mine ? m.cost(kw) : 0;
            apply_move_row<Acc>(m, mine, kw, j, lw, lane, G, leader);
            if (mine && lane == 0) {
              const int64_t nw = m.cost(kw);
              if (old == INT64_MAX) {
                sh_Finf = Finf - 1;
                sh_F = F + nw;
              } else {
                sh_F = F - old + nw;
              }
              ++my_applied;
            }
            improved = true;
          }
          __syncthreads();
          e ^= 1;
        }
        ++cycles;
        if (!improved) break;
        if (cycles >= p.vnd_cap) return -1;
      }
      return cycles;
    };

    auto vnd = [&]() -> int { return rd.mode == 0 ? vnd_p() : vnd_g(); };

    // ---- initial VND and GVNS (Algorithm 2) ----
    int cyc = vnd();
    if (cyc < 0) status = kStatusCap; else cycles_total += cyc;
    int64_t fx = team_total();
    int kk_ = 1;  // neighbourhood index k of Algorithm 2
    uint64_t h = 0;
    int64_t iters_done = 0, accepted = 0;
    const bool log = rd.traj_off >= 0;
    for (int it = 0; it < rd.iters && status == 0; ++it) {
      const int par = it & 1;
      const int ks = kk_;
      // Shake(x, k): k moves of N_k from splitmix64 draws, applied by the
      // owners of the hit rows (first touch saves the row for a rejection).
      const int per = row_moves(T, ks);
      const int64_t size = per > 0 ? (int64_t)K * per : 0;
      int rows[kMaxShake], locs[kMaxShake];
      bool first[kMaxShake];
#pragma unroll
      for (int j = 0; j < kMaxShake; ++j) {
        rows[j] = -1;
        locs[j] = 0;
        first[j] = false;
        if (j < ks && size > 0) {
          const uint64_t d = shake_draw(rd.seed, (uint64_t)it, (uint64_t)ks, (uint64_t)j);
          const int64_t mv = (int64_t)(d % (uint64_t)size);
          rows[j] = (int)(mv / per);
          locs[j] = (int)(mv - (int64_t)rows[j] * per);
          first[j] = true;
          for (int q = 0; q < j; ++q)
            if (rows[q] == rows[j]) first[j] = false;
        }
      }
#pragma unroll
      for (int j = 0; j < kMaxShake; ++j) {
        const bool mine = rows[j] >= 0 && (rows[j] % nsub) == sub;
        if (mine && first[j]) save_row<Acc>(m, rows[j], m.slot_ptr(par, j), lane, G);
        __syncwarp();
        if (mine && lane == 0) {
          RowBits b = m.bits[rows[j]];
          apply_row_move(b, T, ks, locs[j]);
          m.bits[rows[j]] = b;
        }
        __syncwarp();
      }
      if (lane == 0) {
#pragma unroll
        for (int j = 0; j < kMaxShake; ++j) {
          if (rows[j] >= 0 && first[j] && (rows[j] % nsub) == sub) {
            const int k = rows[j];
            int b = T, dummy = 0;
            m.S[k] = build_row<Acc>(m.tab + (int64_t)k * (T + 1), T, m.rc[k],
                                    m.bits[k], m.A + k * T, m.C + k * T, b, dummy);
            m.bad[k] = b;
          }
        }
      }
      __syncwarp();
      // VND(x')
      cyc = vnd();
      if (cyc < 0) {
        status = kStatusCap;
      } else {
        cycles_total += cyc;
      }
      const int64_t f2 = team_total();
      const int acc = f2 < fx;
      if (tid == 0) {
        if (log) {
          TrajEntry te;
          te.it = it;
          te.k = ks;
          te.cost = f2;
          te.accepted = acc;
          te.reserved = 0;
          p.traj[rd.traj_off + it] = te;
        }
        h = splitmix64(h ^ (uint64_t)f2);
        h = splitmix64(h ^ (((uint64_t)it << 32) | ((uint64_t)ks << 1) | (uint64_t)acc));
      }
      ++iters_done;
      if (acc) {
        fx = f2;
        kk_ = 1;
        ++accepted;
      } else {
        // x'' rejected: the shaken rows go back to x (the other rows never
        // moved: they were locally optimal in x).
#pragma unroll
        for (int j = 0; j < kMaxShake; ++j) {
          const bool mine = rows[j] >= 0 && first[j] && (rows[j] % nsub) == sub;
          if (mine) restore_row<Acc>(m, rows[j], m.slot_ptr(par, j), lane, G);
          __syncwarp();
        }
        kk_ = kk_ % rd.kmax + 1;
      }
      if ((it & 255) == 255) {  // keep the 32-bit per-thread counter small
        unsigned long long v = my_segs;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (wlane == 0 && v) atomicAdd(&sh_segs, v);
        my_segs = 0;
      }
    }

    // ---- outputs ----
    for (int k = tid; k < K; k += nthr) p.out_bits[rd.bits_off + k] = m.bits[k];
    {
      unsigned long long v = my_segs, a = my_applied;
      for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(kFull, v, o);
        a += __shfl_xor_sync(kFull, a, o);
      }
      if (wlane == 0) {
        if (v) atomicAdd(&sh_segs, v);
        if (a) atomicAdd(&sh_applied, a);
      }
    }
    __syncthreads();
    if (tid == 0) {
      RunOut o;
      o.best_cost = fx;
      o.traj_hash = h;
      o.moves_evaluated = cycles_total * moves_per_cycle;
      o.evals = cycles_total * 3;
      o.vnd_cycles = cycles_total;
      o.applied = (int64_t)sh_applied;
      o.iterations = iters_done;
      o.accepted = accepted;
      o.segments = (int64_t)sh_segs;
      o.status = status;
      o.reserved = 0;
      p.out[rd.out] = o;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// eval_kernel: rows [blockIdx.x * nsub, +nsub) of instance 0, one per
// sub-warp.
// ---------------------------------------------------------------------------
template <typename Acc>
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

  // layout: tab[nsub][T+1] | C0[nsub] | A[nsub][T] | C[nsub][T]
  int2* tab = (int2*)smem;
  uint32_t o = align16((uint32_t)nsub * (T + 1) * 8u);
  int64_t* C0 = (int64_t*)(smem + o);
  o = align16(o + nsub * 8u);
  int32_t* A = (int32_t*)(smem + o);
  o = align16(o + (uint32_t)nsub * T * 4u);
  Acc* C = (Acc*)(smem + o);

  for (int i = warp; i < nsub; i += nwarps) {
    const int k = row0 + i;
    if (k < K) {
      stage_row_warp(p.ip.D + id.cell_off + (int64_t)k * T,
                     p.ip.R + id.cell_off + (int64_t)k * T, T, wlane,
                     tab + (int64_t)i * (T + 1), p.ip.hM[id.row_off + k],
                     p.ip.hR[id.row_off + k], &C0[i]);
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
  RowCosts rc{0, 0, 0, 0};
  int64_t c0 = 0;
  const int2* tk = tab + (int64_t)sub * (T + 1);
  int32_t* Ak = A + sub * T;
  Acc* Ck = C + sub * T;
  if (valid) {
    const int64_t ro = id.row_off + k;
    rc = RowCosts{p.ip.kM[ro], p.ip.kR[ro], p.ip.hM[ro], p.ip.hR[ro]};
    c0 = C0[sub];
    cur.b = p.bits[k];
    int b = T, dummy = 0;
    if (lane == 0) {
      cur.S = build_row<Acc>(tk, T, rc, cur.b, Ak, Ck, b, dummy);
      cur.bad = b;
    }
  }
  __syncwarp();
  {
    const int leader = wlane & ~(G - 1);
    cur.S = __shfl_sync(kFull, cur.S, leader);
    cur.bad = __shfl_sync(kFull, cur.bad, leader);
  }
  const int64_t rck = valid ? row_cost<Acc>(cur.S, c0) : 0;
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
      int sg = 0;
      const DeltaOut<Acc> d = eval_move<Acc, false>(tk, T, rc, cur, Ak, Ck, j, l, sg);
      const int64_t nc = row_cost<Acc>(d.S, c0);
      bestP = umin64(bestP, pack_key(nc, loff + (uint32_t)l));
      if (p.mode == 1) {
        const int64_t nt =
            (others == INT64_MAX || nc == INT64_MAX) ? INT64_MAX : others + nc;
        bestG = umin64(bestG, pack_key(nt, goff + (uint32_t)(k * M + l)));
      }
      if (j == p.single_j) {
        if (p.move_cost) p.move_cost[(int64_t)k * M + l] = nc;
        if (p.move_win) p.move_win[(int64_t)k * M + l] = sg;
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
// plan_kernel: one thread per row; xM, xR, yM, yR by the decode rule.
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

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_stage(const StageParams& p, int total_rows, cudaStream_t s) {
  if (total_rows <= 0) return cudaSuccess;
  const int threads = 256;
  int blocks = (total_rows * 32 + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  stage_kernel<<<blocks, threads, 0, s>>>(p);
  return cudaGetLastError();
}

size_t eval_smem_bytes(int rows, int T, bool acc64) {
  uint32_t o = align16((uint32_t)rows * (T + 1) * 8u);
  o = align16(o + rows * 8u);
  o = align16(o + (uint32_t)rows * T * 4u);
  o += (uint32_t)rows * T * (acc64 ? 8u : 4u);
  return o;
}

cudaError_t eval_prepare(bool acc64, size_t smem) {
  if (acc64)
    return cudaFuncSetAttribute(eval_kernel<int64_t>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaFuncSetAttribute(eval_kernel<int32_t>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_eval(const EvalParams& p, bool acc64, int blocks,
                        int threads, size_t smem, cudaStream_t s) {
  if (acc64)
    eval_kernel<int64_t><<<blocks, threads, smem, s>>>(p);
  else
    eval_kernel<int32_t><<<blocks, threads, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename Acc, bool TS>
static cudaError_t vns_prepare_t(size_t smem, int threads, int* bps) {
  cudaError_t e = cudaFuncSetAttribute(
      vns_kernel<Acc, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, vns_kernel<Acc, TS>,
                                                       threads, smem);
}

cudaError_t vns_prepare(bool acc64, bool tab_smem, size_t smem, int threads,
                        int* bps) {
  if (acc64)
    return tab_smem ? vns_prepare_t<int64_t, true>(smem, threads, bps)
                    : vns_prepare_t<int64_t, false>(smem, threads, bps);
  return tab_smem ? vns_prepare_t<int32_t, true>(smem, threads, bps)
                  : vns_prepare_t<int32_t, false>(smem, threads, bps);
}

cudaError_t launch_vns(const VnsParams& p, bool acc64, bool tab_smem,
                       int blocks, int threads, size_t smem, cudaStream_t s) {
  if (acc64) {
    if (tab_smem)
      vns_kernel<int64_t, true><<<blocks, threads, smem, s>>>(p);
    else
      vns_kernel<int64_t, false><<<blocks, threads, smem, s>>>(p);
  } else {
    if (tab_smem)
      vns_kernel<int32_t, true><<<blocks, threads, smem, s>>>(p);
    else
      vns_kernel<int32_t, false><<<blocks, threads, smem, s>>>(p);
  }
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
