// elsr_vns.cuh -- persistent GVNS kernel (Algorithm 2 around Algorithm 1's
// VND), included by the per-accumulator translation units.
//
// One run (instance, seed, budget) is executed by a team: the CTAs of one
// thread-block cluster (C >= 1 CTAs).  Product k belongs to CTA k mod C
// (local row q = k / C) and, inside it, to sub-warp q mod nsub (G lanes);
// that sub-warp stages, evaluates, applies, shakes and restores the row, so
// Algorithm 1's product loop needs no barrier between neighbourhoods.  The
// team synchronises once per VND sweep (the "improvement" flag, OR-reduced
// over the cluster through distributed shared memory) and once per GVNS
// iteration (the objective of x'').  Runs come from a device work queue.
// Everything a run touches after staging lives in shared memory, except the
// prefix tables of instances too large for it (TS = false: read from global
// memory through L1).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "elsr_internal.h"

namespace elsr {
namespace vns {

namespace cg = cooperative_groups;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

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
__device__ __forceinline__ void stage_row_warp(const int32_t* __restrict__ D,
                                               const int32_t* __restrict__ R, int T,
                                               int lane, int2* tab, int32_t hM,
                                               int32_t hR, int64_t* C0) {
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

// Shared-memory view of the rows a CTA owns in the current run.
template <typename Acc>
struct Rows {
  const int2* tab;   // TS: local rows [Kc][T+1]; else global table of row 0
  RowCosts* rc;
  int64_t* C0;
  RowBits* bits;
  Acc* S;
  int32_t* bad;
  int32_t* nR;
  int32_t* A;  // [Kc][T]
  Acc* C;      // [Kc][T]
  int2* L;     // [Kc][T]
  unsigned char* save;
  uint32_t slot;
  int T, C_, crank;
  bool ts;

  __device__ __forceinline__ const int2* tab_row(int q) const {
    const int64_t r = ts ? q : (int64_t)q * C_ + crank;
    return tab + r * (T + 1);
  }
  __device__ __forceinline__ RowState<Acc> state(int q) const {
    RowState<Acc> st;
    st.b = bits[q];
    st.S = S[q];
    st.bad = bad[q];
    st.nR = nR[q];
    return st;
  }
  __device__ __forceinline__ int64_t cost(int q) const { return row_cost<Acc>(S[q], C0[q]); }
  __device__ __forceinline__ unsigned char* slot_ptr(int par, int j) const {
    return save + (uint32_t)(par * kMaxShake + j) * slot;
  }
};

template <typename Acc>
__device__ __forceinline__ uint32_t slot_C_off(int T) {
  return 48u + (((uint32_t)T * 4u + 7u) & ~7u);
}
template <typename Acc>
__device__ __forceinline__ uint32_t slot_L_off(int T) {
  return slot_C_off<Acc>(T) + ((((uint32_t)T * (uint32_t)sizeof(Acc)) + 7u) & ~7u);
}

// Full rebuild of local row q's cache (one lane).
template <typename Acc, int NW>
__device__ __forceinline__ void rebuild(const Rows<Acc>& m, int q) {
  const int T = m.T;
  int b = T, nr = 0, dummy = 0;
  m.S[q] = build_row<Acc, NW>(m.tab_row(q), T, m.rc[q], m.bits[q], m.A + q * T,
                              m.C + q * T, m.L + q * T, b, nr, dummy);
  m.bad[q] = b;
  m.nR[q] = nr;
}

// Copy local row q to / from a save slot (sub-warp collective).
template <typename Acc>
__device__ __forceinline__ void save_row(const Rows<Acc>& m, int q, unsigned char* sl,
                                         int lane, int G) {
  const int T = m.T;
  int32_t* sA = (int32_t*)(sl + 48);
  Acc* sC = (Acc*)(sl + slot_C_off<Acc>(T));
  int2* sL = (int2*)(sl + slot_L_off<Acc>(T));
  const int nr = m.nR[q];
  for (int s = lane; s < T; s += G) {
    sA[s] = m.A[q * T + s];
    sC[s] = m.C[q * T + s];
    if (s < nr) sL[s] = m.L[q * T + s];
  }
  if (lane == 0) {
    *(RowBits*)sl = m.bits[q];
    *(int64_t*)(sl + 32) = (int64_t)m.S[q];
    *(int32_t*)(sl + 40) = m.bad[q];
    *(int32_t*)(sl + 44) = nr;
  }
}

template <typename Acc>
__device__ __forceinline__ void restore_row(const Rows<Acc>& m, int q,
                                            const unsigned char* sl, int lane, int G) {
  const int T = m.T;
  const int32_t* sA = (const int32_t*)(sl + 48);
  const Acc* sC = (const Acc*)(sl + slot_C_off<Acc>(T));
  const int2* sL = (const int2*)(sl + slot_L_off<Acc>(T));
  const int nr = *(const int32_t*)(sl + 44);
  for (int s = lane; s < T; s += G) {
    m.A[q * T + s] = sA[s];
    m.C[q * T + s] = sC[s];
    if (s < nr) m.L[q * T + s] = sL[s];
  }
  if (lane == 0) {
    m.bits[q] = *(const RowBits*)sl;
    m.S[q] = (Acc)(*(const int64_t*)(sl + 32));
    m.bad[q] = *(const int32_t*)(sl + 40);
    m.nR[q] = nr;
  }
}

// Best move (packed (row cost, local index) key) of local row q in N_j over
// this lane's share of the candidates.
template <typename Acc, int NW>
__device__ __forceinline__ uint64_t row_best(const Rows<Acc>& m, int q,
                                             const RowState<Acc>& cur, int j, int M,
                                             int lane, int G, uint32_t& steps) {
  const int T = m.T;
  const int2* tk = m.tab_row(q);
  const int32_t* Aq = m.A + q * T;
  const Acc* Cq = m.C + q * T;
  const int2* Lq = m.L + q * T;
  const RowCosts rc = m.rc[q];
  const int64_t c0 = m.C0[q];
  uint64_t best = ~0ull;
  int st = 0;
  for (int l = lane; l < M; l += G) {
    const Acc S = eval_move<Acc, NW>(tk, T, rc, cur, Aq, Cq, Lq, j, l, st);
    best = umin64(best, pack_key(row_cost<Acc>(S, c0), (uint32_t)l));
  }
  steps += (uint32_t)st;
  return best;
}

// Team-wide barrier: the CTA, or the whole cluster.
__device__ __forceinline__ void team_sync(int C) {
  if (C == 1) {
    __syncthreads();
  } else {
    cg::this_cluster().sync();
  }
}

template <typename Acc, int NW, bool TS, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) vns_kernel(const VnsParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int sh_run;
  __shared__ unsigned long long sh_acc[2];
  __shared__ int sh_ninf[2];
  __shared__ int sh_flag[2];
  __shared__ unsigned long long sh_gkey[2];
  __shared__ long long sh_F;
  __shared__ int sh_Finf;
  __shared__ unsigned long long sh_applied, sh_steps;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = p.G;
  const int lane = tid & (G - 1), sub = tid / G, nsub = nthr / G;
  const int wlane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();

  for (;;) {
    if (crank == 0 && tid == 0) sh_run = atomicAdd(p.queue, 1);
    team_sync(C);
    const int r = C == 1 ? sh_run : *cl.map_shared_rank(&sh_run, 0);
    team_sync(C);
    if (r >= p.nruns) return;
    const RunDesc rd = p.runs[r];
    const InstDesc id = p.ip.insts[rd.inst];
    const int K = id.K, T = id.T;
    const int Kc = (K - crank + C - 1) / C;  // rows owned by this CTA
    const int Kmax = (K + C - 1) / C;
    const VnsLayout Lay = vns_layout(Kmax, T, (int)sizeof(Acc), TS);
    Rows<Acc> m;
    m.tab = TS ? (const int2*)(smem + Lay.tab) : (p.ip.gtab + id.tab_off);
    m.rc = (RowCosts*)(smem + Lay.rc);
    m.C0 = (int64_t*)(smem + Lay.C0);
    m.bits = (RowBits*)(smem + Lay.bits);
    m.S = (Acc*)(smem + Lay.S);
    m.bad = (int32_t*)(smem + Lay.bad);
    m.nR = (int32_t*)(smem + Lay.nR);
    m.A = (int32_t*)(smem + Lay.A);
    m.C = (Acc*)(smem + Lay.C);
    m.L = (int2*)(smem + Lay.L);
    m.save = smem + Lay.save;
    m.slot = Lay.slot;
    m.T = T;
    m.C_ = C;
    m.crank = crank;
    m.ts = TS;

    // ---- stage this CTA's rows (one warp per row) ----
    for (int q = warp; q < Kc; q += nwarps) {
      const int k = q * C + crank;
      const int64_t ro = id.row_off + k;
      if (TS) {
        stage_row_warp(p.ip.D + id.cell_off + (int64_t)k * T,
                       p.ip.R + id.cell_off + (int64_t)k * T, T, wlane,
                       (int2*)(smem + Lay.tab) + (int64_t)q * (T + 1), p.ip.hM[ro],
                       p.ip.hR[ro], &m.C0[q]);
      } else if (wlane == 0) {
        m.C0[q] = p.ip.gC0[ro];
      }
      if (wlane == 0) {
        m.rc[q] = RowCosts{p.ip.kM[ro], p.ip.kR[ro], p.ip.hM[ro], p.ip.hR[ro]};
        m.bits[q] = rd.start_off >= 0 ? p.start_bits[rd.start_off + k] : all_open(T);
      }
    }
    if (tid == 0) {
      sh_acc[0] = sh_acc[1] = 0ull;
      sh_ninf[0] = sh_ninf[1] = 0;
      sh_flag[0] = sh_flag[1] = 0;
      sh_gkey[0] = sh_gkey[1] = ~0ull;
      sh_applied = 0ull;
      sh_steps = 0ull;
    }
    __syncthreads();
    if (lane == 0)
      for (int q = sub; q < Kc; q += nsub) rebuild<Acc, NW>(m, q);
    __syncwarp();

    uint32_t my_steps = 0, my_applied = 0;
    const int Kcr = ((Kc + nsub - 1) / nsub) * nsub;  // uniform row-loop bound
    const int64_t moves_per_cycle = (int64_t)K * (2 * T + (T > 1 ? 2 * (T - 1) : 0));
    int status = 0;
    int64_t cycles_total = 0;
    int tp = 0, fp = 0;

    // ---- saturating objective of the team (sum of row costs) ----
    auto team_total = [&]() -> int64_t {
      if (lane == 0) {
        int64_t s = 0;
        int ni = 0;
        for (int q = sub; q < Kc; q += nsub) {
          const int64_t c = m.cost(q);
          if (c == INT64_MAX) ++ni; else s += c;
        }
        if (s) atomicAdd(&sh_acc[tp], (unsigned long long)s);
        if (ni) atomicAdd(&sh_ninf[tp], ni);
      }
      __syncthreads();
      int64_t tot;
      if (C == 1) {
        tot = sh_ninf[tp] ? INT64_MAX : (int64_t)sh_acc[tp];
      } else {
        cl.sync();
        unsigned long long a = 0;
        int ni = 0;
        if (wlane < C) {
          a = *cl.map_shared_rank(&sh_acc[tp], wlane);
          ni = *cl.map_shared_rank(&sh_ninf[tp], wlane);
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(kFull, a, o);
          ni += __shfl_xor_sync(kFull, ni, o);
        }
        tot = ni ? INT64_MAX : (int64_t)a;
      }
      if (tid == 0) {
        sh_acc[tp ^ 1] = 0ull;
        sh_ninf[tp ^ 1] = 0;
      }
      tp ^= 1;
      return tot;
    };

    // ---- VND, mode P (Algorithm 1): every product takes its best strictly
    // improving move of N_j; repeat the j = 1..3 sweep until no product of
    // the team improves.  Returns the sweeps run, or -1 at the cap. ----
    auto vnd_p = [&]() -> int {
      int cycles = 0;
      for (;;) {
        int improved = 0;
        for (int j = 1; j <= 3; ++j) {
          const int M = row_moves(T, j);
          if (M <= 0) continue;
          for (int qq = sub; qq < Kcr; qq += nsub) {
            const bool valid = qq < Kc;
            const int q = valid ? qq : 0;
            uint64_t best = ~0ull;
            if (valid) {
              const RowState<Acc> cur = m.state(q);
              best = row_best<Acc, NW>(m, q, cur, j, M, lane, G, my_steps);
            }
            best = subwarp_min(best, G);
            const bool imp = valid && key_cost(best) < m.cost(q);
            if (imp && lane == 0) {
              RowBits nb = m.bits[q];
              apply_row_move(nb, T, j, key_index(best));
              m.bits[q] = nb;
              rebuild<Acc, NW>(m, q);
              ++my_applied;
            }
            __syncwarp();
            improved |= imp;
          }
        }
        ++cycles;
        int any = __syncthreads_or(improved);
        if (C > 1) {
          if (tid == 0) sh_flag[fp] = any;
          cl.sync();
          const int v = wlane < C ? *cl.map_shared_rank(&sh_flag[fp], wlane) : 0;
          any = __any_sync(kFull, v);
          fp ^= 1;
        }
        if (!any) break;
        if (cycles >= p.vnd_cap) return -1;
      }
      return cycles;
    };

    // ---- VND, mode G (single CTA teams): one best move of the whole
    // neighbourhood by (new objective, global index), applied when it
    // lowers the objective. ----
    auto vnd_g = [&]() -> int {
      if (tid == 0) {
        sh_F = 0;
        sh_Finf = 0;
        sh_gkey[0] = sh_gkey[1] = ~0ull;
      }
      __syncthreads();
      if (lane == 0) {
        long long s = 0;
        int ni = 0;
        for (int q = sub; q < Kc; q += nsub) {
          const int64_t c = m.cost(q);
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
          for (int qq = sub; qq < Kcr; qq += nsub) {
            const bool valid = qq < Kc;
            const int q = valid ? qq : 0;
            uint64_t best = ~0ull;
            if (valid) {
              const RowState<Acc> cur = m.state(q);
              const int64_t rck = m.cost(q);
              const int infk = rck == INT64_MAX;
              const int64_t others = (Finf - infk > 0) ? INT64_MAX : F - (infk ? 0 : rck);
              const int2* tk = m.tab_row(q);
              const RowCosts rc = m.rc[q];
              const int64_t c0 = m.C0[q];
              int st = 0;
              for (int l = lane; l < M; l += G) {
                const Acc S = eval_move<Acc, NW>(tk, T, rc, cur, m.A + q * T, m.C + q * T,
                                                 m.L + q * T, j, l, st);
                const int64_t nc = row_cost<Acc>(S, c0);
                const int64_t nt =
                    (others == INT64_MAX || nc == INT64_MAX) ? INT64_MAX : others + nc;
                best = umin64(best, pack_key(nt, (uint32_t)(q * M + l)));
              }
              my_steps += (uint32_t)st;
            }
            best = subwarp_min(best, G);
            if (valid && lane == 0 && best != ~0ull) atomicMin(&sh_gkey[e], best);
          }
          __syncthreads();
          const uint64_t gk = sh_gkey[e];
          if (tid == 0) sh_gkey[e ^ 1] = ~0ull;
          if (gk != ~0ull && key_cost(gk) < total) {
            const int gi = key_index(gk);
            const int qw = gi / M, lw = gi - qw * M;
            if ((qw % nsub) == sub && lane == 0) {
              const int64_t old = m.cost(qw);
              RowBits nb = m.bits[qw];
              apply_row_move(nb, T, j, lw);
              m.bits[qw] = nb;
              rebuild<Acc, NW>(m, qw);
              const int64_t nw = m.cost(qw);
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

    // ---- initial VND and GVNS (Algorithm 2) ----
    int cyc = rd.mode == 0 ? vnd_p() : vnd_g();
    if (cyc < 0) status = kStatusCap; else cycles_total += cyc;
    int64_t fx = team_total();
    int kk = 1;  // neighbourhood index k of Algorithm 2
    uint64_t h = 0;
    int64_t iters_done = 0, accepted = 0;
    const bool log = rd.traj_off >= 0 && crank == 0;
    for (int it = 0; it < rd.iters && status == 0; ++it) {
      const int par = it & 1;
      const int ks = kk;
      // Shake(x, k): k moves of N_k from splitmix64 draws, applied by the
      // owners of the hit rows; the first touch saves the row so that a
      // rejected x'' can be undone.
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
          for (int q2 = 0; q2 < j; ++q2)
            if (rows[q2] == rows[j]) first[j] = false;
        }
      }
#pragma unroll
      for (int j = 0; j < kMaxShake; ++j) {
        const int k = rows[j];
        const bool mine = k >= 0 && (k % C) == crank && ((k / C) % nsub) == sub;
        if (mine && first[j]) save_row<Acc>(m, k / C, m.slot_ptr(par, j), lane, G);
        __syncwarp();
        if (mine && lane == 0) {
          RowBits b = m.bits[k / C];
          apply_row_move(b, T, ks, locs[j]);
          m.bits[k / C] = b;
        }
        __syncwarp();
      }
      if (lane == 0) {
#pragma unroll
        for (int j = 0; j < kMaxShake; ++j) {
          const int k = rows[j];
          if (k >= 0 && first[j] && (k % C) == crank && ((k / C) % nsub) == sub)
            rebuild<Acc, NW>(m, k / C);
        }
      }
      __syncwarp();
      // VND(x')
      cyc = rd.mode == 0 ? vnd_p() : vnd_g();
      if (cyc < 0) status = kStatusCap; else cycles_total += cyc;
      const int64_t f2 = team_total();
      const int acc = f2 < fx;
      if (tid == 0 && crank == 0) {
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
        kk = 1;
        ++accepted;
      } else {
        // x'' rejected: the shaken rows go back to x; the other rows never
        // moved, being locally optimal in x.
#pragma unroll
        for (int j = 0; j < kMaxShake; ++j) {
          const int k = rows[j];
          const bool mine = k >= 0 && first[j] && (k % C) == crank && ((k / C) % nsub) == sub;
          if (mine) restore_row<Acc>(m, k / C, m.slot_ptr(par, j), lane, G);
          __syncwarp();
        }
        kk = kk % rd.kmax + 1;
      }
      if ((it & 255) == 255) {  // keep the 32-bit per-thread counters small
        unsigned long long v = my_steps;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (wlane == 0 && v) atomicAdd(&sh_steps, v);
        my_steps = 0;
      }
    }

    // ---- outputs ----
    for (int q = tid; q < Kc; q += nthr) p.out_bits[rd.bits_off + q * C + crank] = m.bits[q];
    {
      unsigned long long v = my_steps, a = my_applied;
      for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(kFull, v, o);
        a += __shfl_xor_sync(kFull, a, o);
      }
      if (wlane == 0) {
        if (v) atomicAdd(&sh_steps, v);
        if (a) atomicAdd(&sh_applied, a);
      }
    }
    team_sync(C);
    if (tid == 0 && crank == 0) {
      unsigned long long steps = 0, applied = 0;
      for (int c = 0; c < C; ++c) {
        steps += C == 1 ? sh_steps : *cl.map_shared_rank(&sh_steps, c);
        applied += C == 1 ? sh_applied : *cl.map_shared_rank(&sh_applied, c);
      }
      RunOut o;
      o.best_cost = fx;
      o.traj_hash = h;
      o.moves_evaluated = cycles_total * moves_per_cycle;
      o.evals = cycles_total * 3;
      o.vnd_cycles = cycles_total;
      o.applied = (int64_t)applied;
      o.iterations = iters_done;
      o.accepted = accepted;
      o.segments = (int64_t)steps;
      o.status = status;
      o.reserved = 0;
      p.out[rd.out] = o;
    }
    team_sync(C);
  }
}

}  // namespace vns

template <typename Acc, int NW, bool TS, int MAXT>
cudaError_t vns_prepare_t(size_t smem, int threads, int cluster, int* active) {
  auto kern = vns::vns_kernel<Acc, NW, TS, MAXT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  if (cluster <= 1)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(active, kern, threads, smem);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(active, kern, &cfg);
}

template <typename Acc, int NW, bool TS, int MAXT>
cudaError_t vns_launch_t(const VnsParams& p, int blocks, int threads, size_t smem,
                         int cluster, cudaStream_t s) {
  auto kern = vns::vns_kernel<Acc, NW, TS, MAXT>;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster < 1 ? 1 : cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = cluster > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

}  // namespace elsr
