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

#include <type_traits>

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
// constant C0 = hR * sum R(t)(T-t) - hM * sum D(t)(T-t) + pM * sum D.
// Fresh: load through L2 only (ld.global.cg), for data the host may have
// rewritten while the kernel was resident (the read-only and L1 paths are
// not kept coherent with such writes).
template <bool Fresh = false>
__device__ __forceinline__ int32_t ld_in(const int32_t* p) {
  return Fresh ? __ldcg(p) : __ldg(p);
}

// Four consecutive periods t0 .. t0+3 of a row of T values (0 outside the
// row): one 16-byte load when the four lie in the row and start on a 16-byte
// boundary, else one load per period inside the row.
template <bool Fresh>
__device__ __forceinline__ void load4(const int32_t* __restrict__ row, int T, int t0,
                                      int32_t v[4]) {
  const int32_t* p = row + t0;
  if (t0 >= 0 && t0 + 3 < T && ((uintptr_t)p & 15u) == 0) {
    const int4 q = Fresh ? __ldcg((const int4*)p) : __ldg((const int4*)p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = (t0 + j >= 0 && t0 + j < T) ? ld_in<Fresh>(p + j) : 0;
  }
}

// Stage one row with a full warp: tab[0..T] = {CD[j], CR1[j]} and the row
// constant C0 = hR * sum R(t)(T-t) - hM * sum D(t)(T-t) + pM * sum D.  Lane w
// takes the four periods of the w-th 16-byte window of D's row (from the
// window holding period 0), so its loads are vector loads except at the
// row's ends; a per-lane scan of its four values and a warp scan of the lane
// totals give the prefix sums.  R's row is read at the same periods.
template <bool Fresh = false>
__device__ __forceinline__ void stage_row_warp(const int32_t* __restrict__ D,
                                               const int32_t* __restrict__ R, int T,
                                               int lane, int2* tab, int32_t hM,
                                               int32_t hR, int32_t pM, int64_t* C0) {
  const int mis = (int)(((uintptr_t)D >> 2) & 3u);  // periods before D's first window
  int32_t carryD = 0, carryR = 0;
  int64_t wd = 0, wr = 0;
  for (int base = -mis; base < T; base += 128) {
    const int t0 = base + 4 * lane;
    int32_t d[4], r[4];
    load4<Fresh>(D, T, t0, d);
    load4<Fresh>(R, T, t0, r);
    int32_t sd = 0, sr = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + j;
      wd += (int64_t)d[j] * (T - t);  // 0 outside the row
      wr += (int64_t)r[j] * (T - t);
      sd += d[j];
      sr += r[j];
      d[j] = sd;  // inclusive sums within the lane
      r[j] = sr;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t a = __shfl_up_sync(kFull, sd, o);
      const int32_t b = __shfl_up_sync(kFull, sr, o);
      if (lane >= o) {
        sd += a;
        sr += b;
      }
    }
    const int32_t offD = carryD + sd - d[3], offR = carryR + sr - r[3];  // before this lane
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + j;
      if (t >= 0 && t < T) {
        tab[t + 1].x = offD + d[j];  // CD[t+1]
        tab[t].y = offR + r[j];      // CR1[t]
      }
    }
    carryD += __shfl_sync(kFull, sd, 31);
    carryR += __shfl_sync(kFull, sr, 31);
  }
  wd = warp_sum64(wd);
  wr = warp_sum64(wr);
  if (lane == 0) {
    tab[0].x = 0;
    tab[T].y = carryR;
    *C0 = (int64_t)hR * wr - (int64_t)hM * wd + (int64_t)pM * carryD;
  }
}

// Costs of pool row ro (unit production costs 0 when the pools have none).
template <bool Fresh = false>
__device__ __forceinline__ RowCosts row_costs(const InstPools& ip, int64_t ro) {
  const int32_t pm = ip.pM ? ld_in<Fresh>(ip.pM + ro) : 0;
  const int32_t pr = ip.pR ? ld_in<Fresh>(ip.pR + ro) : 0;
  return RowCosts{ld_in<Fresh>(ip.kM + ro), ld_in<Fresh>(ip.kR + ro), ld_in<Fresh>(ip.hM + ro),
                  ld_in<Fresh>(ip.hR + ro), pr - pm};
}

__device__ __forceinline__ InstDesc ldcg_inst(const InstDesc* d) {
  static_assert(sizeof(InstDesc) == 32, "InstDesc is four 64-bit words");
  InstDesc o;
  unsigned long long* w = (unsigned long long*)&o;
  const unsigned long long* s = (const unsigned long long*)d;
#pragma unroll
  for (int i = 0; i < 4; ++i) w[i] = __ldcg(s + i);
  return o;
}

// The kernel's dynamic shared memory (every extern __shared__ array of a
// kernel starts at the same address).
extern __shared__ __align__(16) unsigned char dyn_smem[];

// Shared-memory view of the rows a CTA owns in the current run.  The arrays
// are held as 32-bit offsets into dynamic shared memory (one register each).
template <typename Acc>
struct Rows {
  const int2* tab;   // TS: local rows [Kc][T+1]; else global table of row 0
  uint32_t o_rc, o_C0, o_bits, o_S, o_mark, o_nR, o_A, o_C, o_L, o_P, o_Q, o_save;
  uint32_t slot;
  int T, C_, crank;
  bool ts;

  __device__ __forceinline__ RowCosts* rc() const { return (RowCosts*)(dyn_smem + o_rc); }
  __device__ __forceinline__ int64_t* C0() const { return (int64_t*)(dyn_smem + o_C0); }
  __device__ __forceinline__ RowBits* bits() const { return (RowBits*)(dyn_smem + o_bits); }
  __device__ __forceinline__ Acc* S() const { return (Acc*)(dyn_smem + o_S); }
  __device__ __forceinline__ RowMark* mark() const { return (RowMark*)(dyn_smem + o_mark); }
  __device__ __forceinline__ int32_t* nR() const { return (int32_t*)(dyn_smem + o_nR); }
  __device__ __forceinline__ int32_t* A() const { return (int32_t*)(dyn_smem + o_A); }
  __device__ __forceinline__ Acc* C() const { return (Acc*)(dyn_smem + o_C); }
  __device__ __forceinline__ int2* L() const { return (int2*)(dyn_smem + o_L); }
  __device__ __forceinline__ int32_t* P() const { return (int32_t*)(dyn_smem + o_P); }
  __device__ __forceinline__ Acc* Q() const { return (Acc*)(dyn_smem + o_Q); }
  __device__ __forceinline__ unsigned char* save() const { return dyn_smem + o_save; }
  // place the arrays at byte offsets of the region starting at base
  __device__ __forceinline__ void place(unsigned char* base, uint32_t rc_, uint32_t C0_,
                                        uint32_t bits_, uint32_t S_, uint32_t mark_,
                                        uint32_t nR_, uint32_t A_, uint32_t C_a, uint32_t L_,
                                        uint32_t P_, uint32_t Q_, uint32_t save_) {
    const uint32_t b = (uint32_t)(base - dyn_smem);
    o_rc = b + rc_; o_C0 = b + C0_; o_bits = b + bits_; o_S = b + S_; o_mark = b + mark_;
    o_nR = b + nR_; o_A = b + A_; o_C = b + C_a; o_L = b + L_; o_P = b + P_; o_Q = b + Q_;
    o_save = b + save_;
  }

  __device__ __forceinline__ const int2* tab_row(int q) const {
    const int64_t r = ts ? q : (int64_t)q * C_ + crank;
    return tab + r * (T + 1);
  }
  __device__ __forceinline__ RowState<Acc> state(int q) const {
    RowState<Acc> st;
    st.b = bits()[q];
    st.S = S()[q];
    const RowMark mk = mark()[q];
    st.bad = mk.bad;
    st.ld = mk.ld;
    st.nR = nR()[q];
    return st;
  }
  __device__ __forceinline__ int64_t cost(int q) const {
    return state_cost<Acc>(S()[q], mark()[q].bad, T, C0()[q]);
  }
  __device__ __forceinline__ unsigned char* slot_ptr(int par, int j) const {
    return save() + (uint32_t)(par * kMaxShake + j) * slot;
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
template <typename Acc>
__device__ __forceinline__ uint32_t slot_P_off(int T) {
  return slot_L_off<Acc>(T) + (uint32_t)T * 8u;
}
template <typename Acc>
__device__ __forceinline__ uint32_t slot_Q_off(int T) {
  return slot_P_off<Acc>(T) + ((((uint32_t)T + 1u) * 4u + 7u) & ~7u);
}

// Copy local row q to / from a save slot (sub-warp collective).
template <typename Acc>
__device__ __forceinline__ void save_row(const Rows<Acc>& m, int q, unsigned char* sl,
                                         int lane, int G) {
  const int T = m.T;
  int32_t* sA = (int32_t*)(sl + 48);
  Acc* sC = (Acc*)(sl + slot_C_off<Acc>(T));
  int2* sL = (int2*)(sl + slot_L_off<Acc>(T));
  int32_t* sP = (int32_t*)(sl + slot_P_off<Acc>(T));
  Acc* sQ = (Acc*)(sl + slot_Q_off<Acc>(T));
  const int nr = m.nR()[q];
  for (int s = lane; s < T; s += G) {
    sA[s] = m.A()[q * T + s];
    sC[s] = m.C()[q * T + s];
    if (s < nr) sL[s] = m.L()[q * T + s];
  }
  for (int s = lane; s <= nr; s += G) {
    sP[s] = m.P()[q * (T + 1) + s];
    sQ[s] = m.Q()[q * (T + 1) + s];
  }
  if (lane == 0) {
    *(RowBits*)sl = m.bits()[q];
    *(int64_t*)(sl + 32) = (int64_t)m.S()[q];
    *(RowMark*)(sl + 40) = m.mark()[q];
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
  const int32_t* sP = (const int32_t*)(sl + slot_P_off<Acc>(T));
  const Acc* sQ = (const Acc*)(sl + slot_Q_off<Acc>(T));
  const int nr = *(const int32_t*)(sl + 44);
  for (int s = lane; s < T; s += G) {
    m.A()[q * T + s] = sA[s];
    m.C()[q * T + s] = sC[s];
    if (s < nr) m.L()[q * T + s] = sL[s];
  }
  for (int s = lane; s <= nr; s += G) {
    m.P()[q * (T + 1) + s] = sP[s];
    m.Q()[q * (T + 1) + s] = sQ[s];
  }
  if (lane == 0) {
    m.bits()[q] = *(const RowBits*)sl;
    m.S()[q] = (Acc)(*(const int64_t*)(sl + 32));
    m.mark()[q] = *(const RowMark*)(sl + 40);
    m.nR()[q] = nr;
  }
}

// Best move (packed (row cost, local index) key) of local row q in N_j over
// this lane's share of the candidates; Count: add their decode steps.
template <typename Acc, int NW, bool Count>
__device__ __forceinline__ uint64_t row_best(const Rows<Acc>& m, int q,
                                             const RowState<Acc>& cur, int j, int M,
                                             int lane, int G, uint32_t& steps) {
  const int T = m.T;
  const int2* tk = m.tab_row(q);
  const int32_t* Aq = m.A() + q * T;
  const Acc* Cq = m.C() + q * T;
  const int2* Lq = m.L() + q * T;
  const int32_t* Pq = m.P() + q * (T + 1);
  const Acc* Qq = m.Q() + q * (T + 1);
  const RowCosts rc = m.rc()[q];
  const int64_t c0 = m.C0()[q];
  uint64_t best = ~0ull;
  int st = 0;
  if (j == 3) {
    // only the swaps that change the row can improve it; lanes take them
    // by rank (null swaps keep the row's cost and never win)
    const SwapMasks sw = swap_masks<NW>(cur.b, T);
    for (int i = lane; i < sw.n; i += G) {
      const int l = swap_of_rank<NW>(sw, T, i);
      const Acc S = eval_move<Acc, NW, Count>(tk, T, rc, cur, Aq, Cq, Lq, Pq, Qq, 3, l, st);
      best = umin64(best, pack_key(row_cost<Acc>(S, c0), (uint32_t)l));
    }
  } else {
    for (int l = lane; l < M; l += G) {
      const Acc S = eval_move<Acc, NW, Count>(tk, T, rc, cur, Aq, Cq, Lq, Pq, Qq, j, l, st);
      best = umin64(best, pack_key(row_cost<Acc>(S, c0), (uint32_t)l));
    }
  }
  if constexpr (Count) steps += (uint32_t)st;
  return best;
}

// ---------------------------------------------------------------------------
// Lane-parallel rebuild of one row's cache (sub-warp collective).
//
// The recoverable stock follows y(t) = F_t(y(t-1)), y(-1) = 0, with
//   F_t(y) = max(y + R(t) - need(t), 0)   at a gR setup (xR = min(avail, need))
//   F_t(y) = y + R(t)                     elsewhere,
// all of the form F(y) = max(y + p, q).  Such functions compose associatively,
//   (F2 o F1)(y) = max(y + p1 + p2, max(q1 + p2, q2)),
// so each lane composes its run of periods, a sub-warp scan hands every lane
// the stock entering its periods, and each lane then fills A, the local part
// of C and its gR-list entries; a second scan offsets C.
// ---------------------------------------------------------------------------
constexpr int64_t kNegInf = -(1ll << 62);

template <typename Acc, int NW>
__device__ __forceinline__ void rebuild_row(const Rows<Acc>& m, int q, int lane, int G,
                                            unsigned smask) {
  const int T = m.T;
  const int2* tab = m.tab_row(q);
  const RowBits b = m.bits()[q];
  const RowCosts rc = m.rc()[q];
  const uint64_t u0 = b.m0 | b.r0, u1 = b.m1 | b.r1;
  int32_t* A = m.A() + q * T;
  Acc* C = m.C() + q * T;
  int2* L = m.L() + q * T;
  int32_t* Pr = m.P() + q * (T + 1);
  Acc* Qr = m.Q() + q * (T + 1);
  const int P = (T + G - 1) / G;
  const int a = lane * P, e = a + P < T ? a + P : T;
  // phase 1: composition of this lane's period functions
  int64_t fp = 0, fq = kNegInf;
  for (int t = a; t < e; ++t) {
    const int2 tt = tab[t];
    const int32_t Rt = tt.y - (t > 0 ? tab[t - 1].y : 0);
    int64_t pt = Rt, qt = kNegInf;
    if (bitat<NW>(b.r0, b.r1, t)) {
      const int n = nxt<NW>(u0, u1, t, T);
      pt = (int64_t)Rt - (int64_t)(tab[n].x - tt.x);
      qt = 0;
    }
    fq = (fq + pt > qt) ? fq + pt : qt;
    fp += pt;
  }
  // phase 2: exclusive scan of the compositions in lane order
  for (int o = 1; o < G; o <<= 1) {
    const int64_t pp = __shfl_up_sync(smask, fp, o, G);
    const int64_t qq = __shfl_up_sync(smask, fq, o, G);
    if (lane >= o) {
      const int64_t nq = qq + fp;
      fq = nq > fq ? nq : fq;
      fp += pp;
    }
  }
  int64_t ep = __shfl_up_sync(smask, fp, 1, G);
  int64_t eq = __shfl_up_sync(smask, fq, 1, G);
  if (lane == 0) {
    ep = 0;
    eq = kNegInf;
  }
  int64_t y = ep > eq ? ep : eq;  // stock entering period a
  // phase 3: cache entries with local prefix sums
  Acc lsum = 0, lwroom = 0;
  int32_t lroom = 0;
  int first_bad = T, last_def = -1;
  const int r_begin = rank_below<NW>(b.r0, b.r1, a);
  int r = r_begin;
  for (int t = a; t < e; ++t) {
    const int2 tt = tab[t];
    const int32_t Rt = tt.y - (t > 0 ? tab[t - 1].y : 0);
    const int32_t avail = (int32_t)(y + Rt);
    if (bit_of(u0, u1, t)) {
      const int n = nxt<NW>(u0, u1, t, T);
      const int32_t need = tab[n].x - tt.x;
      const int gm = bitat<NW>(b.m0, b.m1, t), gr = bitat<NW>(b.r0, b.r1, t);
      const int32_t xr = gr ? (avail < need ? avail : need) : 0;
      if (!gm && xr < need) {  // deficit, taken as manufactured (relaxed decode)
        if (first_bad == T) first_bad = t;
        last_def = r;
      }
      A[t] = avail;
      C[t] = lsum;
      lsum += (Acc)(gm ? rc.kM : 0) + (Acc)(gr ? rc.kR : 0) +
              ((Acc)rc.hM * (Acc)need - (Acc)rc.hR * (Acc)xr) * (Acc)(T - t) +
              (Acc)rc.dP * (Acc)xr;
      if (gr) {
        int2 en;
        en.x = avail - need;
        en.y = t | (gm << 16);
        L[r] = en;
        Pr[r] = lroom;
        Qr[r] = lwroom;
        const int32_t room = need > avail ? need - avail : 0;
        lroom += room;
        lwroom += xr_weight<Acc>(rc, T, t) * (Acc)room;
        ++r;
      }
      y = avail - xr;
    } else {
      y = avail;
    }
  }
  // phase 4: offsets of C, P, Q; first shortfall; totals
  Acc off = lsum, offQ = lwroom;
  int32_t offP = lroom;
  for (int o = 1; o < G; o <<= 1) {
    const Acc v = __shfl_up_sync(smask, off, o, G);
    const Acc vq = __shfl_up_sync(smask, offQ, o, G);
    const int32_t vp = __shfl_up_sync(smask, offP, o, G);
    if (lane >= o) {
      off += v;
      offQ += vq;
      offP += vp;
    }
  }
  const Acc total = __shfl_sync(smask, off, G - 1, G);
  const Acc totQ = __shfl_sync(smask, offQ, G - 1, G);
  const int32_t totP = __shfl_sync(smask, offP, G - 1, G);
  off -= lsum;
  offQ -= lwroom;
  offP -= lroom;
  for (int i = r_begin; i < r; ++i) {
    Pr[i] += offP;
    Qr[i] += offQ;
  }
  for (int o = G >> 1; o > 0; o >>= 1) {
    const int v = __shfl_xor_sync(smask, first_bad, o, G);
    const int w = __shfl_xor_sync(smask, last_def, o, G);
    first_bad = v < first_bad ? v : first_bad;
    last_def = w > last_def ? w : last_def;
  }
  if (off != 0)
    for (int t = a; t < e; ++t)
      if (bit_of(u0, u1, t)) C[t] += off;
  if (lane == 0) {
    const int f = nxt<NW>(u0, u1, -1, T);
    int bad = first_bad;
    if (tab[f].x != 0) bad = -1;  // demand before the first setup
    RowMark mk;
    mk.bad = (int16_t)bad;
    mk.ld = (int16_t)last_def;
    m.mark()[q] = mk;
    m.S()[q] = total;
    const int nr = popc64(b.r0) + (NW == 1 ? 0 : popc64(b.r1));
    m.nR()[q] = nr;
    Pr[nr] = totP;
    Qr[nr] = totQ;
  }
}

// Two-pass variant of rebuild_row for lanes holding at most PM periods: the
// first pass keeps each period's returns, need and setup bits in registers,
// so the second pass writes every cache entry once, with its offsets, and
// reads no table entry again.  Same results as rebuild_row.
template <typename Acc, int NW, int PM>
__device__ __forceinline__ void rebuild_row_regs(const Rows<Acc>& m, int q, int lane, int G,
                                                 unsigned smask) {
  const int T = m.T;
  const int2* tab = m.tab_row(q);
  const RowBits b = m.bits()[q];
  const RowCosts rc = m.rc()[q];
  const uint64_t u0 = b.m0 | b.r0, u1 = b.m1 | b.r1;
  int32_t* A = m.A() + q * T;
  Acc* C = m.C() + q * T;
  int2* L = m.L() + q * T;
  int32_t* Pr = m.P() + q * (T + 1);
  Acc* Qr = m.Q() + q * (T + 1);
  const int P = (T + G - 1) / G;
  const int a = lane * P, e = a + P < T ? a + P : T;
  // the first setup and the demand before it (lane 0 uses them last)
  const int f = nxt<NW>(u0, u1, -1, T);
  const int32_t dfirst = tab[f].x;
  int32_t Rt[PM], need[PM];
  int kind[PM];  // bit 0: setup, bit 1: gM, bit 2: gR
  int64_t fp = 0, fq = kNegInf;
#pragma unroll
  for (int i = 0; i < PM; ++i) {
    const int t = a + i;
    Rt[i] = 0;
    need[i] = 0;
    kind[i] = 0;
    if (t < e) {
      const int2 tt = tab[t];
      Rt[i] = tt.y - (t > 0 ? tab[t - 1].y : 0);
      const int gm = bitat<NW>(b.m0, b.m1, t), gr = bitat<NW>(b.r0, b.r1, t);
      kind[i] = (gm | gr) | (gm << 1) | (gr << 2);
      if (gm | gr) need[i] = tab[nxt<NW>(u0, u1, t, T)].x - tt.x;
      const int64_t pt = gr ? (int64_t)Rt[i] - (int64_t)need[i] : (int64_t)Rt[i];
      const int64_t qt = gr ? 0 : kNegInf;
      fq = (fq + pt > qt) ? fq + pt : qt;
      fp += pt;
    }
  }
  for (int o = 1; o < G; o <<= 1) {
    const int64_t pp = __shfl_up_sync(smask, fp, o, G);
    const int64_t qq = __shfl_up_sync(smask, fq, o, G);
    if (lane >= o) {
      const int64_t nq = qq + fp;
      fq = nq > fq ? nq : fq;
      fp += pp;
    }
  }
  int64_t ep = __shfl_up_sync(smask, fp, 1, G);
  int64_t eq = __shfl_up_sync(smask, fq, 1, G);
  if (lane == 0) {
    ep = 0;
    eq = kNegInf;
  }
  const int32_t y0 = (int32_t)(ep > eq ? ep : eq);  // stock entering period a
  // pass 1: this lane's totals
  Acc lsum = 0, lwroom = 0;
  int32_t lroom = 0;
  int first_bad = T, last_def = -1, nr_lane = 0;
  {
    int32_t y = y0;
#pragma unroll
    for (int i = 0; i < PM; ++i) {
      const int t = a + i;
      const int32_t avail = y + Rt[i];
      if (kind[i] & 1) {
        const int gm = (kind[i] >> 1) & 1, gr = kind[i] >> 2;
        const int32_t xr = gr ? (avail < need[i] ? avail : need[i]) : 0;
        if (!gm && xr < need[i] && first_bad == T) first_bad = t;
        lsum += (Acc)(gm ? rc.kM : 0) + (Acc)(gr ? rc.kR : 0) +
                ((Acc)rc.hM * (Acc)need[i] - (Acc)rc.hR * (Acc)xr) * (Acc)(T - t) +
                (Acc)rc.dP * (Acc)xr;
        if (gr) {
          const int32_t room = need[i] > avail ? need[i] - avail : 0;
          lroom += room;
          lwroom += xr_weight<Acc>(rc, T, t) * (Acc)room;
          ++nr_lane;
        }
        y = avail - xr;
      } else {
        y = avail;
      }
    }
  }
  // exclusive offsets of C, P, Q over the lanes
  Acc off = lsum, offQ = lwroom;
  int32_t offP = lroom;
  for (int o = 1; o < G; o <<= 1) {
    const Acc v = __shfl_up_sync(smask, off, o, G);
    const Acc vq = __shfl_up_sync(smask, offQ, o, G);
    const int32_t vp = __shfl_up_sync(smask, offP, o, G);
    if (lane >= o) {
      off += v;
      offQ += vq;
      offP += vp;
    }
  }
  const Acc total = __shfl_sync(smask, off, G - 1, G);
  const Acc totQ = __shfl_sync(smask, offQ, G - 1, G);
  const int32_t totP = __shfl_sync(smask, offP, G - 1, G);
  off -= lsum;
  offQ -= lwroom;
  offP -= lroom;
  // pass 2: the entries, written once
  {
    int32_t y = y0;
    int r = rank_below<NW>(b.r0, b.r1, a);
#pragma unroll
    for (int i = 0; i < PM; ++i) {
      const int t = a + i;
      const int32_t avail = y + Rt[i];
      if (kind[i] & 1) {
        const int gm = (kind[i] >> 1) & 1, gr = kind[i] >> 2;
        const int32_t xr = gr ? (avail < need[i] ? avail : need[i]) : 0;
        A[t] = avail;
        C[t] = off;
        off += (Acc)(gm ? rc.kM : 0) + (Acc)(gr ? rc.kR : 0) +
               ((Acc)rc.hM * (Acc)need[i] - (Acc)rc.hR * (Acc)xr) * (Acc)(T - t) +
               (Acc)rc.dP * (Acc)xr;
        if (gr) {
          if (!gm && xr < need[i]) last_def = r;
          L[r] = int2{avail - need[i], t | (gm << 16)};
          Pr[r] = offP;
          Qr[r] = offQ;
          const int32_t room = need[i] > avail ? need[i] - avail : 0;
          offP += room;
          offQ += xr_weight<Acc>(rc, T, t) * (Acc)room;
          ++r;
        }
        y = avail - xr;
      } else {
        y = avail;
      }
    }
  }
  if (G == 32) {
    first_bad = (int)__reduce_min_sync(kFull, (unsigned)first_bad);
    last_def = (int)__reduce_max_sync(kFull, (unsigned)(last_def + 1)) - 1;
  } else {
    for (int o = G >> 1; o > 0; o >>= 1) {
      const int v = __shfl_xor_sync(smask, first_bad, o, G);
      const int w = __shfl_xor_sync(smask, last_def, o, G);
      first_bad = v < first_bad ? v : first_bad;
      last_def = w > last_def ? w : last_def;
    }
  }
  if (lane == 0) {
    RowMark mk;
    mk.bad = (int16_t)(dfirst != 0 ? -1 : first_bad);  // -1: demand before the first setup
    mk.ld = (int16_t)last_def;
    m.mark()[q] = mk;
    m.S()[q] = total;
    const int nr = popc64(b.r0) + (NW == 1 ? 0 : popc64(b.r1));
    m.nR()[q] = nr;
    Pr[nr] = totP;
    Qr[nr] = totQ;
  }
}

// Row rebuild by a group of G <= 32 lanes: the two-pass variant when each
// lane holds at most 4 periods, specialised for 2 (rows of at most 64
// periods on 32 lanes, the single-run default).  Inlined: as a called
// function its live registers spill around the call, which costs more than
// its code size.
template <typename Acc, int NW>
__device__ __forceinline__ void rebuild_any(const Rows<Acc>& m, int q, int lane, int G,
                                            unsigned smask) {
  const int P = (m.T + G - 1) / G;
  if (NW == 1 && P <= 2)
    rebuild_row_regs<Acc, NW, 2>(m, q, lane, G, smask);
  else if (P <= 4)
    rebuild_row_regs<Acc, NW, 4>(m, q, lane, G, smask);
  else
    rebuild_row<Acc, NW>(m, q, lane, G, smask);
}

// ---------------------------------------------------------------------------
// Team context: the CTA's view of the run its cluster executes.
// ---------------------------------------------------------------------------
struct CtlShared {
  int run;
  int flag[2];
  int ninf[2];
  int Finf;
  int abort;
  int spec_pos;                 // speculative teams: this round's position (CTA 0's word counts)
  unsigned long long acc[2];
  unsigned long long gkey[2];
  long long F;
  unsigned long long applied, steps;
  unsigned long long gmin[64];  // per row group and warp: partial minima (groups > 32 lanes)
  int stopw[2];                 // wall-clock budget spent (CTA 0's word counts)
  int gstop[2];                 // mode-G speculative teams: CTA 0's verdict on the decision word
  int spec_dec;                 // speculative teams: this round's decision (CTA 0's word counts)
  int spec_pad;
  // a run's bookkeeping that only thread 0 of CTA 0 keeps (gvns_run): in
  // shared memory rather than in every thread's registers
  unsigned long long hash;      // trajectory hash
  long long cycles, accepted;   // VND sweeps, accepted iterations
  long long deadline;           // wall-clock budget's end (ns; 0 = none)
  RunDesc rd;                   // the run's descriptor (gvns_run reads it here)
};
// kSmemLimit leaves 1 KB of the CTA's shared memory to static words.
static_assert(sizeof(CtlShared) <= 768, "static control words outgrow their reserve");

template <typename Acc>
struct Team {
  Rows<Acc> m;
  CtlShared* sh;
  int K, T, Kc, Kcr, C, crank;
  int G, lane, sub, nsub, tid, nthr, wlane, warp, nwarps;
  unsigned smask;
  int tp, fp;
  uint32_t steps, applied;
  int vnd_cap;
  // A CTA may hold several runs at once, one per partition of its threads
  // (instances per CTA): bar = 0 for a team that owns the whole CTA, else
  // the partition's named barrier (1 + partition index) over its nthr threads.
  int bar;
  bool count;  // count decode steps (off while a run is timed)

  __device__ __forceinline__ bool owns(int k) const {
    return k >= 0 && (k % C) == crank && ((k / C) % nsub) == sub;
  }
};

// Row groups wider than a warp (G = 64 or 128 lanes): the group's
// warps meet at named barrier 1 + group index.
template <typename Acc>
__device__ __forceinline__ void group_sync(const Team<Acc>& t) {
  if (t.G <= 32) {
    __syncwarp(t.smask);
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + t.sub), "r"(t.G) : "memory");
  }
}

// Minimum of a key over the row group.
template <typename Acc>
__device__ __forceinline__ uint64_t group_min(const Team<Acc>& t, uint64_t v) {
  if (t.G <= 32) return subwarp_min(v, t.G);
  v = subwarp_min(v, 32);
  if (t.wlane == 0) t.sh->gmin[t.sub * 4 + (t.lane >> 5)] = v;
  group_sync(t);
  uint64_t m = ~0ull;
  for (int w = 0; w < (t.G >> 5); ++w) m = umin64(m, t.sh->gmin[t.sub * 4 + w]);
  group_sync(t);
  return m;
}

// Rebuild of local row q by the row group (its first warp when the group is
// wider than a warp), then a group barrier.
template <typename Acc, int NW>
__device__ __forceinline__ void group_rebuild(const Team<Acc>& t, int q) {
  if (t.G <= 32) {
    rebuild_any<Acc, NW>(t.m, q, t.lane, t.G, t.smask);
  } else if (t.lane < 32) {
    rebuild_any<Acc, NW>(t.m, q, t.lane, 32, kFull);
  }
  group_sync(t);
}

// Barrier over the threads of this CTA that belong to the team: the whole
// CTA, or the team's partition of it.
template <typename Acc>
__device__ __forceinline__ void cta_sync(const Team<Acc>& t) {
  if (t.bar == 0) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(t.bar), "r"(t.nthr) : "memory");
  }
}

// cta_sync that also returns whether `pred` was non-zero on any thread.
template <typename Acc>
__device__ __forceinline__ int cta_sync_or(const Team<Acc>& t, int pred) {
  if (t.bar == 0) return __syncthreads_or(pred);
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred), "r"(t.bar), "r"(t.nthr)
      : "memory");
  return r;
}

// Barrier over the whole team: its CTA share, or every CTA of its cluster.
template <typename Acc>
__device__ __forceinline__ void team_sync(const Team<Acc>& t) {
  if (t.C == 1) {
    cta_sync(t);
  } else {
    cg::this_cluster().sync();
  }
}

// Set up the team for run rd: shared-memory layout, staging of the CTA's
// rows (one warp per row: prefix tables, constants, start bits), control
// words, and the cache of every owned row.
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
  uint32_t v;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}

// Returns false (uniformly over the team) when the launch does not match
// what the run needs: another cluster size than configured, or less shared
// memory in the team's region (`region` bytes from `smem`) than the run's
// layout; nothing is touched then.
template <typename Acc, int NW, bool TS, bool Fresh = false>
__device__ bool team_begin(Team<Acc>& t, unsigned char* smem, uint32_t region, CtlShared* sh,
                           const VnsParams& p, const RunDesc& rd) {
  const InstDesc id = Fresh ? ldcg_inst(p.ip.insts + rd.inst) : p.ip.insts[rd.inst];
  const int K = id.K, T = id.T, C = t.C, crank = t.crank;
  t.sh = sh;
  t.K = K;
  t.T = T;
  t.Kc = (K - crank + C - 1) / C;
  t.Kcr = ((t.Kc + t.nsub - 1) / t.nsub) * t.nsub;
  t.tp = t.fp = 0;
  t.steps = t.applied = 0;
  t.vnd_cap = p.vnd_cap;
  t.count = p.count_steps != 0;
  const int Kmax = (K + C - 1) / C;
  const VnsLayout Lay = vns_layout(Kmax, T, (int)sizeof(Acc), TS);
  if (C != p.cluster || Lay.total > region) return false;
  Rows<Acc>& m = t.m;
  m.tab = TS ? (const int2*)(smem + Lay.tab) : (p.ip.gtab + id.tab_off);
  m.place(smem, Lay.rc, Lay.C0, Lay.bits, Lay.S, Lay.mark, Lay.nR, Lay.A, Lay.C, Lay.L, Lay.P,
          Lay.Q, Lay.save);
  m.slot = Lay.slot;
  m.T = T;
  m.C_ = C;
  m.crank = crank;
  m.ts = TS;
  for (int q = t.warp; q < t.Kc; q += t.nwarps) {
    const int k = q * C + crank;
    const int64_t ro = id.row_off + k;
    if (TS) {
      stage_row_warp<Fresh>(p.ip.D + id.cell_off + (int64_t)k * T,
                            p.ip.R + id.cell_off + (int64_t)k * T, T, t.wlane,
                            (int2*)(smem + Lay.tab) + (int64_t)q * (T + 1),
                            ld_in<Fresh>(p.ip.hM + ro), ld_in<Fresh>(p.ip.hR + ro),
                            p.ip.pM ? ld_in<Fresh>(p.ip.pM + ro) : 0, &m.C0()[q]);
    } else if (t.wlane == 0) {
      m.C0()[q] = p.ip.gC0[ro];
    }
    if (t.wlane == 0) {
      m.rc()[q] = row_costs<Fresh>(p.ip, ro);
      m.bits()[q] = rd.start_off >= 0 ? p.start_bits[rd.start_off + k] : all_open(T);
    }
  }
  if (t.tid == 0) {
    sh->acc[0] = sh->acc[1] = 0ull;
    sh->ninf[0] = sh->ninf[1] = 0;
    sh->flag[0] = sh->flag[1] = 0;
    sh->gkey[0] = sh->gkey[1] = ~0ull;
    sh->applied = 0ull;
    sh->steps = 0ull;
    sh->abort = 0;
  }
  cta_sync(t);
  for (int qq = t.sub; qq < t.Kcr; qq += t.nsub) {
    if (qq < t.Kc) group_rebuild<Acc, NW>(t, qq);
    if (t.G <= 32) __syncwarp();
  }
  return true;
}

__device__ __forceinline__ void write_failed_run(const VnsParams& p, const RunDesc& rd,
                                                 int status) {
  RunOut o = {};
  o.best_cost = INT64_MAX;
  o.status = status;
  p.out[rd.out] = o;
}

__device__ __forceinline__ long long globaltimer_ns() {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return (long long)v;
}

// Objective of the team: F = sum of the feasible rows' costs and ninf = the
// number of infeasible rows over the cluster (every thread gets both).
// With `stop` given (by every thread), thread 0 of CTA 0 also compares the
// global timer with `deadline` (ns; 0 = none, and only that thread's value
// matters) and every thread receives the verdict.
template <typename Acc>
__device__ void team_sums(Team<Acc>& t, int64_t& F, int& ninf, long long deadline = 0,
                          int* stop = nullptr) {
  CtlShared* sh = t.sh;
  const int tp = t.tp;
  if (stop && t.crank == 0 && t.tid == 0)
    sh->stopw[tp] = deadline > 0 && globaltimer_ns() >= deadline;
  if (t.lane == 0) {
    int64_t s = 0;
    int ni = 0;
    for (int q = t.sub; q < t.Kc; q += t.nsub) {
      const int64_t c = t.m.cost(q);
      if (c == INT64_MAX) ++ni; else s += c;
    }
    if (s) atomicAdd(&sh->acc[tp], (unsigned long long)s);
    if (ni) atomicAdd(&sh->ninf[tp], ni);
  }
  cta_sync(t);
  if (t.C == 1) {
    F = (int64_t)sh->acc[tp];
    ninf = sh->ninf[tp];
  } else {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    unsigned long long a = 0;
    int ni = 0;
    if (t.wlane < t.C) {
      a = *cl.map_shared_rank(&sh->acc[tp], t.wlane);
      ni = *cl.map_shared_rank(&sh->ninf[tp], t.wlane);
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      ni += __shfl_xor_sync(kFull, ni, o);
    }
    F = (int64_t)a;
    ninf = ni;
  }
  if (stop) *stop = t.C == 1 ? sh->stopw[tp] : *cg::this_cluster().map_shared_rank(&sh->stopw[tp], 0);
  if (t.tid == 0) {
    sh->acc[tp ^ 1] = 0ull;
    sh->ninf[tp ^ 1] = 0;
  }
  t.tp ^= 1;
}

// Speculative rounds (spec_kernel) decide in a word per round parity that
// holds (tag << 8) | d: the round's tag (round + 1, modulo 2^23) and d, the
// first accepting position (the round's active count when none accepts).
// A word holding another tag is undecided for this round.
constexpr int kSpecTagMask = (1 << 23) - 1;

__device__ __forceinline__ bool spec_moot(const int* word, int tag, int my_index) {
  const int v = *(volatile const int*)word;
  return (v >> 8) == tag && (v & 0xff) < my_index;
}

// Saturating objective of the team (sum of row costs over the cluster);
// deadline / stop as in team_sums.
template <typename Acc>
__device__ int64_t team_total(Team<Acc>& t, long long deadline = 0, int* stop = nullptr) {
  int64_t F;
  int ni;
  team_sums(t, F, ni, deadline, stop);
  return ni ? INT64_MAX : F;
}

// VND of Algorithm 1 (pipe form), mode P: every product takes its best
// strictly improving move of N_j; the j = 1..3 sweep repeats until no product
// of the team improves.  Returns the sweeps run, or -1 at the cap.
// `stop` (speculative teams): the round's decision word in global memory,
// the round's tag and this team's position; the VND gives up (returns -2) at
// a sweep boundary once the word names an earlier position, whose iteration
// makes this one moot.
template <typename Acc, int NW>
__device__ int vnd_p(Team<Acc>& t, const int* stop = nullptr, int tag = 0, int my_index = 0) {
  const int T = t.T;
  int cycles = 0;
  for (;;) {
    int improved = 0;
    for (int j = 1; j <= 3; ++j) {
      const int M = row_moves(T, j);
      if (M <= 0) continue;
      for (int qq = t.sub; qq < t.Kcr; qq += t.nsub) {
        const bool valid = qq < t.Kc;
        const int q = valid ? qq : 0;
        uint64_t best = ~0ull;
        if (valid) {
          const RowState<Acc> cur = t.m.state(q);
          // counting is decided per row, so the per-move loop carries none of it
          best = t.count ? row_best<Acc, NW, true>(t.m, q, cur, j, M, t.lane, t.G, t.steps)
                         : row_best<Acc, NW, false>(t.m, q, cur, j, M, t.lane, t.G, t.steps);
        }
        best = group_min(t, best);
        const bool imp = valid && key_cost(best) < t.m.cost(q);
        if (imp) {
          if (t.lane == 0) {
            RowBits nb = t.m.bits()[q];
            apply_row_move(nb, T, j, key_index(best));
            t.m.bits()[q] = nb;
            ++t.applied;
          }
          group_sync(t);
          group_rebuild<Acc, NW>(t, q);
          improved = 1;
        }
        if (t.G <= 32) __syncwarp();
      }
    }
    ++cycles;
    if (stop && t.C == 1 && t.tid == 0) t.sh->flag[t.fp] = spec_moot(stop, tag, my_index);
    int any = cta_sync_or(t, improved);
    int quit = 0;
    if (t.C > 1) {
      cg::cluster_group cl = cg::this_cluster();
      if (t.tid == 0) {
        int f = any;
        if (stop && t.crank == 0 && spec_moot(stop, tag, my_index)) f |= 2;
        t.sh->flag[t.fp] = f;
      }
      cl.sync();
      const int v = t.wlane < t.C ? *cl.map_shared_rank(&t.sh->flag[t.fp], t.wlane) : 0;
      any = __any_sync(kFull, v & 1);
      quit = __any_sync(kFull, v & 2);
      t.fp ^= 1;
    } else if (stop) {
      quit = t.sh->flag[t.fp];
      t.fp ^= 1;
    }
    if (quit) return -2;
    if (!any) break;
    if (cycles >= t.vnd_cap) return -1;
  }
  return cycles;
}

// VND, mode G: one best move of the whole neighbourhood by (new objective,
// global index), applied when it lowers the objective.  Every CTA of the
// team evaluates its own rows; the CTAs' minima meet through distributed
// shared memory, so all CTAs hold the same winning key.  A winning key's cost
// is the new objective itself (the other rows plus the moved row), which
// every CTA adopts without a further exchange.
// `stop` (speculative teams), as in vnd_p: thread 0 of CTA 0 reads the
// decision word during N3 and passes its verdict with the next sweep's N1
// exchange, after which the whole team gives up (returns -2) at once.
template <typename Acc, int NW>
__device__ int vnd_g(Team<Acc>& t, const int* stop = nullptr, int tag = 0, int my_index = 0) {
  CtlShared* sh = t.sh;
  const int T = t.T, C = t.C;
  int64_t F;    // sum of the feasible rows' costs (team-wide)
  int Finf;     // infeasible rows (team-wide)
  team_sums(t, F, Finf);
  if (t.tid == 0) sh->gkey[0] = sh->gkey[1] = ~0ull;
  team_sync(t);
  const int GW = t.G < 32 ? t.G : 32;  // lanes of the group inside one warp
  int cycles = 0, e = 0;
  int seen = 0;  // thread 0 of CTA 0: the decision word's verdict as read during N3
  for (;;) {
    bool improved = false;
    int quit = 0;
    for (int j = 1; j <= 3; ++j) {
      const int M = row_moves(T, j);
      if (M <= 0) continue;
      const bool lead = stop && t.crank == 0 && t.tid == 0;
      if (lead && j == 3) seen = spec_moot(stop, tag, my_index);
      if (lead && j == 1) sh->gstop[e] = seen;
      const int64_t total = Finf ? INT64_MAX : F;
      // every warp runs the same number of row iterations (the sub-warp
      // minimum below is a full-warp shuffle)
      for (int qq = t.sub; qq < t.Kcr; qq += t.nsub) {
        uint64_t best = ~0ull;
        if (qq < t.Kc) {
          const int q = qq;
          const int kg = q * C + t.crank;  // global row index
          const RowState<Acc> cur = t.m.state(q);
          const int64_t rck = t.m.cost(q);
          const int infk = rck == INT64_MAX;
          const int64_t others = (Finf - infk > 0) ? INT64_MAX : F - (infk ? 0 : rck);
          const int2* tk = t.m.tab_row(q);
          const RowCosts rc = t.m.rc()[q];
          const int64_t c0 = t.m.C0()[q];
          int st = 0;
          const SwapMasks sw = swap_masks<NW>(cur.b, T);
          const int Mj = j == 3 ? sw.n : M;  // N3: non-null swaps only
          // counting is decided per row, so the per-move loop carries none of it
          auto moves = [&](auto counted) {
            for (int i = t.lane; i < Mj; i += t.G) {
              const int l = j == 3 ? swap_of_rank<NW>(sw, T, i) : i;
              const Acc S = eval_move<Acc, NW, decltype(counted)::value>(
                  tk, T, rc, cur, t.m.A() + q * T, t.m.C() + q * T, t.m.L() + q * T,
                  t.m.P() + q * (T + 1), t.m.Q() + q * (T + 1), j, l, st);
              const int64_t nc = row_cost<Acc>(S, c0);
              const int64_t nt =
                  (others == INT64_MAX || nc == INT64_MAX) ? INT64_MAX : others + nc;
              best = umin64(best, pack_key(nt, (uint32_t)(kg * M + l)));
            }
          };
          if (t.count) moves(std::true_type{}); else moves(std::false_type{});
          t.steps += (uint32_t)st;
        }
        best = subwarp_min(best, GW);
        if ((t.tid & (GW - 1)) == 0 && best != ~0ull) atomicMin(&sh->gkey[e], best);
      }
      uint64_t gk;
      if (C == 1) {
        cta_sync(t);
        gk = sh->gkey[e];
        if (stop && j == 1) quit = sh->gstop[e];
      } else {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        uint64_t v = t.wlane < C ? *cl.map_shared_rank(&sh->gkey[e], t.wlane) : ~0ull;
        gk = subwarp_min(v, 32);
        if (stop && j == 1) quit = *cl.map_shared_rank(&sh->gstop[e], 0);
      }
      if (t.tid == 0) sh->gkey[e ^ 1] = ~0ull;
      if (gk != ~0ull && key_cost(gk) < total) {
        const int gi = key_index(gk);
        const int kw = gi / M, lw = gi - kw * M;
        const int qw = kw / C;
        if ((kw % C) == t.crank && (qw % t.nsub) == t.sub) {
          if (t.lane == 0) {
            RowBits nb = t.m.bits()[qw];
            apply_row_move(nb, T, j, lw);
            t.m.bits()[qw] = nb;
            ++t.applied;
          }
          group_sync(t);
          group_rebuild<Acc, NW>(t, qw);
        }
        // the new objective is finite, so every row is feasible now
        F = key_cost(gk);
        Finf = 0;
        improved = true;
      }
      cta_sync(t);
      e ^= 1;
      if (quit) return -2;  // uniform: every thread read CTA 0's verdict
    }
    ++cycles;
    if (!improved) break;
    if (cycles >= t.vnd_cap) return -1;
  }
  return cycles;
}

template <typename Acc, int NW>
__device__ __forceinline__ int vnd(Team<Acc>& t, int mode, const int* stop = nullptr,
                                   int tag = 0, int my_index = 0) {
  return mode == 0 ? vnd_p<Acc, NW>(t, stop, tag, my_index)
                   : vnd_g<Acc, NW>(t, stop, tag, my_index);
}

// Shake(x, k) of Algorithm 2: k moves of N_k from splitmix64 draws keyed by
// (seed, iteration, k, move j); a fork-join worker p draws with move key
// p << 8 | j (key_hi = p << 8).  `first` marks a row's first hit.
struct ShakePlan {
  int rows[kMaxShake], locs[kMaxShake];
  bool first[kMaxShake];
};

__device__ __forceinline__ ShakePlan plan_shake(uint64_t seed, int it, int ks, int K, int T,
                                                uint64_t key_hi = 0) {
  ShakePlan pl;
  const int per = row_moves(T, ks);
  const int64_t size = per > 0 ? (int64_t)K * per : 0;
#pragma unroll
  for (int j = 0; j < kMaxShake; ++j) {
    pl.rows[j] = -1;
    pl.locs[j] = 0;
    pl.first[j] = false;
    if (j < ks && size > 0) {
      const uint64_t d = shake_draw(seed, (uint64_t)it, (uint64_t)ks, key_hi | (uint64_t)j);
      const int64_t mv = (int64_t)(d % (uint64_t)size);
      pl.rows[j] = (int)(mv / per);
      pl.locs[j] = (int)(mv - (int64_t)pl.rows[j] * per);
      pl.first[j] = true;
      for (int q2 = 0; q2 < j; ++q2)
        if (pl.rows[q2] == pl.rows[j]) pl.first[j] = false;
    }
  }
  return pl;
}

// Apply a shake: the owner of each hit row saves it on first touch (for a
// rejection), applies the moves in order, then rebuilds the row.
template <typename Acc, int NW>
__device__ void apply_shake(Team<Acc>& t, const ShakePlan& pl, int ks, int par) {
#pragma unroll
  for (int j = 0; j < kMaxShake; ++j) {
    const int k = pl.rows[j];
    if (t.owns(k)) {  // uniform over the row group
      if (pl.first[j]) save_row<Acc>(t.m, k / t.C, t.m.slot_ptr(par, j), t.lane, t.G);
      group_sync(t);
      if (t.lane == 0) {
        RowBits b = t.m.bits()[k / t.C];
        apply_row_move(b, t.T, ks, pl.locs[j]);
        t.m.bits()[k / t.C] = b;
      }
      group_sync(t);
    }
  }
#pragma unroll
  for (int j = 0; j < kMaxShake; ++j) {
    const int k = pl.rows[j];
    if (t.owns(k) && pl.first[j]) group_rebuild<Acc, NW>(t, k / t.C);
  }
  if (t.G <= 32) __syncwarp();
}

// Undo a shake: the shaken rows go back to x (the other rows never moved:
// they were locally optimal in x).
template <typename Acc>
__device__ void undo_shake(Team<Acc>& t, const ShakePlan& pl, int par) {
#pragma unroll
  for (int j = 0; j < kMaxShake; ++j) {
    const int k = pl.rows[j];
    if (t.owns(k) && pl.first[j]) {
      restore_row<Acc>(t.m, k / t.C, t.m.slot_ptr(par, j), t.lane, t.G);
      group_sync(t);
    }
  }
  if (t.G <= 32) __syncwarp();
}

// Fold this CTA's per-thread counters into its control words.
template <typename Acc>
__device__ void flush_counters(Team<Acc>& t, unsigned long long* steps_dst,
                               unsigned long long* applied_dst) {
  unsigned long long v = t.steps, a = t.applied;
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_xor_sync(kFull, v, o);
    a += __shfl_xor_sync(kFull, a, o);
  }
  if (t.wlane == 0) {
    if (v) atomicAdd(steps_dst, v);
    if (a) atomicAdd(applied_dst, a);
  }
  t.steps = 0;
  t.applied = 0;
}

// Row groups of G lanes over the team's threads.
template <typename Acc>
__device__ __forceinline__ void team_set_lanes(Team<Acc>& t, int G) {
  t.G = G;
  t.lane = t.tid & (G - 1);
  t.sub = t.tid / G;
  t.nsub = t.nthr / G;
  t.smask = G >= 32 ? kFull : (((1u << G) - 1u) << (t.wlane & ~(G - 1)));
}

// The team of this thread: its cluster (every thread of the CTA), or with
// np > 1 one of np equal partitions of the CTA's threads (cluster size 1,
// G <= 32; each partition is a team of its own with its own barrier).
template <typename Acc>
__device__ __forceinline__ void team_init(Team<Acc>& t, int G, int np = 1) {
  cg::cluster_group cl = cg::this_cluster();
  t.C = (int)cl.num_blocks();
  t.crank = (int)cl.block_rank();
  t.nthr = blockDim.x / np;
  const int part = (int)threadIdx.x / t.nthr;
  t.bar = np > 1 ? 1 + part : 0;
  t.tid = threadIdx.x - part * t.nthr;
  t.wlane = t.tid & 31;
  t.warp = t.tid >> 5;
  t.nwarps = t.nthr >> 5;
  team_set_lanes(t, G);
}

// Lanes per row for a run of K products on teams of C CTAs of `threads`
// threads: the widest group (G0 .. 128 lanes) that still leaves a group per
// row, so a small instance spreads each row over more lanes instead of
// leaving groups idle.  Groups wider than a warp must tile the block and use
// at most the 15 named barriers.
__device__ __forceinline__ int run_lanes(int G0, int K, int C, int threads, int gmax = 128) {
  const int Kc = (K + C - 1) / C;
  int G = G0;
  for (int g = G0 * 2; g <= gmax; g *= 2) {
    if (threads / g < Kc) break;
    if (g > 32 && (threads % g != 0 || threads / g > 15)) continue;
    G = g;
  }
  return G;
}

// ---------------------------------------------------------------------------
// vns_kernel: persistent batched GVNS, runs taken from a device work queue.
//
// Phase 1: every team is a whole cluster (or CTA) and takes runs
// [0, p.n_whole) from queue 0.  Phase 2 (p.parts > 1, cluster size 1): each
// CTA splits into p.parts partitions of its threads, and each partition is a
// team that takes runs [p.n_whole, p.nruns) from queue 1, in its own
// p.part_bytes of dynamic shared memory (control words first, then the
// run's rows).  The host puts the runs too large for a partition first, so
// small runs share a CTA instead of leaving most of its row groups idle.
// ---------------------------------------------------------------------------
constexpr uint32_t kCtlBytes = kPartCtlBytes;
static_assert(sizeof(CtlShared) <= kCtlBytes, "partition control words outgrow their room");

// One GVNS run of Algorithm 2 by a team whose rows are staged (team_begin):
// VND from the start (unless resumed), then shake / VND / accept for the
// run's iterations; the run's solution goes to p.out_bits + rd.bits_off and
// its statistics to p.out[rd.out].  Ends with a team barrier.
template <typename Acc, int NW>
__device__ __forceinline__ void gvns_run(Team<Acc>& t, CtlShared* sh, const VnsParams& p,
                                         const RunDesc& rd_in) {
  cg::cluster_group cl = cg::this_cluster();
  // The descriptor is read from shared memory where it is needed rather than
  // held in registers across every VND call.
  if (t.tid == 0) sh->rd = rd_in;
  cta_sync(t);
  const RunDesc& rd = sh->rd;
  const int K = t.K, T = t.T;
  // Thread 0 of CTA 0 keeps the trajectory hash, the counters and the
  // wall-clock budget in shared memory: no other thread needs them, and
  // registers live across every VND call are the kernel's scarcest resource.
  const bool lead = t.crank == 0 && t.tid == 0;
  if (lead) {
    sh->hash = rd.h0;
    sh->cycles = 0;
    sh->accepted = 0;
    sh->deadline = rd.time_limit_ns > 0 ? globaltimer_ns() + rd.time_limit_ns : 0;
  }
  int status = 0, stop = 0;
  if (!rd.resume) {  // a resumed run starts from VND's output
    const int cyc = vnd<Acc, NW>(t, rd.mode);
    if (cyc < 0) status = kStatusCap; else if (lead) sh->cycles += cyc;
  }
  int64_t fx = team_total(t);
  if (rd.resume && fx != rd.f0) status = kStatusState;
  int kk = rd.k0;  // neighbourhood index k of Algorithm 2
  const int it_end = rd.it0 + rd.iters;
  int it = rd.it0;
  for (; it < it_end && status == 0 && !stop; ++it) {
    const int par = it & 1;
    const int ks = kk;
    apply_shake<Acc, NW>(t, plan_shake(rd.seed, it, ks, K, T), ks, par);
    const int cyc = vnd<Acc, NW>(t, rd.mode);
    if (cyc < 0) status = kStatusCap; else if (lead) sh->cycles += cyc;
    const int64_t f2 =
        rd.time_limit_ns > 0 ? team_total(t, lead ? sh->deadline : 0, &stop) : team_total(t);
    const int acc = f2 < fx;
    if (lead) {
      if (rd.traj_off >= 0) {
        TrajEntry te;
        te.it = it;
        te.k = ks;
        te.cost = f2;
        te.accepted = acc;
        te.reserved = 0;
        p.traj[rd.traj_off + (it - rd.it0)] = te;
      }
      uint64_t h = sh->hash;
      h = splitmix64(h ^ (uint64_t)f2);
      h = splitmix64(h ^ (((uint64_t)it << 32) | ((uint64_t)ks << 1) | (uint64_t)acc));
      sh->hash = h;
      sh->accepted += acc;
    }
    if (acc) {
      fx = f2;
      kk = 1;
    } else {
      // the shake is drawn again from its keys rather than kept live across VND
      undo_shake<Acc>(t, plan_shake(rd.seed, it, ks, K, T), par);
      kk = kk % rd.kmax + 1;
    }
    if ((it & 255) == 255) flush_counters(t, &sh->steps, &sh->applied);
  }
  cta_sync(t);  // restores of the last iteration are complete
  for (int q = t.tid; q < t.Kc; q += t.nthr)
    p.out_bits[rd.bits_off + q * t.C + t.crank] = t.m.bits()[q];
  flush_counters(t, &sh->steps, &sh->applied);
  team_sync(t);
  if (lead) {
    unsigned long long steps = 0, applied = 0;
    for (int c = 0; c < t.C; ++c) {
      steps += t.C == 1 ? sh->steps : *cl.map_shared_rank(&sh->steps, c);
      applied += t.C == 1 ? sh->applied : *cl.map_shared_rank(&sh->applied, c);
    }
    const int64_t moves_per_cycle = (int64_t)K * (2 * T + (T > 1 ? 2 * (T - 1) : 0));
    RunOut o;
    o.best_cost = fx;
    o.traj_hash = sh->hash;
    o.moves_evaluated = sh->cycles * moves_per_cycle;
    o.evals = sh->cycles * 3;
    o.vnd_cycles = sh->cycles;
    o.applied = (int64_t)applied;
    o.iterations = it - rd.it0;
    o.accepted = sh->accepted;
    o.segments = p.count_steps ? (int64_t)steps : 0;
    o.status = status;
    o.reserved = 0;
    o.k_next = kk;
    o.pad = 0;
    p.out[rd.out] = o;
  }
  team_sync(t);
}

// One team's run loop: runs [first, end) from `queue`, in `region` bytes of
// shared memory from `base`, control words in `sh`.  Inlined into each phase
// of vns_kernel, so neither phase keeps the other's state live.
template <typename Acc, int NW, bool TS>
__device__ __forceinline__ void run_loop(Team<Acc>& t, unsigned char* base, uint32_t region,
                                         CtlShared* sh, const VnsParams& p, int* queue,
                                         int first, int end, int gmax) {
  cg::cluster_group cl = cg::this_cluster();
  for (;;) {
    if (t.crank == 0 && t.tid == 0) sh->run = first + atomicAdd(queue, 1);
    team_sync(t);
    const int r = t.C == 1 ? sh->run : *cl.map_shared_rank(&sh->run, 0);
    team_sync(t);
    if (r >= end) return;
    const RunDesc rd = p.runs[r];
    team_set_lanes(t, p.adaptive_G ? run_lanes(p.G, p.ip.insts[rd.inst].K, t.C, t.nthr, gmax)
                                   : p.G);
    if (!team_begin<Acc, NW, TS>(t, base, region, sh, p, rd)) {
      if (t.crank == 0 && t.tid == 0) write_failed_run(p, rd, kStatusLaunch);
      team_sync(t);
      continue;
    }
    gvns_run<Acc, NW>(t, sh, p, rd);
  }
}

template <typename Acc, int NW, bool TS, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) vns_kernel(const VnsParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtlShared sh;
  Team<Acc> t;
  team_init(t, p.G);
  if constexpr (MAXT < 512) {
    // the host packs runs only into blocks of 512 threads or more
    run_loop<Acc, NW, TS>(t, smem, dynamic_smem_bytes(), &sh, p, p.queue, 0, p.nruns, 128);
  } else {
    // phase 1: whole teams
    run_loop<Acc, NW, TS>(t, smem, dynamic_smem_bytes(), &sh, p, p.queue, 0, p.n_whole, 128);
    if (p.n_whole >= p.nruns) return;
    // phase 2: every thread of the CTA left phase 1 together (queue 0 was
    // empty), so its named barriers are complete
    __syncthreads();
    const int np = p.parts;
    unsigned char* base = smem;
    uint32_t region = dynamic_smem_bytes();
    CtlShared* psh = &sh;
    int gmax = 128;
    if (np > 1 && t.C == 1 && (int)blockDim.x % (32 * np) == 0 && p.G <= 32 &&
        (uint32_t)np * p.part_bytes <= region && p.part_bytes > kCtlBytes) {
      team_init(t, p.G, np);
      base = smem + (size_t)((int)threadIdx.x / t.nthr) * p.part_bytes;
      psh = (CtlShared*)base;
      base += kCtlBytes;
      region = p.part_bytes - kCtlBytes;
      gmax = 32;
    }  // else (not a shape the host launches) the whole team takes these runs too
    run_loop<Acc, NW, TS>(t, base, region, psh, p, p.queue + 1, p.n_whole, p.nruns, gmax);
  }
}

// ---------------------------------------------------------------------------
// srv_kernel: serving.  Requests arrive while kernels run: the host stages a
// request's instance into the pools, appends its slot to the queue of its
// class (CTAs per team, words per bit row) and publishes the new tail.  Each
// team (a cluster of the launch) claims the next published position, runs
// that request's GVNS, writes its statistics and solution to host-mapped
// memory and then its retire word, so every request retires on its own and
// a request published after the launch began joins it.  Nothing waits: a
// team whose claim finds the queue empty exits, and so does one that has
// served q.max_runs requests (its SMs go to the launches of other classes);
// the host launches again while published requests remain unclaimed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int srv_claim(const SrvQueue& q) {
  // bounded: each failed exchange means another team claimed a position, and
  // far fewer teams than this are ever in flight
  for (int tries = 0; tries < (1 << 16); ++tries) {
    const int h = *(volatile const int*)q.head;
    const int tl = *(volatile const int*)q.tail;
    if (h >= tl) return -1;
    if (atomicCAS(q.head, h, h + 1) == h) return h;
  }
  return -1;
}

__device__ __forceinline__ RunDesc ldcg_run(const RunDesc* d) {
  static_assert(sizeof(RunDesc) % 8 == 0, "RunDesc is whole 64-bit words");
  RunDesc o;
  unsigned long long* w = (unsigned long long*)&o;
  const unsigned long long* s = (const unsigned long long*)d;
#pragma unroll
  for (int i = 0; i < (int)(sizeof(RunDesc) / 8); ++i) w[i] = __ldcg(s + i);
  return o;
}

// Lanes per row of a batched run of T periods before any widening (the
// host's batch default).
__device__ __forceinline__ int batch_lanes(int T) { return T <= 8 ? 4 : (T <= 24 ? 8 : 16); }

template <typename Acc, int NW, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) srv_kernel(const VnsParams p, const SrvQueue q) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtlShared sh;
  Team<Acc> t;
  team_init(t, 16);
  cg::cluster_group cl = cg::this_cluster();
  for (int served = 0; served < q.max_runs; ++served) {
    if (t.crank == 0 && t.tid == 0) sh.run = srv_claim(q);
    team_sync(t);
    const int r = t.C == 1 ? sh.run : *cl.map_shared_rank(&sh.run, 0);
    team_sync(t);
    if (r < 0) return;
    const int slot = __ldcg(q.slots + (r % q.cap));
    const RunDesc rd = ldcg_run(p.runs + slot);
    const InstDesc id = ldcg_inst(p.ip.insts + rd.inst);
    team_set_lanes(t, run_lanes(batch_lanes(id.T), id.K, t.C, t.nthr, 128));
    if (team_begin<Acc, NW, true, true>(t, smem, dynamic_smem_bytes(), &sh, p, rd)) {
      gvns_run<Acc, NW>(t, &sh, p, rd);
    } else {
      if (t.crank == 0 && t.tid == 0) write_failed_run(p, rd, kStatusLaunch);
      team_sync(t);
    }
    // every thread's solution words reach the host before the retire word
    __threadfence_system();
    team_sync(t);
    if (t.crank == 0 && t.tid == 0) *(volatile int32_t*)(q.done + slot) = rd.tag + 1;
  }
}

// ---------------------------------------------------------------------------
// spec_kernel: one GVNS run (mode P or G) executed by W teams that speculate on
// consecutive iterations.  In a round every team starts from the same
// incumbent x; the team at position i runs iteration it0 + i (its k assumes
// iterations it0 .. it0 + i - 1 were rejected) and publishes f(x'') and its
// changed rows.  The round commits iterations in order up to the first
// acceptance a, exactly as the sequential loop would: every team undoes its
// own shake, adopts the changed rows of position a, and the next round starts
// at it0 + a + 1 (or it0 + W when nothing was accepted).  Trajectory,
// solution and counters are those of the sequential run; work of discarded
// speculative iterations is not counted.
//
// No grid barrier separates the rounds.  A team takes its position in the
// next round by ticket as soon as it knows the decision, so the teams that
// waited for it take the first positions and the teams whose iterations
// became moot, which notice at their next sweep boundary, take the last.
// Slots, published rows and decision words alternate between two round
// parities; a team takes a ticket of round r + 1 only once every team holds
// one of round r, so nobody still reads round r - 1's data when it is
// overwritten.
// ---------------------------------------------------------------------------
constexpr long kSpinLimit = 1l << 24;  // grid-barrier polls (x ~200 ns) before giving up

// Grid barrier over the W teams.  Returns false (and the team must stop)
// when the wait exceeded its limit.
template <typename Acc>
__device__ bool grid_barrier(Team<Acc>& t, int* bar, int W) {
  __threadfence();
  team_sync(t);
  if (t.crank == 0 && t.tid == 0) {
    volatile int* vgen = bar + 1;
    const int gen = *vgen;
    __threadfence();
    if (atomicAdd(bar, 1) == W - 1) {
      atomicExch(bar, 0);
      __threadfence();
      atomicAdd(bar + 1, 1);
    } else {
      long n = 0;
      while (*vgen == gen) {
        if (++n > kSpinLimit) {
          t.sh->abort = 1;
          break;
        }
        __nanosleep(200);
      }
    }
    __threadfence();
  }
  team_sync(t);
  cg::cluster_group cl = cg::this_cluster();
  const int ab = t.C == 1 ? t.sh->abort : *cl.map_shared_rank(&t.sh->abort, 0);
  return ab == 0;
}

__device__ __forceinline__ RowBits ldcg_bits(const RowBits* p) {
  RowBits b;
  b.m0 = __ldcg(&p->m0);
  b.m1 = __ldcg(&p->m1);
  b.r0 = __ldcg(&p->r0);
  b.r1 = __ldcg(&p->r1);
  return b;
}

// The team's position in round `round` (by ticket, in order of arrival),
// taken once every team holds a ticket of the previous round; bit 16 set when
// the round is already decided for an earlier position (the iteration is
// moot).  -1 when the wait exceeded its limit.
template <typename Acc>
__device__ int spec_ticket(Team<Acc>& t, unsigned* tickets, int W, int round, const int* dec,
                           int tag) {
  if (t.crank == 0 && t.tid == 0) {
    const unsigned base = (unsigned)W * (unsigned)round;
    int v = 0;
    long n = 0;
    while ((int)(*(volatile unsigned*)tickets - base) < 0) {
      if (++n > kSpinLimit) {
        v = -1;
        break;
      }
      __nanosleep(100);
    }
    if (v == 0) {
      __threadfence();
      const int pos = (int)(atomicAdd(tickets, 1u) - base);
      // every team holds one ticket per round, so pos < W; anything else is
      // reported like a wait that ran out
      v = pos >= 0 && pos < W ? pos | (spec_moot(dec, tag, pos) ? 0x10000 : 0) : -1;
    }
    t.sh->spec_pos = v;
  }
  team_sync(t);
  if (t.C == 1) return t.sh->spec_pos;
  cg::cluster_group cl = cg::this_cluster();
  return *cl.map_shared_rank(&t.sh->spec_pos, 0);
}

// The round's first accepting position (its active count when none accepts),
// once a finished prefix of positions holds it; -1 when the wait exceeded its
// limit.
template <typename Acc>
__device__ int spec_decision(Team<Acc>& t, const int* dec, int tag) {
  if (t.crank == 0 && t.tid == 0) {
    int v;
    long n = 0;
    for (;;) {
      v = *(volatile const int*)dec;
      if ((v >> 8) == tag) {
        v &= 0xff;
        break;
      }
      if (++n > kSpinLimit) {
        v = -1;
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    t.sh->spec_dec = v;
  }
  team_sync(t);
  if (t.C == 1) return t.sh->spec_dec;
  cg::cluster_group cl = cg::this_cluster();
  return *cl.map_shared_rank(&t.sh->spec_dec, 0);
}

template <typename Acc, int NW, bool TS, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) spec_kernel(const VnsParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtlShared sh;
  Team<Acc> t;
  team_init(t, p.G);
  cg::cluster_group cl = cg::this_cluster();
  const int W = p.spec_teams;
  const int team = blockIdx.x / t.C;
  const RunDesc rd = p.runs[0];
  if (W < 2 || (int)gridDim.x != W * t.C || !team_begin<Acc, NW, TS>(t, smem, dynamic_smem_bytes(), &sh, p, rd)) {
    if (blockIdx.x == 0 && t.tid == 0) write_failed_run(p, rd, kStatusLaunch);
    return;
  }
  const int K = t.K, T = t.T;
  const int64_t moves_per_cycle = (int64_t)K * (2 * T + (T > 1 ? 2 * (T - 1) : 0));
  int status = 0;
  int64_t cycles_total = 0;
  int cyc = 0;
  if (!rd.resume) {  // a resumed run starts from VND's output
    cyc = vnd<Acc, NW>(t, rd.mode);
    if (cyc < 0) status = kStatusCap; else cycles_total += cyc;
  }
  int64_t fx = team_total(t);
  if (rd.resume && fx != rd.f0) status = kStatusState;
  flush_counters(t, &sh.steps, &sh.applied);  // the initial VND counts once (team 0)
  unsigned long long c_steps = 0, c_applied = 0;  // committed speculative work
  uint64_t h = rd.h0;
  int64_t accepted = 0;
  int it0 = rd.it0, k0 = rd.k0, round = 0;
  const int it_end = rd.it0 + rd.iters;
  const bool leader = team == 0 && t.crank == 0 && t.tid == 0;
  unsigned* const tickets = reinterpret_cast<unsigned*>(p.spec_bar);
  while (it0 < it_end && status == 0) {
    const int par = round & 1;
    const int tag = (round + 1) & kSpecTagMask;
    const int nact = (it_end - it0) < W ? (it_end - it0) : W;
    int* dec = p.spec_dec + par;
    const int tk = spec_ticket(t, tickets, W, round, dec, tag);
    if (tk < 0) {
      status = kStatusTimeout;
      break;
    }
    const int pos = tk & 0xffff;
    const bool shaken = pos < nact && !(tk & 0x10000);
    const int ks = (k0 - 1 + pos) % rd.kmax + 1;
    SpecSlot* slot = p.spec_slots + par * W + pos;
    SpecSlot* slots_w = p.spec_slots + par * W;
    ShakePlan pl;
    if (shaken) {
      if (t.crank == 0 && t.tid == 0) {
        slot->applied = 0ull;
        slot->steps = 0ull;
      }
      pl = plan_shake(rd.seed, it0 + pos, ks, K, T);
      apply_shake<Acc, NW>(t, pl, ks, par);
      cyc = vnd<Acc, NW>(t, rd.mode, dec, tag, pos);
      if (cyc != -2) {  // -2: an earlier position's iteration was accepted
        const int64_t f2 = team_total(t);
        flush_counters(t, &slot->steps, &slot->applied);
#pragma unroll
        for (int j = 0; j < kMaxShake; ++j)
          if (t.owns(pl.rows[j]) && pl.first[j] && t.lane == 0)
            p.spec_rows[(par * W + pos) * kMaxShake + j] = t.m.bits()[pl.rows[j] / t.C];
        __threadfence();
        team_sync(t);
        if (t.crank == 0 && t.warp == 0) {
          if (t.wlane == 0) {
            slot->f2 = f2;
            slot->cycles = cyc;
            __threadfence();
            atomicExch(&slot->done, 2 * round + (f2 < fx ? 1 : 0));
          }
          __syncwarp();
          // Done word, fence, then the scan: of two teams that finish at the
          // same time, at least one sees the other's done word, so the team
          // that completes the prefix always finds it complete.
          __threadfence();
          // The round is decided once a finished prefix of the positions
          // holds the first acceptance (or every position finished without
          // one); whoever completes that prefix writes the decision.
          int d = -1;
          for (int base = 0; base < nact && d < 0; base += 32) {
            const int i = base + t.wlane;
            const int v = i < nact ? *(volatile const int*)&slots_w[i].done : -1;
            const unsigned fin = __ballot_sync(kFull, i < nact && (v >> 1) == round);
            const unsigned acc = __ballot_sync(kFull, i < nact && (v >> 1) == round && (v & 1));
            const int nfin = __ffs(~fin) - 1;  // finished prefix of this chunk (-1: all 32)
            const unsigned pre = nfin < 0 ? kFull : ((1u << nfin) - 1u);
            if (acc & pre) {
              d = base + __ffs(acc & pre) - 1;
            } else if (nfin >= 0 && base + nfin < nact) {
              break;  // an unfinished position precedes any acceptance
            } else if (base + 32 >= nact) {
              d = nact;  // every position finished, none accepted
            }
          }
          if (t.wlane == 0 && d >= 0) {
            __threadfence();
            atomicExch(dec, (tag << 8) | d);
          }
        }
      } else {
        t.steps = 0;
        t.applied = 0;
      }
    }
    const int d = spec_decision(t, dec, tag);
    if (d < 0) {
      status = kStatusTimeout;
      break;
    }
    // commit in iteration order up to the first acceptance
    const SpecSlot* slots = p.spec_slots + par * W;
    const int a = d < nact ? d : -1;
    const int ncommit = a >= 0 ? a + 1 : nact;
    int capped = 0;
    for (int base = 0; base < ncommit; base += 32) {
      const int i = base + t.wlane;
      const int c = i < ncommit ? __ldcg(&slots[i].cycles) : 0;
      capped |= __any_sync(kFull, c < 0);
      int cs = c > 0 ? c : 0;
      for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(kFull, cs, o);
      cycles_total += cs;
    }
    if (team == 0 && t.crank == 0 && t.warp == 0) {
      for (int base = 0; base < ncommit; base += 32) {
        const int i = base + t.wlane;
        const bool in = i < ncommit;
        const int64_t f2i = in ? __ldcg(&slots[i].f2) : 0;
        unsigned long long st = in ? __ldcg(&slots[i].steps) : 0ull;
        unsigned long long ap = in ? __ldcg(&slots[i].applied) : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
          st += __shfl_xor_sync(kFull, st, o);
          ap += __shfl_xor_sync(kFull, ap, o);
        }
        const int n = ncommit - base < 32 ? ncommit - base : 32;
        for (int jj = 0; jj < n; ++jj) {
          const int64_t f2 = __shfl_sync(kFull, f2i, jj);
          if (t.wlane == 0) {
            const int ii = base + jj;
            const int ki = (k0 - 1 + ii) % rd.kmax + 1;
            const int acc = ii == a;
            if (rd.traj_off >= 0) {
              TrajEntry te;
              te.it = it0 + ii;
              te.k = ki;
              te.cost = f2;
              te.accepted = acc;
              te.reserved = 0;
              p.traj[rd.traj_off + (it0 + ii - rd.it0)] = te;
            }
            h = splitmix64(h ^ (uint64_t)f2);
            h = splitmix64(h ^ (((uint64_t)(it0 + ii) << 32) | ((uint64_t)ki << 1) | (uint64_t)acc));
          }
        }
        if (t.wlane == 0) {
          c_steps += st;
          c_applied += ap;
        }
      }
    }
    if (capped) {
      status = kStatusCap;
      break;
    }
    // every team moves to the committed solution
    if (shaken && pos != a) undo_shake<Acc>(t, pl, par);
    if (a >= 0 && pos != a) {
      const int ka = (k0 - 1 + a) % rd.kmax + 1;
      const ShakePlan pw = plan_shake(rd.seed, it0 + a, ka, K, T);
#pragma unroll
      for (int j = 0; j < kMaxShake; ++j) {
        const int k = pw.rows[j];
        if (t.owns(k) && pw.first[j]) {
          if (t.lane == 0)
            t.m.bits()[k / t.C] = ldcg_bits(p.spec_rows + (par * W + a) * kMaxShake + j);
          group_sync(t);
          group_rebuild<Acc, NW>(t, k / t.C);
        }
        if (t.G <= 32) __syncwarp();
      }
    }
    if (a >= 0) {
      fx = __ldcg(&slots[a].f2);
      k0 = 1;
      ++accepted;
    } else {
      k0 = (k0 - 1 + nact) % rd.kmax + 1;
    }
    it0 += ncommit;
    ++round;
  }
  // outputs (team 0)
  cta_sync(t);  // undo / adoption of the last round are complete
  if (team == 0) {
    for (int q = t.tid; q < t.Kc; q += t.nthr)
      p.out_bits[rd.bits_off + q * t.C + t.crank] = t.m.bits()[q];
  }
  team_sync(t);
  if (leader) {
    unsigned long long steps = c_steps, applied = c_applied;
    for (int c = 0; c < t.C; ++c) {
      steps += t.C == 1 ? sh.steps : *cl.map_shared_rank(&sh.steps, c);
      applied += t.C == 1 ? sh.applied : *cl.map_shared_rank(&sh.applied, c);
    }
    RunOut o;
    o.best_cost = fx;
    o.traj_hash = h;
    o.moves_evaluated = cycles_total * moves_per_cycle;
    o.evals = cycles_total * 3;
    o.vnd_cycles = cycles_total;
    o.applied = (int64_t)applied;
    o.iterations = it0 - rd.it0;
    o.accepted = accepted;
    o.segments = p.count_steps ? (int64_t)steps : 0;
    o.status = status;
    o.reserved = 0;
    o.k_next = k0;
    o.pad = 0;
    p.out[rd.out] = o;
  }
  team_sync(t);
}

// ---------------------------------------------------------------------------
// fj_kernel: Algorithm 2 as the paper runs it (Section 3, fork-join model):
// W teams (clusters), the workers, hold the same incumbent x.  In every
// iteration worker p shakes x with the iteration's k and its own draws (move
// key p << 8 | j), runs VND (mode P or G), and publishes f(x''_p) and the
// rows it changed (only shaken rows can change: the others stay locally
// optimal).  After a bounded grid barrier every worker takes the least
// (f(x''_p), p); when it is below f(x), every worker undoes its own shake and
// adopts the winner's rows, else all undo.  All workers' VND work counts.
// ---------------------------------------------------------------------------
template <typename Acc, int NW, bool TS, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) fj_kernel(const VnsParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtlShared sh;
  Team<Acc> t;
  team_init(t, p.G);
  cg::cluster_group cl = cg::this_cluster();
  const int W = p.fj_workers;
  const int team = blockIdx.x / t.C;
  const RunDesc rd = p.runs[0];
  if (W < 1 || (int)gridDim.x != W * t.C || !team_begin<Acc, NW, TS>(t, smem, dynamic_smem_bytes(), &sh, p, rd)) {
    if (blockIdx.x == 0 && t.tid == 0) write_failed_run(p, rd, kStatusLaunch);
    return;
  }
  const int K = t.K, T = t.T;
  const int64_t moves_per_cycle = (int64_t)K * (2 * T + (T > 1 ? 2 * (T - 1) : 0));
  const bool leader = team == 0 && t.crank == 0 && t.tid == 0;
  // wall-clock budget from the run's start (worker 0's leader keeps time)
  const long long deadline = rd.time_limit_ns > 0 && leader ? globaltimer_ns() + rd.time_limit_ns : 0;
  int status = 0, stop = 0;
  int64_t cycles_total = 0;
  int cyc = 0;
  if (!rd.resume) {  // every worker descends from the start; counted once
    cyc = vnd<Acc, NW>(t, rd.mode);
    if (cyc < 0) status = kStatusCap; else cycles_total += cyc;
  }
  int64_t fx = team_total(t);
  if (rd.resume && fx != rd.f0) status = kStatusState;
  flush_counters(t, &sh.steps, &sh.applied);
  unsigned long long c_steps = 0, c_applied = 0;  // the workers' iterations (leader)
  uint64_t h = rd.h0;
  int64_t accepted = 0;
  int it = rd.it0, kk = rd.k0;
  const int it_end = rd.it0 + rd.iters;
  for (; it < it_end && status == 0 && !stop; ++it) {
    const int par = it & 1;
    SpecSlot* slot = p.spec_slots + par * W + team;
    if (t.crank == 0 && t.tid == 0) {
      slot->applied = 0ull;
      slot->steps = 0ull;
    }
    const ShakePlan pl = plan_shake(rd.seed, it, kk, K, T, (uint64_t)team << 8);
    apply_shake<Acc, NW>(t, pl, kk, par);
    cyc = vnd<Acc, NW>(t, rd.mode);
    int spent = 0;  // worker 0: the budget is spent
    const int64_t f2 = team_total(t, deadline, &spent);  // cluster barrier: the slot reset is visible
    flush_counters(t, &slot->steps, &slot->applied);
#pragma unroll
    for (int j = 0; j < kMaxShake; ++j)
      if (t.owns(pl.rows[j]) && pl.first[j] && t.lane == 0)
        p.spec_rows[(par * W + team) * kMaxShake + j] = t.m.bits()[pl.rows[j] / t.C];
    if (t.crank == 0 && t.tid == 0) {
      slot->f2 = f2;
      slot->cycles = cyc;
      slot->done = spent;
    }
    if (!grid_barrier(t, p.spec_bar, W)) {
      status = kStatusTimeout;
      break;
    }
    // least (f(x''_p), p) over the workers; VND caps; committed work
    const SpecSlot* slots = p.spec_slots + par * W;
    uint64_t best = ~0ull;
    int capped = 0, cs = 0;
    for (int base = 0; base < W; base += 32) {
      const int i = base + t.wlane;
      if (i < W) {
        best = umin64(best, pack_key(__ldcg(&slots[i].f2), (uint32_t)i));
        const int c = __ldcg(&slots[i].cycles);
        capped |= c < 0;
        cs += c > 0 ? c : 0;
      }
    }
    best = subwarp_min(best, 32);
    capped = __any_sync(kFull, capped);
    for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(kFull, cs, o);
    cycles_total += cs;
    const int a = key_index(best);
    const int64_t fa = key_cost(best);
    const int acc = fa < fx;
    stop = __ldcg(&slots[0].done);  // worker 0's verdict on the budget
    if (team == 0 && t.crank == 0 && t.warp == 0) {
      unsigned long long st = 0ull, ap = 0ull;
      for (int i = t.wlane; i < W; i += 32) {
        st += __ldcg(&slots[i].steps);
        ap += __ldcg(&slots[i].applied);
      }
      for (int o = 16; o > 0; o >>= 1) {
        st += __shfl_xor_sync(kFull, st, o);
        ap += __shfl_xor_sync(kFull, ap, o);
      }
      if (t.wlane == 0) {
        c_steps += st;
        c_applied += ap;
        if (rd.traj_off >= 0) {
          TrajEntry te;
          te.it = it;
          te.k = kk;
          te.cost = fa;
          te.accepted = acc;
          te.reserved = a;
          p.traj[rd.traj_off + (it - rd.it0)] = te;
        }
        h = splitmix64(h ^ (uint64_t)fa);
        h = splitmix64(h ^ (((uint64_t)it << 32) | ((uint64_t)kk << 1) | (uint64_t)acc));
      }
    }
    if (capped) {
      status = kStatusCap;
      break;
    }
    // every worker moves to the new incumbent
    if (!(acc && team == a)) undo_shake<Acc>(t, pl, par);
    if (acc && team != a) {
      const ShakePlan pw = plan_shake(rd.seed, it, kk, K, T, (uint64_t)a << 8);
#pragma unroll
      for (int j = 0; j < kMaxShake; ++j) {
        const int k = pw.rows[j];
        if (t.owns(k) && pw.first[j]) {
          if (t.lane == 0)
            t.m.bits()[k / t.C] = ldcg_bits(p.spec_rows + (par * W + a) * kMaxShake + j);
          group_sync(t);
          group_rebuild<Acc, NW>(t, k / t.C);
        }
        if (t.G <= 32) __syncwarp();
      }
    }
    if (acc) {
      fx = fa;
      kk = 1;
      ++accepted;
    } else {
      kk = kk % rd.kmax + 1;
    }
  }
  // outputs (worker 0)
  cta_sync(t);  // undo / adoption of the last iteration are complete
  if (team == 0) {
    for (int q = t.tid; q < t.Kc; q += t.nthr)
      p.out_bits[rd.bits_off + q * t.C + t.crank] = t.m.bits()[q];
  }
  team_sync(t);
  if (leader) {
    unsigned long long steps = c_steps, applied = c_applied;
    for (int c = 0; c < t.C; ++c) {
      steps += t.C == 1 ? sh.steps : *cl.map_shared_rank(&sh.steps, c);
      applied += t.C == 1 ? sh.applied : *cl.map_shared_rank(&sh.applied, c);
    }
    RunOut o;
    o.best_cost = fx;
    o.traj_hash = h;
    o.moves_evaluated = cycles_total * moves_per_cycle;
    o.evals = cycles_total * 3;
    o.vnd_cycles = cycles_total;
    o.applied = (int64_t)applied;
    o.iterations = it - rd.it0;
    o.accepted = accepted;
    o.segments = p.count_steps ? (int64_t)steps : 0;
    o.status = status;
    o.reserved = W;
    o.k_next = kk;
    o.pad = 0;
    p.out[rd.out] = o;
  }
  team_sync(t);
}

}  // namespace vns

template <typename Acc, int NW, bool TS, int MAXT>
cudaError_t vns_prepare_t(size_t smem, int threads, int cluster, int* active) {
  auto kern = vns::vns_kernel<Acc, NW, TS, MAXT>;
  void (*const all[3])(const VnsParams) = {kern, vns::spec_kernel<Acc, NW, TS, MAXT>,
                                            vns::fj_kernel<Acc, NW, TS, MAXT>};
  for (auto f : all) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && cluster > 8)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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

// Launch the batched kernel, the fork-join one when p.fj_workers > 0, or the
// speculative one when p.spec_teams > 1.  The last two take blocks = teams x
// cluster; the host sizes the teams to what the occupancy query reports
// resident, and the grid barrier's waits are bounded, so teams that could
// not all be resident end with a timeout status instead of waiting forever.
template <typename Acc, int NW, bool TS, int MAXT>
cudaError_t vns_launch_t(const VnsParams& p, int blocks, int threads, size_t smem,
                         int cluster, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (cluster > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = cluster;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = na;
  if (p.fj_workers > 0) return cudaLaunchKernelEx(&cfg, vns::fj_kernel<Acc, NW, TS, MAXT>, p);
  if (p.spec_teams <= 1) return cudaLaunchKernelEx(&cfg, vns::vns_kernel<Acc, NW, TS, MAXT>, p);
  return cudaLaunchKernelEx(&cfg, vns::spec_kernel<Acc, NW, TS, MAXT>, p);
}

template <typename Acc, int NW>
cudaError_t srv_prepare_t(size_t smem, int threads, int cluster, int* active) {
  auto kern = vns::srv_kernel<Acc, NW, 1024>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && cluster > 8)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  if (cluster <= 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(active, kern, threads, smem);
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

template <typename Acc, int NW>
cudaError_t srv_launch_t(const VnsParams& p, const SrvQueue& q, int blocks, int threads,
                         size_t smem, int cluster, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  int na = 0;
  if (cluster > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    na = 1;
  }
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, vns::srv_kernel<Acc, NW, 1024>, p, q);
}

}  // namespace elsr
