// elsr_row.cuh -- per-product-row arithmetic of the ELSR neighbourhood
// evaluation: segment decode over prefix tables, delta re-decode of a moved
// row, and the row cache that the delta re-decode starts and merges from.
//
// Model (Section 2 of Antoniadis & Sifaleras 2017): a row (product k) has T
// periods, demand D(t), returns R(t), setup costs kM, kR, holding costs hM,
// hR and setup bits gM(t), gR(t).  Decode rule (reading of the formulation
// the paper defers to [SK2016]): a setup at s covers the demand of the
// periods up to the next setup n, "need" = sum D[s..n); remanufacturing
// takes xR = min(avail, need) when gR(s) = 1, where avail = recoverable
// stock entering s plus R(s); manufacturing covers the rest when
// gM(s) = 1, and a shortfall is infeasible.  Demand before the first setup
// is infeasible.
//
// GB300 formulation (not the paper's, which re-ran a per-period loop):
// with exclusive demand prefixes CD[j] = sum_{i<j} D(i) and inclusive return
// prefixes CR1[j] = sum_{i<=j} R(i), one setup segment [s, n) costs O(1):
//   need  = CD[n] - CD[s]
//   xR    = gR(s) ? min(avail, need) : 0
//   cost += kM*gM(s) + kR*gR(s) + (hM*need - hR*xR) * (T - s)
//   avail = avail - xR + CR1[n] - CR1[s]          (stock entering n)
// because the holding cost of a whole row telescopes: sum_t yM(t) =
// sum_t (xM+xR-D)(t)*(T-t) and sum_t yR(t) = sum_t (R-xR)(t)*(T-t).  The row
// cost is S + C0 with S the sum of segment terms and the per-row constant
// C0 = hR * sum_t R(t)(T-t) - hM * sum_t D(t)(T-t).
//
// With unit production costs pM, pR (Algorithm 1's signature) the row adds
// pM * sum D to C0 and every remanufactured unit's weight hR*(T-s) becomes
// hR*(T-s) - (pR - pM) (see xr_weight).
//
// Row cache (per setup s of the current row, from its relaxed decode):
// A[s] = avail at s and C[s] = S accumulated before s, plus the list of gR
// setups with prefix sums of their room.  A move changes
// periods t1..t2 (t2 <= t1+1); its re-decode starts at s0, the last period
// <= t1 that is a setup both before and after the move (see eval_move).
//
// Functions are __host__ __device__ so that the same arithmetic can be
// exercised by host-side unit tests of this header.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define ELSR_HD __host__ __device__ __forceinline__
#else
// Host-only compilation (unit tests of this header): CUDA's int2.
#define ELSR_HD static inline
struct int2 {
  int x, y;
};
#endif

namespace elsr {

// Sentinels for an infeasible row in the 32- and 64-bit accumulators.
template <typename Acc> struct Inf;
template <> struct Inf<int32_t> { static constexpr int32_t value = INT32_MAX; };
template <> struct Inf<int64_t> { static constexpr int64_t value = INT64_MAX; };

ELSR_HD int lowbit(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __ffsll((long long)x) - 1;
#else
  return __builtin_ctzll(x);
#endif
}

ELSR_HD int highbit(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return 63 - __clzll((long long)x);
#else
  return 63 - __builtin_clzll(x);
#endif
}

// Setup bits of one row: T <= 128 periods in two 64-bit words per type.
struct RowBits {
  uint64_t m0, m1;  // gM(t): bit t of m0 for t < 64, bit t-64 of m1
  uint64_t r0, r1;  // gR(t)
};

ELSR_HD int bit_of(uint64_t w0, uint64_t w1, int t) {
  return (int)(((t < 64) ? (w0 >> t) : (w1 >> (t - 64))) & 1ull);
}

ELSR_HD void flip(uint64_t& w0, uint64_t& w1, int t) {
  if (t < 64) w0 ^= (1ull << t); else w1 ^= (1ull << (t - 64));
}

// First set bit strictly after s (s >= -1), or T when none.  Bits at or
// above T are always zero.
ELSR_HD int next_set(uint64_t u0, uint64_t u1, int s, int T) {
  int p = s + 1;
  if (p < 64) {
    uint64_t m = u0 & (~0ull << p);
    if (m) return lowbit(m);
    p = 64;
  }
  if (p < 128) {
    uint64_t m = u1 & (~0ull << (p - 64));
    if (m) return 64 + lowbit(m);
  }
  return T;
}

// Last set bit strictly before t (t >= 0), or -1 when none.
ELSR_HD int prev_set(uint64_t u0, uint64_t u1, int t) {
  if (t > 64) {
    int q = t - 64;
    uint64_t m = (q >= 64) ? u1 : (u1 & ((1ull << q) - 1ull));
    if (m) return 64 + highbit(m);
    t = 64;
  }
  uint64_t m = (t >= 64) ? u0 : (u0 & ((1ull << t) - 1ull));
  return m ? highbit(m) : -1;
}

// Number of moves of N_j in one row (N1, N2: T; N3: 2(T-1)).
ELSR_HD int row_moves(int T, int j) { return j == 3 ? 2 * (T - 1) : T; }

// Apply move `local` of N_j to a row (N1 flip gM, N2 flip gR, N3 swap).
ELSR_HD void apply_row_move(RowBits& b, int T, int j, int local) {
  if (j == 1) {
    flip(b.m0, b.m1, local);
  } else if (j == 2) {
    flip(b.r0, b.r1, local);
  } else {
    const int c = local >= (T - 1);
    const int t = local - c * (T - 1);
    uint64_t& w0 = c ? b.r0 : b.m0;
    uint64_t& w1 = c ? b.r1 : b.m1;
    if (bit_of(w0, w1, t) != bit_of(w0, w1, t + 1)) {
      flip(w0, w1, t);
      flip(w0, w1, t + 1);
    }
  }
}

// Per-row constants: costs and the row's prefix table tab[0..T] =
// {CD[j], CR1[j]} (CR1[T] = total returns).  dP = pR - pM, the difference
// of the unit production costs of Algorithm 1's signature (0 when the
// instance has none).
struct RowCosts {
  int32_t kM, kR, hM, hR, dP;
};

// What one more unit remanufactured (and one less manufactured) at setup s
// saves: hR per period of recoverable stock to the horizon, less the unit
// cost difference dP.  With xM + xR = need at every setup, a segment costs
// hM*need*(T-s) - xr_weight*xR, and the row's production cost is pM * sum D
// (in C0) plus dP * sum xR.
template <typename Acc>
ELSR_HD Acc xr_weight(const RowCosts& rc, int T, int s) {
  return (Acc)rc.hR * (Acc)(T - s) - (Acc)rc.dP;
}

// One segment [s, n) with setup flags gm, gr at s.  ts = tab[s], tn = tab[n].
// Updates avail (stock entering n) and S; returns false on a shortfall.
template <typename Acc>
ELSR_HD bool seg_step(int s, int gm, int gr, int2 ts, int2 tn, int T,
                      const RowCosts& rc, int32_t& avail, Acc& S) {
  const int32_t need = tn.x - ts.x;
  const int32_t xr = gr ? (avail < need ? avail : need) : 0;
  if (!gm && xr < need) return false;
  S += (Acc)(gm ? rc.kM : 0) + (Acc)(gr ? rc.kR : 0) +
       ((Acc)rc.hM * (Acc)need - (Acc)rc.hR * (Acc)xr) * (Acc)(T - s) + (Acc)rc.dP * (Acc)xr;
  avail = avail - xr + (tn.y - ts.y);
  return true;
}

// Cache of the current row (per product), from its relaxed decode: the
// decode rule applied to every setup, where a remanufacture-only setup whose
// stock falls short still takes xR = avail and its deficit is treated as
// manufactured.  For a feasible row this is the decode itself.
//   A[s], C[s]  at every setup s: stock entering s and S accumulated before s
//   L[0..nR)    the row's gR setups in period order:
//               {surplus(s) = A[s] - need(s), s | gM(s)<<16}
//   P, Q[0..nR] exclusive prefix sums over L of room = max(0, need - A) and
//               xr_weight(s)*room
// bad = T when the row is feasible; else its first setup that falls short
// (-1 when demand precedes the first setup: then nothing is cached); ld = the
// L index of its last setup that falls short (-1 when none).
template <typename Acc>
struct RowState {
  RowBits b;
  Acc S;    // segment sum of the relaxed decode
  int bad;
  int nR;   // entries of L
  int ld;
};

// Per-row marks as stored with the row cache.
struct RowMark {
  int16_t bad, ld;
};

// Objective of a row from its state: Inf when it falls short anywhere.
template <typename Acc>
ELSR_HD int64_t state_cost(Acc S, int bad, int T, int64_t C0) {
  return bad < T ? INT64_MAX : (int64_t)S + C0;
}

// Bit helpers specialised on the number of 64-bit words per bit row (NW = 1
// when T <= 64).
template <int NW>
ELSR_HD int nxt(uint64_t u0, uint64_t u1, int s, int T) {
  if (NW == 1) {
    const int p = s + 1;
    const uint64_t m = p >= 64 ? 0ull : (u0 & (~0ull << p));
    return m ? lowbit(m) : T;
  }
  return next_set(u0, u1, s, T);
}

template <int NW>
ELSR_HD int prv(uint64_t u0, uint64_t u1, int t) {
  if (NW == 1) {
    const uint64_t m = t >= 64 ? u0 : (u0 & ((1ull << t) - 1ull));
    return m ? highbit(m) : -1;
  }
  return prev_set(u0, u1, t);
}

template <int NW>
ELSR_HD int bitat(uint64_t w0, uint64_t w1, int t) {
  if (NW == 1) return (int)((w0 >> t) & 1ull);
  return bit_of(w0, w1, t);
}

ELSR_HD int popc64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __popcll((long long)x);
#else
  return __builtin_popcountll(x);
#endif
}

// Number of set bits strictly below position s.
template <int NW>
ELSR_HD int rank_below(uint64_t w0, uint64_t w1, int s) {
  if (NW == 1 || s <= 64) return popc64(s >= 64 ? w0 : (w0 & ((1ull << s) - 1ull)));
  return popc64(w0) + popc64(s >= 128 ? w1 : (w1 & ((1ull << (s - 64)) - 1ull)));
}

// Position of the set bit of rank i (0-based) in a 32-bit word holding more
// than i set bits, by halving with population counts.
ELSR_HD int select32(uint32_t w, int i) {
  int base = 0;
#if defined(__CUDA_ARCH__)
#define ELSR_POPC32(x) __popc(x)
#else
#define ELSR_POPC32(x) __builtin_popcount(x)
#endif
  int c = ELSR_POPC32(w & 0xFFFFu);
  if (i >= c) { i -= c; w >>= 16; base += 16; }
  c = ELSR_POPC32(w & 0xFFu);
  if (i >= c) { i -= c; w >>= 8; base += 8; }
  c = ELSR_POPC32(w & 0xFu);
  if (i >= c) { i -= c; w >>= 4; base += 4; }
  c = ELSR_POPC32(w & 0x3u);
  if (i >= c) { i -= c; w >>= 2; base += 2; }
  if (i >= (int)(w & 1u)) base += 1;
#undef ELSR_POPC32
  return base;
}

// Position of the set bit of rank i in a bit row (w0: bits 0..63, w1: bits
// 64..127); the row holds more than i set bits.
template <int NW>
ELSR_HD int select_bit(uint64_t w0, uint64_t w1, int i) {
  if (NW == 2) {
    const int c0 = popc64(w0);
    if (i >= c0) return 64 + select_bit<1>(w1, 0, i - c0);
  }
  const int c = popc64(w0 & 0xFFFFFFFFull);
  if (i < c) return select32((uint32_t)w0, i);
  return 32 + select32((uint32_t)(w0 >> 32), i - c);
}

// The swaps of N3 that change the row: positions t <= T-2 whose bit differs
// from bit t+1, for the gM row (x0, x1) and the gR row (y0, y1).  A null swap
// leaves the row as it is, so it can never be a strictly improving move.
struct SwapMasks {
  uint64_t x0, x1, y0, y1;
  int nm, n;  // non-null swaps of gM, of both rows
};

template <int NW>
ELSR_HD SwapMasks swap_masks(const RowBits& b, int T) {
  SwapMasks s;
  const int P = T - 1;  // swap positions 0..T-2
  const uint64_t k0 = P >= 64 ? ~0ull : (P <= 0 ? 0ull : ((1ull << P) - 1ull));
  const uint64_t k1 = P > 64 ? ((P >= 128) ? ~0ull : ((1ull << (P - 64)) - 1ull)) : 0ull;
  if (NW == 1) {
    s.x0 = (b.m0 ^ (b.m0 >> 1)) & k0;
    s.y0 = (b.r0 ^ (b.r0 >> 1)) & k0;
    s.x1 = s.y1 = 0ull;
  } else {
    s.x0 = (b.m0 ^ ((b.m0 >> 1) | (b.m1 << 63))) & k0;
    s.x1 = (b.m1 ^ (b.m1 >> 1)) & k1;
    s.y0 = (b.r0 ^ ((b.r0 >> 1) | (b.r1 << 63))) & k0;
    s.y1 = (b.r1 ^ (b.r1 >> 1)) & k1;
  }
  s.nm = popc64(s.x0) + popc64(s.x1);
  s.n = s.nm + popc64(s.y0) + popc64(s.y1);
  return s;
}

// Local N3 index of the non-null swap of rank i (i < s.n): gM swaps first,
// then gR swaps, each in period order (so ranks keep the index order).
template <int NW>
ELSR_HD int swap_of_rank(const SwapMasks& s, int T, int i) {
  return i < s.nm ? select_bit<NW>(s.x0, s.x1, i)
                  : (T - 1) + select_bit<NW>(s.y0, s.y1, i - s.nm);
}

// Relaxed decode of a whole row from its bits, writing the cache.  Returns
// the relaxed S and sets bad, nR and ld.  P, Q ([nR+1]) receive exclusive
// prefix sums over the gR list of room(r) = max(0, need - avail) and
// xr_weight(s)*room(r).  segs counts the segments walked.
template <typename Acc, int NW>
ELSR_HD Acc build_row(const int2* tab, int T, const RowCosts& rc,
                      const RowBits& b, int32_t* A, Acc* C, int2* L,
                      int32_t* P, Acc* Q, int& bad, int& nR, int& ld, int& segs) {
  const uint64_t u0 = b.m0 | b.r0, u1 = b.m1 | b.r1;
  nR = 0;
  ld = -1;
  P[0] = 0;
  Q[0] = 0;
  int s = nxt<NW>(u0, u1, -1, T);
  int2 ts = tab[s];
  if (ts.x != 0) {  // demand before the first setup
    bad = -1;
    return 0;
  }
  bad = T;
  int32_t avail = ts.y;
  Acc S = 0;
  while (s < T) {
    A[s] = avail;
    C[s] = S;
    const int n = nxt<NW>(u0, u1, s, T);
    const int2 tn = tab[n];
    const int gm = bitat<NW>(b.m0, b.m1, s), gr = bitat<NW>(b.r0, b.r1, s);
    const int32_t need = tn.x - ts.x;
    const int32_t xr = gr ? (avail < need ? avail : need) : 0;
    ++segs;
    if (gr) {
      int2 e;
      e.x = avail - need;
      e.y = s | (gm << 16);
      L[nR] = e;
      const int32_t room = need > avail ? need - avail : 0;
      P[nR + 1] = P[nR] + room;
      Q[nR + 1] = Q[nR] + xr_weight<Acc>(rc, T, s) * (Acc)room;
      if (!gm && xr < need) {  // deficit, taken as manufactured
        if (bad == T) bad = s;
        ld = nR;
      }
      ++nR;
    }
    S += (Acc)(gm ? rc.kM : 0) + (Acc)(gr ? rc.kR : 0) +
         (Acc)rc.hM * (Acc)need * (Acc)(T - s) - xr_weight<Acc>(rc, T, s) * (Acc)xr;
    avail = avail - xr + (tn.y - ts.y);
    s = n;
    ts = tn;
  }
  return S;
}

// Delta re-decode of the row after move `local` of N_j (Section 3's "find
// the best neighbour" for one candidate).  Returns the new segment sum (Inf
// when the moved row is infeasible).  steps counts the decode steps of the
// move, a work measure: the segments of the changed region, then every setup
// from s1 on while the moved row enters it with other stock than the row
// before the move (relaxed decode), up to the one where it falls short; the
// closed forms below skip most of these setups, the count does not.
//
// Changed region: from s0 (the last period <= t1 that is a setup before and
// after the move) segment by segment while the segment start is <= t2 (to
// the end of the row when the current row has demand before its first
// setup, where nothing is cached).  At the first setup s1 > t2 both rows
// have the same setups from there on and differ only in the recoverable
// stock, by delta = avail_new - A[s1].  With the telescoped cost the suffix
// then costs its cached (relaxed) value plus, at every later gR setup,
// -xr_weight(s)*dx where dx is the change of xR = min(avail, need); delta
// shrinks by dx, and the walk stops when it reaches 0.  A setup of the
// current row that falls short (a deficit in the relaxed decode) is fixed
// only when delta still covers its room there, so the moved row is feasible
// only when delta covers the rooms of all such setups from s1 on.
template <typename Acc, int NW, bool Count = true>
ELSR_HD Acc eval_move(const int2* tab, int T, const RowCosts& rc,
                      const RowState<Acc>& cur, const int32_t* A,
                      const Acc* C, const int2* L, const int32_t* P,
                      const Acc* Q, int j, int local, int& steps) {
  constexpr bool count = Count;
  RowBits nb = cur.b;
  int t1, other;
  if (j == 1) {
    t1 = local;
    flip(nb.m0, nb.m1, t1);
    other = bitat<NW>(nb.r0, nb.r1, t1);
  } else if (j == 2) {
    t1 = local;
    flip(nb.r0, nb.r1, t1);
    other = bitat<NW>(nb.m0, nb.m1, t1);
  } else {
    const int c = local >= (T - 1);
    t1 = local - c * (T - 1);
    uint64_t& w0 = c ? nb.r0 : nb.m0;
    uint64_t& w1 = c ? nb.r1 : nb.m1;
    if (bitat<NW>(w0, w1, t1) == bitat<NW>(w0, w1, t1 + 1))  // null swap
      return cur.bad < T ? Inf<Acc>::value : cur.S;
    flip(w0, w1, t1);
    flip(w0, w1, t1 + 1);
    other = c ? bitat<NW>(nb.m0, nb.m1, t1) : bitat<NW>(nb.r0, nb.r1, t1);
  }
  const int t2 = (j == 3) ? t1 + 1 : t1;
  const uint64_t u0 = nb.m0 | nb.r0, u1 = nb.m1 | nb.r1;
  const int s0 = other ? t1 : prv<NW>(u0, u1, t1);
  int s;
  int32_t avail;
  Acc S;
  if (cur.bad < 0) {
    // Nothing cached (demand precedes the row's first setup): the moved row
    // is feasible only if the move adds a setup before all demand, and is
    // then decoded to its end.
    if (s0 >= 0) return Inf<Acc>::value;
    s = nxt<NW>(u0, u1, -1, T);
    int2 ts = tab[s];
    if (ts.x != 0) return Inf<Acc>::value;
    avail = ts.y;
    S = 0;
    while (s < T) {
      const int n = nxt<NW>(u0, u1, s, T);
      const int2 tn = tab[n];
      if constexpr (count) ++steps;
      if (!seg_step<Acc>(s, bitat<NW>(nb.m0, nb.m1, s), bitat<NW>(nb.r0, nb.r1, s),
                         ts, tn, T, rc, avail, S))
        return Inf<Acc>::value;
      s = n;
      ts = tn;
    }
    return S;
  }
  if (s0 > cur.bad) return Inf<Acc>::value;  // unchanged prefix falls short
  // The changed region has at most three segments of the moved row, starting
  // at a0 (s0, or the row's first setup), t1 and t1 + 1 (when they hold
  // setups of the moved row after a0), and ends at s1, the first setup after
  // t2 (the same in both rows).  Their bounds come from the bits alone, so
  // every table entry they need is loaded up front.
  const int s1 = nxt<NW>(u0, u1, t2, T);
  int a0;
  if (s0 >= 0) {
    a0 = s0;
  } else {
    a0 = nxt<NW>(u0, u1, -1, T);
  }
  const int2 ta0 = tab[a0];
  const int2 tt1 = tab[t1];
  const int2 tt2 = tab[t2];
  const int2 ts1 = tab[s1];
  // cache entries at s1, issued together with the region's (s1 = T reads an
  // unused in-range entry)
  const int sc = s1 < T ? s1 : T - 1;
  const int32_t A1 = A[sc];
  const Acc C1 = C[sc];
  if (s0 >= 0) {
    avail = A[s0];
    S = C[s0];
  } else {
    if (ta0.x != 0) return Inf<Acc>::value;  // demand before the first setup
    avail = ta0.y;
    S = 0;
  }
  const bool v0 = a0 <= t2;
  const bool v1 = t1 > a0 && bitat<NW>(u0, u1, t1);
  const bool v2 = j == 3 && t2 > a0 && bitat<NW>(u0, u1, t2);
  if (v0) {
    if constexpr (count) ++steps;
    const int2 te = v1 ? tt1 : (v2 ? tt2 : ts1);
    if (!seg_step<Acc>(a0, bitat<NW>(nb.m0, nb.m1, a0), bitat<NW>(nb.r0, nb.r1, a0), ta0,
                       te, T, rc, avail, S))
      return Inf<Acc>::value;
  }
  if (v1) {
    if constexpr (count) ++steps;
    if (!seg_step<Acc>(t1, bitat<NW>(nb.m0, nb.m1, t1), bitat<NW>(nb.r0, nb.r1, t1), tt1,
                       v2 ? tt2 : ts1, T, rc, avail, S))
      return Inf<Acc>::value;
  }
  if (v2) {
    if constexpr (count) ++steps;
    if (!seg_step<Acc>(t2, bitat<NW>(nb.m0, nb.m1, t2), bitat<NW>(nb.r0, nb.r1, t2), tt2,
                       ts1, T, rc, avail, S))
      return Inf<Acc>::value;
  }
  if (s1 >= T) return S;
  // suffix: cached cost plus the effect of the stock difference delta
  int32_t delta = avail - A1;
  S += cur.S - C1;
  const int r0 = rank_below<NW>(cur.b.r0, cur.b.r1, s1);
  if (delta == 0) return cur.ld >= r0 ? Inf<Acc>::value : S;
  // the step count takes the setups from s1 through the last one the stock
  // difference reaches; from s1 on the current row has the moved row's
  // setups, and its bits stay live in the caller anyway.  Callers that time
  // the search instantiate Count = false: no counting code at all.
  const uint64_t w0 = cur.b.m0 | cur.b.r0, w1 = cur.b.m1 | cur.b.r1;
  int u_s1 = 0;
  if constexpr (count) u_s1 = rank_below<NW>(w0, w1, s1);
  if (delta > 0) {
    // More stock: each later gR setup absorbs up to its room (need minus the
    // stock it had), lowering xM by as much, until delta is used up.  With
    // the prefix sums P (room) and Q (xr_weight*room) the setup z where the
    // rest of delta is absorbed is a binary search, and the cost is closed
    // form.  The step count takes every setup from s1 through z (through
    // the horizon when delta is never used up).  A deficit setup after z,
    // or at z with room left over, still falls short.
    const int32_t P0 = P[r0], Pn = P[cur.nR];
    const Acc Q0 = Q[r0], Qn = Q[cur.nR];
    const int32_t target = P0 + delta;
    if (Pn < target) {
      if constexpr (count) steps += rank_below<NW>(w0, w1, T) - u_s1;
      return S - (Qn - Q0);
    }
    // smallest z in [r0, nR) with P[z+1] >= target: the answer stays in
    // [lo, lo + n) with P[lo + n] >= target while n halves
    int lo = r0, n = cur.nR - r0;
    while (n > 1) {
      const int half = n >> 1;
      lo = P[lo + half] < target ? lo + half : lo;
      n -= half;
    }
    const int32_t Pz = P[lo], Pz1 = P[lo + 1];
    const Acc Qz = Q[lo];
    const int sz = L[lo].y & 0xFFFF;
    if constexpr (count) steps += rank_below<NW>(w0, w1, sz + 1) - u_s1;
    if (cur.ld > lo || (cur.ld == lo && Pz1 != target)) return Inf<Acc>::value;
    return S - (Qz - Q0) - xr_weight<Acc>(rc, T, sz) * (Acc)(target - Pz);
  }
  // Less stock: walk the gR setups while delta < 0 (a shortfall at a
  // remanufacture-only setup is infeasible, and so is any deficit left).
  // With surplus sg = A - need, xR = need + min(sg, 0), so the change of xR
  // is min(sg + delta, 0) - min(sg, 0).
  int last = T - 1;  // the difference lasts to the horizon unless it ends
  for (int r = r0; r < cur.nR; ++r) {
    const int2 e = L[r];
    const int sr = e.y & 0xFFFF;
    const int32_t sg = e.x, sn = sg + delta;
    if (!(e.y >> 16) && sn < 0) {
      if constexpr (count) steps += rank_below<NW>(w0, w1, sr + 1) - u_s1;
      return Inf<Acc>::value;
    }
    const int32_t dx = (sn < 0 ? sn : 0) - (sg < 0 ? sg : 0);
    S -= (Acc)rc.hR * (Acc)(T - sr) * (Acc)dx - (Acc)rc.dP * (Acc)dx;
    delta -= dx;
    if (delta == 0) {
      last = sr;
      break;
    }
  }
  if constexpr (count) steps += rank_below<NW>(w0, w1, last + 1) - u_s1;
  return cur.ld >= r0 ? Inf<Acc>::value : S;
}

// Row cost = S + C0 as int64 (ELSR_INF when infeasible).
template <typename Acc>
ELSR_HD int64_t row_cost(Acc S, int64_t C0) {
  return S == Inf<Acc>::value ? INT64_MAX : (int64_t)S + C0;
}

// Packed argmin key: cost in the top 40 bits (all ones = infeasible), move
// index in the low 24; a smaller key is a lexicographically smaller
// (cost, index).  Costs are below 2^40 - 1 by the create-time bound.
ELSR_HD uint64_t pack_key(int64_t cost, uint32_t idx) {
  const uint64_t c = (cost == INT64_MAX) ? 0xFFFFFFFFFFull : (uint64_t)cost;
  return (c << 24) | (uint64_t)(idx & 0xFFFFFFu);
}
ELSR_HD int64_t key_cost(uint64_t key) {
  const uint64_t c = key >> 24;
  return c == 0xFFFFFFFFFFull ? INT64_MAX : (int64_t)c;
}
ELSR_HD int key_index(uint64_t key) { return (int)(key & 0xFFFFFFu); }

// One splitmix64 step (Steele, Lea & Flood 2014): advance the state by the
// golden-ratio increment, then the published output mix.
ELSR_HD uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Shake draw j of strength k at iteration it (keyed by seed, iteration,
// neighbourhood and move).
ELSR_HD uint64_t shake_draw(uint64_t seed, uint64_t it, uint64_t k,
                            uint64_t j) {
  return splitmix64(splitmix64(splitmix64(seed) ^ it) ^ ((k << 32) | j));
}

}  // namespace elsr
