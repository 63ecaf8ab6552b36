// Host build of the CUDA path's row arithmetic (elsr_row.cuh), for unit tests
// that compare its delta re-decode against the CPU oracle without a GPU.
// Test-only: the library never contains this file.
#include <stdint.h>
#include <string.h>
#include <vector>

#include "elsr_row.cuh"

using namespace elsr;

namespace {

template <typename Acc>
struct HostRow {
  int T;
  std::vector<int2> tab;
  RowCosts rc;
  int64_t C0;
  RowState<Acc> st;
  std::vector<int32_t> A;
  std::vector<Acc> C;
};

template <typename Acc>
void make_row(HostRow<Acc>& r, int T, const int32_t* D, const int32_t* R,
              const int32_t* costs, const uint8_t* gM, const uint8_t* gR) {
  r.T = T;
  r.tab.assign(T + 1, int2{0, 0});
  int32_t cd = 0, cr = 0;
  int64_t wd = 0, wr = 0;
  for (int t = 0; t < T; ++t) {
    r.tab[t].x = cd;
    cd += D[t];
    cr += R[t];
    r.tab[t].y = cr;
    wd += (int64_t)D[t] * (T - t);
    wr += (int64_t)R[t] * (T - t);
  }
  r.tab[T].x = cd;
  r.tab[T].y = cr;
  r.rc = RowCosts{costs[0], costs[1], costs[2], costs[3]};
  r.C0 = (int64_t)costs[3] * wr - (int64_t)costs[2] * wd;
  RowBits b{0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    if (gM[t]) flip(b.m0, b.m1, t);
    if (gR[t]) flip(b.r0, b.r1, t);
  }
  r.st.b = b;
  r.A.assign(T, 0);
  r.C.assign(T, 0);
  int segs = 0;
  r.st.S = build_row<Acc>(r.tab.data(), T, r.rc, b, r.A.data(), r.C.data(),
                          r.st.bad, segs);
}

template <typename Acc>
int64_t move_costs(int T, const int32_t* D, const int32_t* R,
                   const int32_t* costs, const uint8_t* gM, const uint8_t* gR,
                   int j, int64_t* out, int32_t* segs_out) {
  HostRow<Acc> r;
  make_row<Acc>(r, T, D, R, costs, gM, gR);
  const int M = row_moves(T, j);
  for (int m = 0; m < M; ++m) {
    int segs = 0;
    DeltaOut<Acc> d = eval_move<Acc, false>(r.tab.data(), T, r.rc, r.st,
                                            r.A.data(), r.C.data(), j, m, segs);
    out[m] = row_cost<Acc>(d.S, r.C0);
    segs_out[m] = segs;
  }
  return row_cost<Acc>(r.st.S, r.C0);
}

// Apply move m with the cache patch (WRITE walk + delta shift) and compare
// against a fresh decode.  Returns 0 if equal, 1 if not, -1 if not applicable.
template <typename Acc>
int apply_check(int T, const int32_t* D, const int32_t* R,
                const int32_t* costs, const uint8_t* gM, const uint8_t* gR,
                int j, int m) {
  HostRow<Acc> r;
  make_row<Acc>(r, T, D, R, costs, gM, gR);
  if (r.st.bad < T) return -1;
  int segs = 0;
  DeltaOut<Acc> d = eval_move<Acc, true>(r.tab.data(), T, r.rc, r.st,
                                         r.A.data(), r.C.data(), j, m, segs);
  if (d.S == Inf<Acc>::value) return -1;
  RowBits nb = r.st.b;
  apply_row_move(nb, T, j, m);
  const uint64_t u0 = nb.m0 | nb.r0, u1 = nb.m1 | nb.r1;
  for (int s = d.merge; s < T; ++s)
    if (bit_of(u0, u1, s)) r.C[s] += d.delta;
  std::vector<int32_t> A2(T, 0);
  std::vector<Acc> C2(T, 0);
  int bad2 = 0;
  Acc S2 = build_row<Acc>(r.tab.data(), T, r.rc, nb, A2.data(), C2.data(),
                          bad2, segs);
  if (S2 != d.S || bad2 != T) return 1;
  for (int s = 0; s < T; ++s)
    if (bit_of(u0, u1, s) && (A2[s] != r.A[s] || C2[s] != r.C[s])) return 1;
  return 0;
}

}  // namespace

extern "C" {

int64_t hc_move_costs(int32_t acc64, int32_t T, const int32_t* D,
                      const int32_t* R, const int32_t* costs,
                      const uint8_t* gM, const uint8_t* gR, int32_t j,
                      int64_t* out, int32_t* segs) {
  return acc64 ? move_costs<int64_t>(T, D, R, costs, gM, gR, j, out, segs)
               : move_costs<int32_t>(T, D, R, costs, gM, gR, j, out, segs);
}

int32_t hc_apply_check(int32_t acc64, int32_t T, const int32_t* D,
                       const int32_t* R, const int32_t* costs,
                       const uint8_t* gM, const uint8_t* gR, int32_t j,
                       int32_t m) {
  return acc64 ? apply_check<int64_t>(T, D, R, costs, gM, gR, j, m)
               : apply_check<int32_t>(T, D, R, costs, gM, gR, j, m);
}

uint64_t hc_shake_draw(uint64_t seed, uint64_t it, uint64_t k, uint64_t j) {
  return shake_draw(seed, it, k, j);
}

}
