// Host build of the CUDA path's row arithmetic (elsr_row.cuh), for unit tests
// that compare its delta re-decode against the CPU oracle without a GPU.
// Test-only: the library never contains this file.
#include <stdint.h>
#include <string.h>
#include <vector>

#include "elsr_row.cuh"

using namespace elsr;

namespace {

template <typename Acc, int NW>
int64_t move_costs(int T, const int32_t* D, const int32_t* R,
                   const int32_t* costs, const uint8_t* gM, const uint8_t* gR,
                   int j, int64_t* out, int32_t* steps_out) {
  std::vector<int2> tab(T + 1, int2{0, 0});
  int32_t cd = 0, cr = 0;
  int64_t wd = 0, wr = 0;
  for (int t = 0; t < T; ++t) {
    tab[t].x = cd;
    cd += D[t];
    cr += R[t];
    tab[t].y = cr;
    wd += (int64_t)D[t] * (T - t);
    wr += (int64_t)R[t] * (T - t);
  }
  tab[T].x = cd;
  tab[T].y = cr;
  // costs: kM, kR, hM, hR, pM, pR
  const RowCosts rc{costs[0], costs[1], costs[2], costs[3], costs[5] - costs[4]};
  const int64_t C0 = (int64_t)costs[3] * wr - (int64_t)costs[2] * wd + (int64_t)costs[4] * cd;
  RowState<Acc> st;
  st.b = RowBits{0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    if (gM[t]) flip(st.b.m0, st.b.m1, t);
    if (gR[t]) flip(st.b.r0, st.b.r1, t);
  }
  std::vector<int32_t> A(T, 0);
  std::vector<Acc> C(T, 0);
  std::vector<int2> L(T, int2{0, 0});
  std::vector<int32_t> Pv(T + 1, 0);
  std::vector<Acc> Qv(T + 1, 0);
  int segs = 0;
  st.S = build_row<Acc, NW>(tab.data(), T, rc, st.b, A.data(), C.data(), L.data(),
                            Pv.data(), Qv.data(), st.bad, st.nR, st.ld, segs);
  const int M = row_moves(T, j);
  for (int m = 0; m < M; ++m) {
    int steps = 0;
    const Acc S = eval_move<Acc, NW>(tab.data(), T, rc, st, A.data(), C.data(),
                                     L.data(), Pv.data(), Qv.data(), j, m, steps);
    out[m] = row_cost<Acc>(S, C0);
    steps_out[m] = steps;
  }
  return state_cost<Acc>(st.S, st.bad, T, C0);
}

}  // namespace

extern "C" {

int64_t hc_move_costs(int32_t acc64, int32_t nw, int32_t T, const int32_t* D,
                      const int32_t* R, const int32_t* costs,
                      const uint8_t* gM, const uint8_t* gR, int32_t j,
                      int64_t* out, int32_t* steps) {
  if (nw == 1)
    return acc64 ? move_costs<int64_t, 1>(T, D, R, costs, gM, gR, j, out, steps)
                 : move_costs<int32_t, 1>(T, D, R, costs, gM, gR, j, out, steps);
  return acc64 ? move_costs<int64_t, 2>(T, D, R, costs, gM, gR, j, out, steps)
               : move_costs<int32_t, 2>(T, D, R, costs, gM, gR, j, out, steps);
}

// Local N3 indices of the non-null swaps of a row, by rank; returns their
// number.
int32_t hc_swaps(int32_t nw, int32_t T, const uint8_t* gM, const uint8_t* gR,
                 int32_t* out) {
  RowBits b{0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    if (gM[t]) flip(b.m0, b.m1, t);
    if (gR[t]) flip(b.r0, b.r1, t);
  }
  if (nw == 1) {
    const SwapMasks s = swap_masks<1>(b, T);
    for (int i = 0; i < s.n; ++i) out[i] = swap_of_rank<1>(s, T, i);
    return s.n;
  }
  const SwapMasks s = swap_masks<2>(b, T);
  for (int i = 0; i < s.n; ++i) out[i] = swap_of_rank<2>(s, T, i);
  return s.n;
}

uint64_t hc_shake_draw(uint64_t seed, uint64_t it, uint64_t k, uint64_t j) {
  return shake_draw(seed, it, k, j);
}

}
