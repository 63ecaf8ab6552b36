// elsr_vns_i32.cu -- instantiations of the persistent GVNS kernel with
// int32_t row accumulators (one translation unit per width, built in parallel).
#include "elsr_vns.cuh"

namespace elsr {

namespace {

template <int NW, bool TS>
cudaError_t prep2(int maxt, size_t smem, int threads, int cluster, int* active) {
  return maxt == 256 ? vns_prepare_t<int32_t, NW, TS, 256>(smem, threads, cluster, active)
                     : vns_prepare_t<int32_t, NW, TS, 1024>(smem, threads, cluster, active);
}

template <int NW, bool TS>
cudaError_t launch2(int maxt, const VnsParams& p, int blocks, int threads, size_t smem,
                    int cluster, cudaStream_t s) {
  return maxt == 256 ? vns_launch_t<int32_t, NW, TS, 256>(p, blocks, threads, smem, cluster, s)
                     : vns_launch_t<int32_t, NW, TS, 1024>(p, blocks, threads, smem, cluster, s);
}

}  // namespace

cudaError_t vns_prepare_i32(int nw, bool ts, int maxt, size_t smem, int threads,
                            int cluster, int* active) {
  if (nw == 1)
    return ts ? prep2<1, true>(maxt, smem, threads, cluster, active)
              : prep2<1, false>(maxt, smem, threads, cluster, active);
  return ts ? prep2<2, true>(maxt, smem, threads, cluster, active)
            : prep2<2, false>(maxt, smem, threads, cluster, active);
}

cudaError_t vns_launch_i32(int nw, bool ts, int maxt, const VnsParams& p, int blocks,
                           int threads, size_t smem, int cluster, cudaStream_t s) {
  if (nw == 1)
    return ts ? launch2<1, true>(maxt, p, blocks, threads, smem, cluster, s)
              : launch2<1, false>(maxt, p, blocks, threads, smem, cluster, s);
  return ts ? launch2<2, true>(maxt, p, blocks, threads, smem, cluster, s)
            : launch2<2, false>(maxt, p, blocks, threads, smem, cluster, s);
}

}  // namespace elsr
