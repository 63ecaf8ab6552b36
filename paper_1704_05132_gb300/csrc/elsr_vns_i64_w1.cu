// elsr_vns_i64_w1.cu -- instantiations of the GVNS kernels with int64_t row
// accumulators and 1 64-bit word(s) per setup-bit row (one translation unit
// per combination, built in parallel).
#include "elsr_vns.cuh"

namespace elsr {

template <bool TS>
static cudaError_t prep2(int maxt, size_t smem, int threads, int cluster, int* active) {
  if (maxt == 256) return vns_prepare_t<int64_t, 1, TS, 256>(smem, threads, cluster, active);
  if (maxt == 512) return vns_prepare_t<int64_t, 1, TS, 512>(smem, threads, cluster, active);
  return vns_prepare_t<int64_t, 1, TS, 1024>(smem, threads, cluster, active);
}

template <bool TS>
static cudaError_t launch2(int maxt, const VnsParams& p, int blocks, int threads, size_t smem,
                           int cluster, cudaStream_t s) {
  if (maxt == 256) return vns_launch_t<int64_t, 1, TS, 256>(p, blocks, threads, smem, cluster, s);
  if (maxt == 512) return vns_launch_t<int64_t, 1, TS, 512>(p, blocks, threads, smem, cluster, s);
  return vns_launch_t<int64_t, 1, TS, 1024>(p, blocks, threads, smem, cluster, s);
}

cudaError_t vns_prepare_i64_w1(bool ts, int maxt, size_t smem, int threads, int cluster,
                                  int* active) {
  return ts ? prep2<true>(maxt, smem, threads, cluster, active)
            : prep2<false>(maxt, smem, threads, cluster, active);
}

cudaError_t vns_launch_i64_w1(bool ts, int maxt, const VnsParams& p, int blocks,
                                 int threads, size_t smem, int cluster, cudaStream_t s) {
  return ts ? launch2<true>(maxt, p, blocks, threads, smem, cluster, s)
            : launch2<false>(maxt, p, blocks, threads, smem, cluster, s);
}

}  // namespace elsr
