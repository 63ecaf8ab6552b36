// elsr_vns_dispatch.cu -- run-time choice among the compiled instantiations
// of the persistent GVNS kernels and the serving kernel (each lives in its own object built from
// elsr_vns_inst.cu; only their declarations are visible here).
#include "elsr_internal.h"

namespace elsr {

namespace {

template <typename Acc, int NW, bool TS>
cudaError_t prepare_m(int maxt, size_t smem, int threads, int cluster, int* active) {
  if (maxt == 256) return vns_prepare_t<Acc, NW, TS, 256>(smem, threads, cluster, active);
  if (maxt == 512) return vns_prepare_t<Acc, NW, TS, 512>(smem, threads, cluster, active);
  return vns_prepare_t<Acc, NW, TS, 1024>(smem, threads, cluster, active);
}

template <typename Acc, int NW, bool TS>
cudaError_t launch_m(int maxt, const VnsParams& p, int blocks, int threads, size_t smem,
                     int cluster, cudaStream_t s) {
  if (maxt == 256) return vns_launch_t<Acc, NW, TS, 256>(p, blocks, threads, smem, cluster, s);
  if (maxt == 512) return vns_launch_t<Acc, NW, TS, 512>(p, blocks, threads, smem, cluster, s);
  return vns_launch_t<Acc, NW, TS, 1024>(p, blocks, threads, smem, cluster, s);
}

template <typename Acc>
cudaError_t prepare_a(int nw, bool ts, int maxt, size_t smem, int threads, int cluster,
                      int* active) {
  if (nw == 1)
    return ts ? prepare_m<Acc, 1, true>(maxt, smem, threads, cluster, active)
              : prepare_m<Acc, 1, false>(maxt, smem, threads, cluster, active);
  return ts ? prepare_m<Acc, 2, true>(maxt, smem, threads, cluster, active)
            : prepare_m<Acc, 2, false>(maxt, smem, threads, cluster, active);
}

template <typename Acc>
cudaError_t launch_a(int nw, bool ts, int maxt, const VnsParams& p, int blocks, int threads,
                     size_t smem, int cluster, cudaStream_t s) {
  if (nw == 1)
    return ts ? launch_m<Acc, 1, true>(maxt, p, blocks, threads, smem, cluster, s)
              : launch_m<Acc, 1, false>(maxt, p, blocks, threads, smem, cluster, s);
  return ts ? launch_m<Acc, 2, true>(maxt, p, blocks, threads, smem, cluster, s)
            : launch_m<Acc, 2, false>(maxt, p, blocks, threads, smem, cluster, s);
}

}  // namespace

cudaError_t vns_prepare(bool acc64, int nw, bool ts, int maxt, size_t smem, int threads,
                        int cluster, int* active) {
  return acc64 ? prepare_a<int64_t>(nw, ts, maxt, smem, threads, cluster, active)
               : prepare_a<int32_t>(nw, ts, maxt, smem, threads, cluster, active);
}

cudaError_t vns_launch(bool acc64, int nw, bool ts, int maxt, const VnsParams& p,
                       int blocks, int threads, size_t smem, int cluster, cudaStream_t s) {
  return acc64 ? launch_a<int64_t>(nw, ts, maxt, p, blocks, threads, smem, cluster, s)
               : launch_a<int32_t>(nw, ts, maxt, p, blocks, threads, smem, cluster, s);
}

cudaError_t srv_prepare(bool acc64, int nw, size_t smem, int threads, int cluster, int* active) {
  if (acc64)
    return nw == 1 ? srv_prepare_t<int64_t, 1>(smem, threads, cluster, active)
                   : srv_prepare_t<int64_t, 2>(smem, threads, cluster, active);
  return nw == 1 ? srv_prepare_t<int32_t, 1>(smem, threads, cluster, active)
                 : srv_prepare_t<int32_t, 2>(smem, threads, cluster, active);
}

cudaError_t srv_launch(bool acc64, int nw, const VnsParams& p, const SrvQueue& q, int blocks,
                       int threads, size_t smem, int cluster, cudaStream_t s) {
  if (acc64)
    return nw == 1 ? srv_launch_t<int64_t, 1>(p, q, blocks, threads, smem, cluster, s)
                   : srv_launch_t<int64_t, 2>(p, q, blocks, threads, smem, cluster, s);
  return nw == 1 ? srv_launch_t<int32_t, 1>(p, q, blocks, threads, smem, cluster, s)
                 : srv_launch_t<int32_t, 2>(p, q, blocks, threads, smem, cluster, s);
}

}  // namespace elsr
