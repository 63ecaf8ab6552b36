// elsr_srv_inst.cu -- one instantiation of the serving kernel (srv_kernel in
// elsr_vns.cuh), selected by the build:
//   ELSR_INST_ACC  row accumulator type (int32_t or int64_t)
//   ELSR_INST_NW   64-bit words per setup-bit row (1: T <= 64, 2: T <= 128)
// The build compiles this file once per combination, in parallel.
#include "elsr_vns.cuh"

#if !defined(ELSR_INST_ACC) || !defined(ELSR_INST_NW)
#error "elsr_srv_inst.cu needs ELSR_INST_ACC and ELSR_INST_NW"
#endif

namespace elsr {

template cudaError_t srv_prepare_t<ELSR_INST_ACC, ELSR_INST_NW>(size_t, int, int, int*);
template cudaError_t srv_launch_t<ELSR_INST_ACC, ELSR_INST_NW>(const VnsParams&, const SrvQueue&,
                                                               int, int, size_t, int,
                                                               cudaStream_t);

}  // namespace elsr
