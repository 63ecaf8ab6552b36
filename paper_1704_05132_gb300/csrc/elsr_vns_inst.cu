// elsr_vns_inst.cu -- one instantiation of the persistent GVNS kernels
// (batched, speculative and fork-join), selected by the build:
//   ELSR_INST_ACC  row accumulator type (int32_t or int64_t)
//   ELSR_INST_NW   64-bit words per setup-bit row (1: T <= 64, 2: T <= 128)
//   ELSR_INST_TS   prefix tables in shared memory (1) or global memory (0)
//   ELSR_INST_MAXT block size bound (256, 512 or 1024)
// The build compiles this file once per combination, in parallel.
#include "elsr_vns.cuh"

#if !defined(ELSR_INST_ACC) || !defined(ELSR_INST_NW) || !defined(ELSR_INST_TS) || \
    !defined(ELSR_INST_MAXT)
#error "elsr_vns_inst.cu needs ELSR_INST_ACC, ELSR_INST_NW, ELSR_INST_TS and ELSR_INST_MAXT"
#endif

namespace elsr {

template cudaError_t vns_prepare_t<ELSR_INST_ACC, ELSR_INST_NW, (bool)ELSR_INST_TS,
                                   ELSR_INST_MAXT>(size_t, int, int, int*);
template cudaError_t vns_launch_t<ELSR_INST_ACC, ELSR_INST_NW, (bool)ELSR_INST_TS,
                                  ELSR_INST_MAXT>(const VnsParams&, int, int, size_t, int,
                                                  cudaStream_t);

}  // namespace elsr
