// elsr_probe.cu -- integer-issue probe: the rate at which the GPU retires
// 32-bit integer operations of the kinds a decode step is made of (add,
// minimum, logic, multiply-add), measured instead of taken from unit counts.
// It is the denominator of the integer roofline that the benchmark reports
// for the GVNS kernels; it computes nothing of the method.
//
// Every thread runs eight independent chains (enough independent work per
// warp to keep the pipes busy), each step of a chain doing one add, one
// minimum, one exclusive-or and one multiply-add on operands loaded at run
// time, so nothing folds at compile time; the chains' sum is stored so that
// nothing is dead.
#include <cuda_runtime.h>
#include <stdint.h>

#include "elsr.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kOpsPerStep = 4;  // add, min, xor, multiply-add

__global__ void __launch_bounds__(256) int_issue_kernel(const int32_t* __restrict__ src,
                                                        int32_t iters, int32_t* __restrict__ sink) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = src[(tid + c) & 31];
  const int32_t y = src[32], z = src[33], w = src[34], m = src[35];
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        int32_t v = x[c] + y;
        v = v < z ? v : z;
        v ^= w;
        x[c] = v * m + x[(c + 1) % kChains];
      }
    }
  }
  int32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  sink[tid] = s;
}

}  // namespace

extern "C" int elsr_int_issue_probe(void* stream, int32_t blocks, int32_t iters,
                                    const int32_t* src, int32_t* sink, int64_t* ops) {
  if (blocks <= 0 || iters <= 0 || !src || !sink || !ops) return ELSR_E_ARG;
  const int threads = 256;
  int_issue_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(src, iters, sink);
  if (cudaGetLastError() != cudaSuccess) return ELSR_E_CUDA;
  *ops = (int64_t)blocks * threads * iters * kUnroll * kChains * kOpsPerStep;
  return ELSR_OK;
}
