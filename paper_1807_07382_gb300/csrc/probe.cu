// Throughput probe of the FP64 pipe: the denominator of the FP64 solves' compute
// roofline.  The paper has no counterpart; it measures the GPU at hand.
//
// Every thread runs eight independent chains of fused multiply-adds (enough
// independent work per warp to keep the pipe busy at any occupancy), so the
// kernel's rate is the pipe's issue rate times two flops per FMA.
#include <cstdint>

#include "../../include/pentbatch.h"

namespace pent {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_probe_fp64(int64_t iters, double seed, double* sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double m = 0.999999, k = 1e-7;  // a <- a m + k stays bounded
#pragma unroll 1
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.0) *sink = s;  // never true for these values; keeps the chains alive
}

}  // namespace
}  // namespace pent

extern "C" pent_status pent_probe_fp64_fma(int64_t blocks, int64_t iters, double* d_sink, void* cuda_stream,
                                           double* flops) {
  if (blocks < 1 || blocks > (int64_t)INT32_MAX || iters < 1 || !d_sink || !flops) return PENT_EINVAL;
  if (((uintptr_t)d_sink) % sizeof(double)) return PENT_EINVAL;
  pent::k_probe_fp64<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(iters, 0.5, d_sink);
  *flops = 2.0 * (double)blocks * 256.0 * (double)iters * 16.0 * pent::kChains;
  return cudaGetLastError() == cudaSuccess ? PENT_OK : PENT_ECUDA;
}
