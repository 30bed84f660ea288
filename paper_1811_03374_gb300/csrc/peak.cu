// peak.cu -- FP32 FMA throughput microbenchmark, the measured cross-check of
// the FP32 FMA roofline (152 SMs x 128 lanes x 2 flop x clock) that the
// traversal's achieved arithmetic is reported against.
//
// Every thread runs eight independent FMA chains (enough to cover the FMA
// latency with a few warps per scheduler); the grid fills every SM.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace fx {
namespace {

constexpr int kPeakBlock = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ float g_peak_sink;

__global__ void __launch_bounds__(kPeakBlock) k_ffma(int iters, float seed) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed + 1e-3f * (float)(threadIdx.x + k);
  const float m = 0.999999f, b = 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, b);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s < 0.0f) g_peak_sink = s;  // never true (the chains stay positive); keeps them live
}

}  // namespace

cudaError_t fma_peak(int sm_count, int blocks_per_sm, int iters, float* ms, double* flops, cudaStream_t s) {
  const int grid = sm_count * blocks_per_sm;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  k_ffma<<<grid, kPeakBlock, 0, s>>>(iters, 1.0f);  // warm-up
  e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    k_ffma<<<grid, kPeakBlock, 0, s>>>(iters, 1.0f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  *flops = 2.0 * (double)grid * kPeakBlock * kChains * kUnroll * (double)iters;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace fx
