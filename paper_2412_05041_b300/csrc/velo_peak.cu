// FP32 ALU ceiling of the current device, measured (velo_measure_fp32_peak).
//
// The reconstruction has no dense contraction: its second ceiling after HBM
// bandwidth is the plain FP32 pipe.  This microbenchmark keeps every SM's
// FMA pipes busy with independent multiply-add chains (8 per thread, 8 warps
// per scheduler, no memory traffic inside the timed loop) and reports
// 2 flops per FMA over the CUDA-event time of the launch.
#include <cuda_runtime.h>

#include "velo.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;
constexpr int kIters = 2048;

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float* sink, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
  const float m = 0.999999f, k = 1e-7f;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], m, k);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678f) sink[blockIdx.x] = s;  // never true: keeps the chains alive
}

}  // namespace

extern "C" int velo_measure_fp32_peak(double* flops_per_s, void* stream) {
  if (!flops_per_s) return VELO_EINVAL;
  *flops_per_s = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return VELO_ECUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = sms * 8;  // 2048 threads per SM
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaMalloc(&sink, sizeof(float) * blocks) == cudaSuccess;
  ok = ok && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  float best_ms = 0.0f;
  for (int rep = 0; ok && rep < 4; ++rep) {  // the first launch warms up
    ok = cudaEventRecord(e0, s) == cudaSuccess;
    k_fma_peak<<<blocks, kPeakThreads, 0, s>>>(sink, 1.0f);
    ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.0f;
    ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (ok && rep > 0 && (best_ms == 0.0f || ms < best_ms)) best_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (!ok || best_ms <= 0.0f || cudaGetLastError() != cudaSuccess) return VELO_ECUDA;
  const double flops = 2.0 * kChains * (double)kIters * kPeakThreads * blocks;
  *flops_per_s = flops / (best_ms * 1e-3);
  return VELO_OK;
}
