// FP32 fused multiply-add rate of the current GPU, measured: the denominator
// of the ALU view of the roofline (the copy bandwidth and the tensor rates
// are measured elsewhere; nothing publishes this one for GB300).
//
// Every thread runs kChains independent dependency chains a <- a * b + c
// (the chains converge to c / (1 - b) = 1, so no value leaves the normal
// range) for `iters` iterations; the grid is several resident waves of
// 256-thread CTAs on every SM.  The result is stored only if it is negative,
// which never happens but which the compiler cannot rule out, so no FMA is
// removed.  Time: CUDA events on the caller's stream around one launch,
// after one warm-up launch.
#include <cuda_runtime.h>

#include "brahms.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_rate_kernel(int iters, float b, float c, float* never) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 0.5f + 0.01f * (float)k + 1e-6f * (float)(threadIdx.x & 7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s < 0.f) never[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" brahms_status brahms_fp32_fma_rate(void* cuda_stream, double* tflops) {
  if (!tflops) return BRAHMS_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate_kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
    return BRAHMS_E_CUDA;
  const int blocks = sms * per_sm * 4;  // four resident waves
  const int iters = 1 << 14;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BRAHMS_E_CUDA;
  fma_rate_kernel<<<blocks, kThreads, 0, s>>>(iters / 8, 0.999f, 0.001f, nullptr);
  cudaEventRecord(e0, s);
  fma_rate_kernel<<<blocks, kThreads, 0, s>>>(iters, 0.999f, 0.001f, nullptr);
  cudaEventRecord(e1, s);
  brahms_status st = BRAHMS_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
    st = BRAHMS_E_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BRAHMS_OK) return st;
  const double flops = 2.0 * (double)kChains * iters * (double)blocks * kThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return BRAHMS_OK;
}
