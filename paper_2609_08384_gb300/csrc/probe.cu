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

// ---------------------------------------------------------------------------
// All-to-all exchange rate of distributed shared memory within a thread-block
// cluster: the exchange a step that kept whole (x, y) planes on chip would
// make twice per plane.  Each CTA of a cluster holds `smem_bytes` of shared
// memory cut into C chunks; per round it sends chunk j to CTA j's slot for it
// (remote stores through the cluster's shared window), then the cluster
// synchronises.  The rate counts the bytes that cross to other CTAs.
#include <cooperative_groups.h>

namespace {

namespace cg = cooperative_groups;

template <int C>
__global__ void dsmem_a2a_kernel(int rounds, int nf4, float* never) {
  extern __shared__ float4 buf[];
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const int chunk = nf4 / C;
  for (int i = threadIdx.x; i < nf4; i += blockDim.x) buf[i] = make_float4((float)r, (float)i, 0.f, 1.f);
  cl.sync();
  float acc = 0.f;
  for (int it = 0; it < rounds; ++it) {
    for (int j = 1; j < C; ++j) {
      const int dst = (r + j) % C;
      float4* remote = cl.map_shared_rank(buf, dst);
      for (int o = threadIdx.x; o < chunk; o += blockDim.x) {
        const float4 v = buf[dst * chunk + o];
        acc += v.w;
        remote[r * chunk + o] = v;
      }
    }
    cl.sync();  // every remote store of this round has landed before the next reads
  }
  if (acc < 0.f) never[threadIdx.x] = acc;
}

template <int C>
brahms_status dsmem_rate(int smem_bytes, cudaStream_t s, double* tbps) {
  const int nf4 = smem_bytes / 16 / C * C;
  if (nf4 < C) return BRAHMS_E_ARG;
  const size_t smem = (size_t)nf4 * 16;
  if (cudaFuncSetAttribute(dsmem_a2a_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return BRAHMS_E_CUDA;
  if (C > 8 && cudaFuncSetAttribute(dsmem_a2a_kernel<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                   cudaSuccess)
    return BRAHMS_E_CUDA;
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.gridDim = dim3(C);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, dsmem_a2a_kernel<C>, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return BRAHMS_E_SIZE;  // no cluster of this shape fits
  }
  cfg.gridDim = dim3(C * clusters);  // one resident wave
  const int rounds = 200;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BRAHMS_E_CUDA;
  brahms_status st = BRAHMS_OK;
  if (cudaLaunchKernelEx(&cfg, dsmem_a2a_kernel<C>, 10, nf4, (float*)nullptr) != cudaSuccess) st = BRAHMS_E_CUDA;
  cudaEventRecord(e0, s);
  if (st == BRAHMS_OK && cudaLaunchKernelEx(&cfg, dsmem_a2a_kernel<C>, rounds, nf4, (float*)nullptr) != cudaSuccess)
    st = BRAHMS_E_CUDA;
  cudaEventRecord(e1, s);
  float ms = 0.f;
  if (st == BRAHMS_OK &&
      (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)))
    st = BRAHMS_E_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BRAHMS_OK) return st;
  const double remote = (double)cfg.gridDim.x * nf4 * 16.0 * (C - 1) / C * rounds;
  *tbps = remote / (ms * 1e-3) / 1e12;
  return BRAHMS_OK;
}

}  // namespace

extern "C" brahms_status brahms_dsmem_exchange_rate(int cluster_ctas, int smem_bytes, void* cuda_stream,
                                                    double* tbps) {
  if (!tbps || smem_bytes < 1024 || smem_bytes > 227 * 1024) return BRAHMS_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  switch (cluster_ctas) {
    case 2: return dsmem_rate<2>(smem_bytes, s, tbps);
    case 4: return dsmem_rate<4>(smem_bytes, s, tbps);
    case 8: return dsmem_rate<8>(smem_bytes, s, tbps);
    case 16: return dsmem_rate<16>(smem_bytes, s, tbps);
    default: return BRAHMS_E_ARG;
  }
}
