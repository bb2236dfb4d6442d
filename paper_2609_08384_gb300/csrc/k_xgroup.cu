// Grouped x-pass of the batched form: one launch applies the same x-pass
// (inverse x-FFT, the RK4 half steps, forward x-FFT) to every active instance
// of one grid shape.  The instances of a shape lie one after another in one
// array ([instance][field][tau][y][x]), so instance i's field f starts at
// (2 i + f) fstride.  Each CTA's rows belong to one instance (the rows of an
// instance are a whole number of CTA tiles), whose step size, coupling and
// mismatch come from a per-instance table and its stage factors from a table
// formed on the host as the single-instance path forms them; the mode
// (middle or last x-pass of the instance's propagation) follows from its
// step count.
#include "kernels.cuh"
#include "launch_cfg.h"

namespace brahms {

template <int NX>
__global__ void __launch_bounds__(xpass_threads<NX>(), xpass_min_blocks<NX, 2>())
    xpass_group_kernel(const XPassArgs base, const GroupInst* __restrict__ gi, const float2* __restrict__ ecoef,
                       int stride, int step, long long tiles_per_inst) {
  constexpr int THREADS = xpass_threads<NX>();
  extern __shared__ float4 sm4[];
  float2* coef = reinterpret_cast<float2*>(sm4);
  float2* rowbuf = coef + 6 * 2;
  // tiles from the last down, as the single-instance x-pass
  const long long t = (long long)gridDim.x - 1 - blockIdx.x;
  const int i = (int)(t / tiles_per_inst);
  const long long lt = t - (long long)i * tiles_per_inst;
  const GroupInst g = gi[i];
  XPassArgs p = base;
  p.data = base.data + (long long)i * 2 * base.fstride;
  p.dz = g.dz;
  p.kh[0] = g.kh[0];
  p.kh[1] = g.kh[1];
  p.kh2[0] = g.kh2[0];
  p.kh2[1] = g.kh2[1];
  p.mode = step < 0 ? XM_NL_FIRST : (step == g.nz - 1 ? XM_NL_LAST : XM_NL_MID);
  if (threadIdx.x < 6) coef[threadIdx.x] = ecoef[(long long)i * stride + (step + 1) * 6 + threadIdx.x];
  __syncthreads();
  xpass_tile<NX, 2, THREADS>(p, lt, coef, rowbuf);
}

template <int NX>
static cudaError_t launch_group(const XPassArgs& base, const GroupInst* gi, const float2* ecoef, int stride, int step,
                                int ninst, cudaStream_t s) {
  constexpr int ROWS = xpass_rows<NX>();
  constexpr int THREADS = xpass_threads<NX>();
  const size_t smem = (size_t)xpass_smem_floats2<NX>(2) * sizeof(float2);
  static SmemOnce once;
  cudaError_t e = raise_smem_limit(xpass_group_kernel<NX>, smem, once);
  if (e != cudaSuccess) return e;
  if (base.rows % ROWS != 0) return cudaErrorInvalidValue;  // an instance's rows must fill whole CTAs
  const long long tiles = base.rows / ROWS;
  const long long grid = tiles * ninst;
  if (grid <= 0) return cudaSuccess;
  xpass_group_kernel<NX><<<(unsigned)grid, THREADS, smem, s>>>(base, gi, ecoef, stride, step, tiles);
  return cudaPeekAtLastError();
}

cudaError_t run_xpass_group(int nx, const XPassArgs& base, const GroupInst* gi, const float2* ecoef, int stride,
                            int step, int ninst, cudaStream_t s) {
  switch (nx) {
#define BRAHMS_G_CASE(N) \
  case N:                \
    return launch_group<N>(base, gi, ecoef, stride, step, ninst, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_G_CASE)
#undef BRAHMS_G_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

int xpass_rows_of(int nx) {
  switch (nx) {
#define BRAHMS_R2_CASE(N) \
  case N:                 \
    return xpass_rows<N>();
    BRAHMS_FOR_EACH_SIZE(BRAHMS_R2_CASE)
#undef BRAHMS_R2_CASE
    default:
      return 0;
  }
}

}  // namespace brahms
