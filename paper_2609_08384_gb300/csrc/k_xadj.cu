// The reverse x-pass of the adjoint (kernel in xadj.cuh): map-free
// instantiations, dispatch, and the fixed-order reduction of the per-CTA
// stage-phase sensitivities.
#include "xadj.cuh"

namespace brahms {

__global__ void __launch_bounds__(256) sens_boundary_kernel(const double* __restrict__ partial, long long ncta,
                                                            double* sensA, double* sensB) {
  __shared__ double red[8][6];
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long c = threadIdx.x; c < ncta; c += blockDim.x)
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] += partial[c * 6 + k];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    if (threadIdx.x < 3) {
      if (sensA) sensA[threadIdx.x] = s;
    } else if (sensB) {
      sensB[threadIdx.x - 3] = s;
    }
  }
}


cudaError_t run_xpass_adjoint(int nx, int nf, const XAdjArgs& a, long long* ncta, cudaStream_t s) {
  if (a.emap) return run_xpass_adjoint_map(nx, nf, a, ncta, s);
  switch (nx) {
#define BRAHMS_XA_CASE(N) \
  case N:                 \
    return nf == 3 ? launch_adjoint<N, 3, false>(a, ncta, s) : launch_adjoint<N, 2, false>(a, ncta, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_XA_CASE)
#undef BRAHMS_XA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

long long xpass_adjoint_ctas(int nx, long long rows) {
  switch (nx) {
#define BRAHMS_XC_CASE(N) \
  case N:                 \
    return (rows + xpass_rows<N>() - 1) / xpass_rows<N>();
    BRAHMS_FOR_EACH_SIZE(BRAHMS_XC_CASE)
#undef BRAHMS_XC_CASE
    default:
      return 0;
  }
}

cudaError_t run_sens_boundary(const double* partial, long long ncta, double* sensA, double* sensB, cudaStream_t s) {
  sens_boundary_kernel<<<1, 256, 0, s>>>(partial, ncta, sensA, sensB);
  return cudaPeekAtLastError();
}

}  // namespace brahms
