// The reverse x-pass of the adjoint (kernel in xadj.cuh): map-free
// instantiations, dispatch, and the fixed-order reduction of the per-CTA
// stage-phase sensitivities.
#include <cmath>

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


// i kappa_f h e^{-/+ i Phi} at the start, middle and end of a half step that
// starts at phase phi_a with mismatch dk: the phase in FP64, reduced mod 2 pi,
// cos and sin in FP64 rounded to float (the forward x-pass's stage factors),
// the products with kappa_f h in float as the device forms them
static void coef_sets(double phi_a, double dk, double h, const float* kh, int nf, float2* c) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int s = 0; s < 3; ++s) {
    const double phi = phi_a + dk * (0.5 * h * s);
    const double r = phi - two_pi * std::rint(phi / two_pi);
    const float2 em = make_float2((float)std::cos(r), -(float)std::sin(r));  // e^{-i Phi}
    for (int f = 0; f < nf; ++f) {
      const float k = kh[f];
      c[s * nf + f] = f == 0 ? make_float2(-em.y * k, em.x * k) : make_float2(em.y * k, em.x * k);
    }
  }
}

cudaError_t run_xpass_adjoint(int nx, int nf, const XAdjArgs& a0, long long* ncta, cudaStream_t s) {
  if (a0.emap) return run_xpass_adjoint_map(nx, nf, a0, ncta, s);
  XAdjArgs a = a0;
  coef_sets(a.phiA, a.dkA, a.h, a.kh, nf, a.cset[0]);
  coef_sets(a.phiB, a.dkB, a.h, a.kh, nf, a.cset[1]);
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
