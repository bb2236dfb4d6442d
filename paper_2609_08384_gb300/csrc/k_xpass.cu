// x-pass instantiations and dispatch.
#include <cmath>

#include "kernels.cuh"
#include "launch_cfg.h"

namespace brahms {

void fill_stage_factors(XPassArgs& a) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int s = 0; s < 6; ++s) {
    const double phi = s < 3 ? a.phiB + a.dkB * (0.5 * a.dz + 0.25 * a.dz * s) : a.phiA + a.dkA * (0.25 * a.dz * (s - 3));
    const double r = phi - two_pi * std::rint(phi / two_pi);
    a.ecoef[s] = make_float2((float)std::cos(r), (float)std::sin(r));
  }
}

template <int NX, int F, bool MAP>
static cudaError_t launch_x_variant(const XPassArgs& a0, cudaStream_t s) {
  XPassArgs a = a0;
  fill_stage_factors(a);
  constexpr int ROWS = xpass_rows<NX>();
  constexpr int THREADS = xpass_threads<NX>();
  const size_t smem = (size_t)xpass_smem_floats2<NX>(F) * sizeof(float2);
  static SmemOnce once;
  cudaError_t e = raise_smem_limit(xpass_kernel<NX, F, MAP>, smem, once);
  if (e != cudaSuccess) return e;
  const long long grid = (a.rows + ROWS - 1) / ROWS;
  if (grid <= 0) return cudaSuccess;
  xpass_kernel<NX, F, MAP><<<(unsigned)grid, THREADS, smem, s>>>(a);
  return cudaPeekAtLastError();
}

template <int NX, int F>
static cudaError_t launch_x(const XPassArgs& a, cudaStream_t s) {
  return a.emap ? launch_x_variant<NX, F, true>(a, s) : launch_x_variant<NX, F, false>(a, s);
}

cudaError_t run_xpass(int nx, int nf, const XPassArgs& a, cudaStream_t s) {
  switch (nx) {
#define BRAHMS_X_CASE(N) \
  case N:                \
    return nf == 3 ? launch_x<N, 3>(a, s) : launch_x<N, 2>(a, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_X_CASE)
#undef BRAHMS_X_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

bool size_supported(int n) {
  switch (n) {
#define BRAHMS_S_CASE(N) case N:
    BRAHMS_FOR_EACH_SIZE(BRAHMS_S_CASE)
#undef BRAHMS_S_CASE
    return true;
    default:
      return false;
  }
}

}  // namespace brahms
