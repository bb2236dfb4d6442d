// x-pass instantiations and dispatch.
#include "kernels.cuh"
#include "launch_cfg.h"

namespace brahms {

template <int NX, int F, bool MAP>
static cudaError_t launch_x_variant(const XPassArgs& a, cudaStream_t s) {
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
