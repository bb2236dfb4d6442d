// The recording forward x-pass of the adjoint's segment recomputation: the
// plain x-pass that also writes the real-space states entering its B and A
// half steps (the forward states the reverse x-pass linearises about).
#include "kernels.cuh"

namespace brahms {

namespace {

template <int NX, int F>
cudaError_t launch_record(const XPassArgs& a, cudaStream_t s) {
  constexpr int ROWS = xpass_rows<NX>();
  constexpr int THREADS = xpass_threads<NX>();
  const size_t smem = (size_t)xpass_smem_floats2<NX>(F) * sizeof(float2);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(xpass_kernel<NX, F, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const long long grid = (a.rows + ROWS - 1) / ROWS;
  if (grid <= 0) return cudaSuccess;
  xpass_kernel<NX, F, false, true><<<(unsigned)grid, THREADS, smem, s>>>(a);
  return cudaPeekAtLastError();
}

}  // namespace

cudaError_t run_xpass_record(int nx, int nf, const XPassArgs& a, cudaStream_t s) {
  switch (nx) {
#define BRAHMS_XR_CASE(N) \
  case N:                 \
    return nf == 3 ? launch_record<N, 3>(a, s) : launch_record<N, 2>(a, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_XR_CASE)
#undef BRAHMS_XR_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace brahms
