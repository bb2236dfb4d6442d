// y-pass and tau-pass instantiations and dispatch.
#include "kernels.cuh"

namespace brahms {

template <class K>
static cudaError_t set_smem(K kernel, size_t smem, bool& configured) {
  if (configured) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) configured = true;
  return e;
}

template <int N, bool INV, int AXIS>
static cudaError_t launch_axis(const AxisArgs& a, cudaStream_t s) {
  using PL = FftPlan<N>;
  constexpr int TPC = tiles_per_cta<PL>();
  constexpr int THREADS = TPC * tile_threads<PL>();
  const size_t smem = (size_t)axis_smem_floats2<PL>() * sizeof(float2);
  static bool configured = false;
  cudaError_t e = set_smem(axis_fft_kernel<PL, INV, AXIS>, smem, configured);
  if (e != cudaSuccess) return e;
  const long long grid = (a.ntiles + TPC - 1) / TPC;
  if (grid <= 0) return cudaSuccess;
  axis_fft_kernel<PL, INV, AXIS><<<(unsigned)grid, THREADS, smem, s>>>(a);
  return cudaPeekAtLastError();
}

template <int N>
static cudaError_t launch_tprop(const AxisArgs& a, cudaStream_t s) {
  using PL = TauPlan<N>;
  constexpr int TPC = tiles_per_cta<PL>();
  constexpr int THREADS = TPC * tile_threads<PL>();
  const size_t smem = (size_t)axis_smem_floats2<PL>() * sizeof(float2);
  static bool configured = false;
  cudaError_t e = set_smem(tpass_prop_kernel<PL>, smem, configured);
  if (e != cudaSuccess) return e;
  const long long grid = (a.ntiles + TPC - 1) / TPC;
  if (grid <= 0) return cudaSuccess;
  tpass_prop_kernel<PL><<<(unsigned)grid, THREADS, smem, s>>>(a);
  return cudaPeekAtLastError();
}

cudaError_t run_axis_fft(int n, int axis, bool inv, const AxisArgs& a, cudaStream_t s) {
  switch (n) {
#define BRAHMS_A_CASE(N)                                                        \
  case N:                                                                       \
    if (axis == 1) return inv ? launch_axis<N, true, 1>(a, s) : launch_axis<N, false, 1>(a, s); \
    return inv ? launch_axis<N, true, 2>(a, s) : launch_axis<N, false, 2>(a, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_A_CASE)
#undef BRAHMS_A_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t run_tpass_prop(int nt, const AxisArgs& a, cudaStream_t s) {
  switch (nt) {
#define BRAHMS_T_CASE(N) \
  case N:                \
    return launch_tprop<N>(a, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_T_CASE)
#undef BRAHMS_T_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

int col_tile_of(int n) {
  switch (n) {
#define BRAHMS_C_CASE(N) \
  case N:                \
    return col_tile_n(N);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_C_CASE)
#undef BRAHMS_C_CASE
    default:
      return 0;
  }
}

}  // namespace brahms
