// y-pass and tau-pass instantiations and dispatch.
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "launch_cfg.h"

namespace brahms {

template <int N, bool INV, int AXIS>
static cudaError_t launch_axis(const AxisArgs& a, cudaStream_t s) {
  using PL = FftPlan<N>;
  constexpr int TPC = tiles_per_cta<PL>();
  constexpr int THREADS = TPC * tile_threads<PL>();
  const size_t smem = (size_t)axis_kernel_smem_floats2<PL, INV, AXIS>() * sizeof(float2);
  static SmemOnce once;
  cudaError_t e = raise_smem_limit(axis_fft_kernel<PL, INV, AXIS>, smem, once);
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
  static SmemOnce once;
  cudaError_t e = raise_smem_limit(tpass_prop_kernel<PL>, smem, once);
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

int tw_table_size_of(int n) {
  switch (n) {
#define BRAHMS_W_CASE(N) \
  case N:                \
    return tw_table_size<FftPlan<N>>();
    BRAHMS_FOR_EACH_SIZE(BRAHMS_W_CASE)
#undef BRAHMS_W_CASE
    default:
      return 0;
  }
}

static int plan_radices(int n, int* r) {
  switch (n) {
#define BRAHMS_R_CASE(N)                                              \
  case N:                                                             \
    for (int p = 0; p < FftPlan<N>::NP; ++p) r[p] = FftPlan<N>::r(p); \
    return FftPlan<N>::NP;
    BRAHMS_FOR_EACH_SIZE(BRAHMS_R_CASE)
#undef BRAHMS_R_CASE
    default:
      return 0;
  }
}

// Per-pass twiddle blocks (the layout of tw_pass_off): for each direction
// and pass P >= 1 with radix R after stride NS, entries [r][m] =
// exp(sign 2 pi i (r m mod NS R) / (NS R)), sign -1 forward and +1 inverse,
// evaluated in FP64 and split into hi + lo floats.
cudaError_t upload_twiddles(float4* tw, int n, cudaStream_t s) {
  int rad[8];
  const int np = plan_radices(n, rad);
  if (np <= 0) return cudaErrorInvalidValue;
  std::vector<float4> h;
  for (int dir = 0; dir < 2; ++dir) {
    const double sign = dir == 0 ? -1.0 : 1.0;
    int ns = 1;
    for (int q = 0; q < np; ++q) {
      const int R = dir == 0 ? rad[q] : rad[np - 1 - q];
      if (q > 0) {
        for (int r = 0; r < R; ++r)
          for (int mm = 0; mm < ns; ++mm) {
            const long long k = ((long long)r * mm) % ((long long)ns * R);
            const double ang = sign * 6.283185307179586476925286766559 * (double)k / (double)(ns * R);
            const double c = std::cos(ang), sn = std::sin(ang);
            const float ch = (float)c, sh = (float)sn;
            h.push_back(make_float4(ch, sh, (float)(c - (double)ch), (float)(sn - (double)sh)));
          }
      }
      ns *= R;
    }
  }
  if (h.empty()) h.push_back(make_float4(1.f, 0.f, 0.f, 0.f));
  if ((int)h.size() != tw_table_size_of(n)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyAsync(tw, h.data(), sizeof(float4) * h.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);  // h is a local buffer
}

int tau_col_tile_of(int n) {
  switch (n) {
#define BRAHMS_TC_CASE(N) \
  case N:                 \
    return ColTile<TauPlan<N>>::value;
    BRAHMS_FOR_EACH_SIZE(BRAHMS_TC_CASE)
#undef BRAHMS_TC_CASE
    default:
      return 0;
  }
}

int col_tile_of(int n) {
  switch (n) {
#define BRAHMS_C_CASE(N) \
  case N:                \
    return ColTile<FftPlan<N>>::value;
    BRAHMS_FOR_EACH_SIZE(BRAHMS_C_CASE)
#undef BRAHMS_C_CASE
    default:
      return 0;
  }
}

}  // namespace brahms
