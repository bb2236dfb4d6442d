// Diagnostics of the fields: the temporal power trace and the energy
// spectrum over Omega (the Sec. 6 power formula resolved in tau or Omega).
// Neither kernel writes the state.
#include "kernels.cuh"
#include "launch_cfg.h"

namespace brahms {

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// sum_{x,y} |A_f(x, y, tau_k)|^2 for every (k, f): one CTA per plane; two
// points per 16-byte load, their squares summed in FP32 and accumulated in
// FP64 (planes hold an even number of points)
__global__ void __launch_bounds__(256) power_trace_kernel(const float2* __restrict__ data, long long plane,
                                                          int nt, long long fstride, double* out) {
  const int k = blockIdx.x, f = blockIdx.y;
  const float2* a = data + (long long)f * fstride + (long long)k * plane;
  double s = 0.0;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const long long n2 = plane / 2;
  long long i = threadIdx.x;
  // four loads in flight per thread; each pair's FP32 sum goes into FP64 as before
  for (; i + 3 * (long long)blockDim.x < n2; i += 4 * (long long)blockDim.x) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = __ldcg(a4 + i + u * (long long)blockDim.x);
#pragma unroll
    for (int u = 0; u < 4; ++u) s += (double)fmaf(v[u].x, v[u].x, fmaf(v[u].y, v[u].y, fmaf(v[u].z, v[u].z, v[u].w * v[u].w)));
  }
  for (; i < n2; i += blockDim.x) {
    const float4 v = __ldcg(a4 + i);
    s += (double)fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w)));
  }
  if ((plane & 1) && threadIdx.x == 0) {
    const float2 v = __ldcg(a + plane - 1);
    s += (double)fmaf(v.x, v.x, v.y * v.y);
  }
  __shared__ double red[8];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum_d(v);
    if (threadIdx.x == 0) out[f * nt + k] = v;
  }
}

}  // namespace

// sum_{x,y} |DFT_tau A_f|^2 (m) for every (m, f), added into out (zeroed by
// the caller).  Each CTA walks a contiguous range of its tau-tiles (TX
// neighbouring columns of one field and y), transforms them forward in
// registers like the tau-pass, writes the squared moduli (FP32) to shared
// memory and adds their sum over the tile's columns (pairwise in FP32) to
// per-thread FP64 accumulators of its bins; a change of field and the end of
// the range flush them with one atomicAdd per bin.  (Summing the columns in
// FP64 made the FP64 pipe the bound: 0.94 against 0.60 ms per call with the
// power trace on the OPG state.)
template <class PL>
__global__ void __launch_bounds__(tiles_per_cta<PL>() * tile_threads<PL>())
    tau_spectrum_kernel(const AxisArgs p, long long range, double* out) {
  constexpr int N = PL::N, E = PL::E, T = PL::T, TX = ColTile<PL>::value;
  constexpr int GT = T * TX;                       // threads of one tile group
  constexpr int THREADS = tiles_per_cta<PL>() * GT;
  constexpr int TPC = tiles_per_cta<PL>();
  constexpr int R0 = fft_radix<PL, false>(0), RL = fft_radix<PL, false>(PL::NP - 1);
  constexpr int S0 = N / R0, SL = N / RL;
  constexpr int BPT = (N + GT - 1) / GT;  // bins per thread
  extern __shared__ float4 sm4[];
  float2* xch = reinterpret_cast<float2*>(sm4);
  if constexpr (tw_in_smem<PL>()) {
    for (int i = threadIdx.x; i < tw_table_size<PL>(); i += THREADS) sm4[i] = p.tw[i];
    __syncthreads();
    xch = reinterpret_cast<float2*>(sm4 + tw_table_size<PL>());
  }
  const int lt = threadIdx.x % GT, tl = threadIdx.x / GT;
  const int tx = lt % TX, t = lt / TX;
  const XchCol<TX> xc{xch + tl * N * TX, tx};
  // squared moduli of this group's tile, [TX][N + 1] (padded: the writes
  // vary the column fastest, the reads the bin)
  float* q = reinterpret_cast<float*>(xch + tl * N * TX);
  double acc[BPT];
#pragma unroll
  for (int j = 0; j < BPT; ++j) acc[j] = 0.0;
  int cur_f = -1;
  const long long ctiles = (p.ntiles + TPC - 1) / TPC;
  const long long first = (long long)blockIdx.x * range;
  const long long last = first + range < ctiles ? first + range : ctiles;
  for (long long ct = first; ct < last; ++ct) {
    const long long tile = ct * TPC + tl;
    const int ftile = tile < p.ntiles ? (int)((tile / p.xtiles) / p.ny) : cur_f;
    if (ftile != cur_f) {
      if (cur_f >= 0) {
#pragma unroll
        for (int j = 0; j < BPT; ++j)
          if (lt + j * GT < N) atomicAdd(out + (long long)cur_f * N + lt + j * GT, acc[j]);
      }
#pragma unroll
      for (int j = 0; j < BPT; ++j) acc[j] = 0.0;
      cur_f = ftile;
    }
    const AxisTile<N, 2, TX> a(p, tile, tx);
    float2 v[E];
#pragma unroll
    for (int b = 0; b < E / R0; ++b)
#pragma unroll
      for (int r = 0; r < R0; ++r)
        v[b * R0 + r] = a.act ? __ldcg(a.base + (t + b * T + r * S0) * a.stride) : make_float2(0.f, 0.f);
    if constexpr (tw_in_smem<PL>()) fft_run<PL, false, 0, XchCol<TX>, SyncBlock, TwShared>(v, t, xc, TwShared{sm4});
    else fft_run<PL, false, 0, XchCol<TX>, SyncBlock, TwGlobal>(v, t, xc, TwGlobal{p.tw});
    __syncthreads();  // every read of the exchange space is done
#pragma unroll
    for (int b = 0; b < E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const float2 w = v[b * RL + r];
        q[tx * (N + 1) + t + b * T + r * SL] = fmaf(w.x, w.x, w.y * w.y);
      }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
      const int k = lt + j * GT;
      if (k < N) {
        // the tile's columns summed pairwise in FP32, then one FP64 add per bin
        float c2[TX];
#pragma unroll
        for (int c = 0; c < TX; ++c) c2[c] = q[c * (N + 1) + k];
#pragma unroll
        for (int w = TX / 2; w > 0; w >>= 1)
#pragma unroll
          for (int c = 0; c < w; ++c) c2[c] += c2[c + w];
        acc[j] += (double)c2[0];
      }
    }
    __syncthreads();  // q is the next tile's exchange space
  }
  if (cur_f >= 0) {
#pragma unroll
    for (int j = 0; j < BPT; ++j)
      if (lt + j * GT < N) atomicAdd(out + (long long)cur_f * N + lt + j * GT, acc[j]);
  }
}

cudaError_t run_power_trace(const float2* data, int nx, int ny, int nt, int nf, long long fstride, double* out,
                            cudaStream_t s) {
  power_trace_kernel<<<dim3(nt, nf), 256, 0, s>>>(data, (long long)nx * ny, nt, fstride, out);
  return cudaPeekAtLastError();
}

template <int N>
static cudaError_t launch_spectrum(const AxisArgs& a, double* out, cudaStream_t s) {
  using PL = FftPlan<N>;
  constexpr int TPC = tiles_per_cta<PL>();
  constexpr int THREADS = TPC * tile_threads<PL>();
  const size_t smem = (size_t)axis_smem_floats2<PL>() * sizeof(float2);
  static SmemOnce once;
  cudaError_t e = raise_smem_limit(tau_spectrum_kernel<PL>, smem, once);
  if (e != cudaSuccess) return e;
  const long long ctiles = (a.ntiles + TPC - 1) / TPC;
  if (ctiles <= 0) return cudaSuccess;
  const long long grid = ctiles < 2 * 152 ? ctiles : 2 * 152;
  const long long range = (ctiles + grid - 1) / grid;
  tau_spectrum_kernel<PL><<<(unsigned)((ctiles + range - 1) / range), THREADS, smem, s>>>(a, range, out);
  return cudaPeekAtLastError();
}

cudaError_t run_tau_spectrum(int nt, const AxisArgs& a, double* out, cudaStream_t s) {
  switch (nt) {
#define BRAHMS_SP_CASE(N) \
  case N:                 \
    return launch_spectrum<N>(a, out, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_SP_CASE)
#undef BRAHMS_SP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace brahms
