// The reverse x-pass of the adjoint: takes the adjoint through one boundary
// between z-steps (the recording forward x-pass is in k_xrec.cu).
//
// Forward, the x-pass at boundary b (between steps b-1 and b) maps the state
// a2 = L(N_A(A_{b-1})) (after its inverse x-FFT) through N_B of step b-1 to
// A_b and through N_A of step b.  In reverse the same boundary takes the
// adjoint through the inverse x-FFT, the reverse of N_A at A_b, the reverse
// of N_B at a2 and the forward x-FFT -- the structure of the forward x-pass
// with each RK4 replaced by its vector-Jacobian product (rk4_vjp_point).
// Between two such passes the adjoint of the linear step, IDFT3(conj(P)
// DFT3), runs as the usual y-forward, tau-propagator (conjugated) and
// y-inverse passes.
//
// MAP: under a transverse mismatch map every point has its own stage phases,
// T V^s (s = 0, 1, 2) from the same tables as the forward x-pass; the
// coefficient sets are formed per point instead of once per CTA.  The
// sensitivities to the stage phases keep their meaning: the map term of
// Phi(x, y, z) does not depend on the per-step mismatch.  Instantiated by
// k_xadj.cu (map-free) and k_xadj_map.cu.
#pragma once

#include "launch_cfg.h"
#include "vjp.cuh"

namespace brahms {

// i kappa_f h e^{-/+ i Phi} at the start, middle and end of a half step from
// the point's start factor e0 = e^{i Phi_0} and quarter-step factor v
template <int F>
__device__ __forceinline__ void map_coef_sets(float2 e0, float2 v, const float* kh, float2 (&c)[3 * F]) {
  float2 e = e0;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
#pragma unroll
    for (int f = 0; f < F; ++f) {
      const float k = kh[f];
      c[s * F + f] = f == 0 ? make_float2(e.y * k, e.x * k) : make_float2(-e.y * k, e.x * k);
    }
    if (s < 2) e = cmul(e, v);
  }
}

template <int NX, int F, int THREADS, bool MAP>
__device__ __forceinline__ void xpass_adj_tile(const XAdjArgs& p, long long tile, const float2* cA, const float2* cB,
                                               float2* rowbuf, float (&sens)[6]) {
  using PL = FftPlan<NX>;
  constexpr int E = PL::E;
  constexpr int T = PL::T;
  constexpr int ROWS = xtile_rows<NX, THREADS>();
  constexpr int PITCH = XchRow::pitch(NX);
  constexpr int RF0 = fft_radix<PL, false>(0);
  constexpr int RFL = fft_radix<PL, false>(PL::NP - 1);
  constexpr int SF0 = NX / RF0, SFL = NX / RFL;
  using SY = typename std::conditional<xpass_warp_sync<NX>(), SyncWarp, SyncBlock>::type;
  static_assert(ROWS >= 1 && ROWS * T == THREADS, "CTA must hold whole rows");
  const TwGlobal tw{p.tw};

  const int t = threadIdx.x % T;
  const int rl = threadIdx.x / T;
  const long long row = tile * ROWS + rl;
  const bool act = row < p.rows;
  float2* myrow = rowbuf + rl * PITCH;

  // 1. every field: load, inverse transform (from k-space), park
#pragma unroll 1
  for (int f = 0; f < F; ++f) {
    const XchRow xr{myrow + f * ROWS * PITCH};
    const float2* src = p.g + f * p.fstride + (act ? row : 0) * NX;
    float2 v[E];
    if (p.from_k) {
#pragma unroll
      for (int b = 0; b < E / RFL; ++b)
#pragma unroll
        for (int r = 0; r < RFL; ++r)
          v[b * RFL + r] = act ? __ldcg(src + t + b * T + r * SFL) : make_float2(0.f, 0.f);
      fft_run<PL, true, 0, XchRow, SY, TwGlobal>(v, t, xr, tw);
    } else {
#pragma unroll
      for (int b = 0; b < E / RF0; ++b)
#pragma unroll
        for (int r = 0; r < RF0; ++r)
          v[b * RF0 + r] = act ? __ldcg(src + t + b * T + r * SF0) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < E / RF0; ++b)
#pragma unroll
      for (int r = 0; r < RF0; ++r) xr.st(t + b * T + r * SF0, v[b * RF0 + r]);
  }

  // 2. reverse of N_A (at xa), then of N_B (at xb), point by point
  if (act) {
    const long long nxy = (long long)p.ny * NX;
    const float2* emap = MAP ? p.emap + (row % p.ny) * NX : nullptr;
    // the recorded states (and under a map the stage-factor tables) of the next
    // point are requested while this one is reversed (measured on the adjoint
    // workload: backward 152 -> 143 ms, under a fan-out map 168 -> 153 ms;
    // requesting both states of the same point up front gained nothing)
    float2 na[F], nb[F], nm[4];
    {
      const long long at0 = row * NX + t;
#pragma unroll
      for (int f = 0; f < F; ++f) {
        na[f] = p.xa ? __ldcg(p.xa + f * p.fstride + at0) : make_float2(0.f, 0.f);
        nb[f] = p.xb ? __ldcg(p.xb + f * p.fstride + at0) : make_float2(0.f, 0.f);
      }
      if constexpr (MAP) {
#pragma unroll
        for (int q = 0; q < 4; ++q) nm[q] = __ldg(emap + q * nxy + t);
      }
    }
#pragma unroll 1
    for (int e = 0; e < E; ++e) {
      const int pos = t + (e / RF0) * T + (e % RF0) * SF0;
      const int off = pos + (pos >> 4);
      float2 g[F], x[F], xbv[F], cm[4];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        x[f] = na[f];
        xbv[f] = nb[f];
      }
      if constexpr (MAP) {
#pragma unroll
        for (int q = 0; q < 4; ++q) cm[q] = nm[q];
      }
      if (e + 1 < E) {
        const int pn = t + ((e + 1) / RF0) * T + ((e + 1) % RF0) * SF0;
        const long long an = row * NX + pn;
#pragma unroll
        for (int f = 0; f < F; ++f) {
          if (p.xa) na[f] = __ldcg(p.xa + f * p.fstride + an);
          if (p.xb) nb[f] = __ldcg(p.xb + f * p.fstride + an);
        }
        if constexpr (MAP) {
#pragma unroll
          for (int q = 0; q < 4; ++q) nm[q] = __ldg(emap + q * nxy + pn);
        }
      }
#pragma unroll
      for (int f = 0; f < F; ++f) g[f] = myrow[f * ROWS * PITCH + off];
      if (p.xa) {
        if constexpr (MAP) {
          float2 c[3 * F];
          map_coef_sets<F>(cm[2], cm[3], p.kh, c);
          rk4_vjp_point<F>(x, g, c, sens[0], sens[1], sens[2]);
        } else {
          rk4_vjp_point<F>(x, g, cA, sens[0], sens[1], sens[2]);
        }
      }
      if (p.xb) {
#pragma unroll
        for (int f = 0; f < F; ++f) x[f] = xbv[f];
        if constexpr (MAP) {
          float2 c[3 * F];
          map_coef_sets<F>(cm[0], cm[1], p.kh, c);
          rk4_vjp_point<F>(x, g, c, sens[3], sens[4], sens[5]);
        } else {
          rk4_vjp_point<F>(x, g, cB, sens[3], sens[4], sens[5]);
        }
      }
#pragma unroll
      for (int f = 0; f < F; ++f) myrow[f * ROWS * PITCH + off] = g[f];
    }
  }

  // 3. every field: unpark, forward transform (or leave in real space), store
#pragma unroll 1
  for (int f = 0; f < F; ++f) {
    const XchRow xr{myrow + f * ROWS * PITCH};
    float2* dst = p.g + f * p.fstride + (act ? row : 0) * NX;
    float2 v[E];
#pragma unroll
    for (int b = 0; b < E / RF0; ++b)
#pragma unroll
      for (int r = 0; r < RF0; ++r) v[b * RF0 + r] = xr.ld(t + b * T + r * SF0);
    if (!p.to_k) {
      if (act) {
#pragma unroll
        for (int b = 0; b < E / RF0; ++b)
#pragma unroll
          for (int r = 0; r < RF0; ++r) dst[t + b * T + r * SF0] = v[b * RF0 + r];
      }
    } else {
      fft_run<PL, false, 0, XchRow, SY, TwGlobal>(v, t, xr, tw);
      if (act) {
#pragma unroll
        for (int b = 0; b < E / RFL; ++b)
#pragma unroll
          for (int r = 0; r < RFL; ++r) dst[t + b * T + r * SFL] = v[b * RFL + r];
      }
    }
    SY::sync();
  }
}

template <int NX, int F, bool MAP>
__global__ void __launch_bounds__(xpass_threads<NX>(), xpass_threads<NX>() <= 128 ? 4 : 1)
    xpass_adj_kernel(const XAdjArgs p) {
  constexpr int THREADS = xpass_threads<NX>();
  extern __shared__ float4 sm4[];
  float2* cA = reinterpret_cast<float2*>(sm4);  // [3][F]
  float2* cB = cA + 3 * F;                      // [3][F]
  float2* rowbuf = cA + 6 * F;
  __shared__ double red[THREADS / 32][6];
  if constexpr (!MAP) {
    // coefficient sets from the launch (formed on the host in FP64)
    if (threadIdx.x < 3 * F) {
      cA[threadIdx.x] = p.cset[0][threadIdx.x];
      cB[threadIdx.x] = p.cset[1][threadIdx.x];
    }
  }
  __syncthreads();
  float sens[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  xpass_adj_tile<NX, F, THREADS, MAP>(p, blockIdx.x, cA, cB, rowbuf, sens);
  // block sums in FP64, fixed order (deterministic)
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double v = (double)sens[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) v += red[w][threadIdx.x];
    p.partial[(long long)blockIdx.x * 6 + threadIdx.x] = v;
  }
}

template <int NX, int F, bool MAP>
cudaError_t launch_adjoint(const XAdjArgs& a, long long* ncta, cudaStream_t s) {
  constexpr int ROWS = xpass_rows<NX>();
  constexpr int THREADS = xpass_threads<NX>();
  const size_t smem = (size_t)xpass_smem_floats2<NX>(F) * sizeof(float2);
  static SmemOnce once;
  cudaError_t e = raise_smem_limit(xpass_adj_kernel<NX, F, MAP>, smem, once);
  if (e != cudaSuccess) return e;
  const long long grid = (a.rows + ROWS - 1) / ROWS;
  *ncta = grid;
  if (grid <= 0) return cudaSuccess;
  xpass_adj_kernel<NX, F, MAP><<<(unsigned)grid, THREADS, smem, s>>>(a);
  return cudaPeekAtLastError();
}


}  // namespace brahms
