// Kernels of one split-step z-step (Sec. 3.1, Eq. expon) on the layout
// fields[f][tau][y][x] (x fastest), complex64.
//
// A z-step is four HBM passes per field:
//   x-pass  inverse x-FFT, the second RK4 half step of step j, the first RK4
//           half step of step j+1, forward x-FFT (all fields of a row at once,
//           the nonlinear coupling is pointwise across fields)
//   y-pass  forward y-FFT
//   t-pass  forward tau-FFT, multiply by the linear propagator
//           P = Px(kx) Py(ky) Pt(Omega) / (NX NY NT), inverse tau-FFT
//   y-pass  inverse y-FFT
// Between calls the state is in real space; the first and the last step of
// a call peel the x-pass (NL_FIRST / NL_LAST).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fft_core.cuh"

namespace brahms {

enum XMode : int { XM_FWD = 0, XM_INV = 1, XM_NL_FIRST = 2, XM_NL_MID = 3, XM_NL_LAST = 4 };

struct XPassArgs {
  float2* data;        // [nf][rows][nx]
  long long fstride;   // elements between fields
  long long rows;      // ny * nt
  const float4* tw;    // per-pass twiddle table of the x transform (hi/lo pairs)
  int mode;            // XMode
  double phiA, dkA;    // step whose first half is applied: Phi(z_j), dk_j
  double phiB, dkB;    // step whose second half is applied
  double dz;
  float kh[3];         // kappa_f * dz/2, including the 1/2 SH factor for 2 fields
  float kh2[3];        // kh / 2 (exact)
  float scale;         // output scale for XM_INV
  // transverse mismatch map: per-(x, y) stage phase factors [4][ny][nx]
  // (B start, B quarter-step, A start, A quarter-step; see run_map_tables),
  // or NULL for a mismatch uniform across the grid
  const float2* emap;
  int ny;
  // recording (adjoint recomputation): real-space copies of the state that
  // enters the B half step and of the state that enters the A half step, or NULL
  float2* rec_b;
  float2* rec_a;
  // the six stage factors e^{+i Phi} (B half: start, 3/4, end; A half: start,
  // 1/4, 1/2 of the step) from the phases above, written by the host
  // dispatchers in FP64 (map-free x-passes read them instead of computing
  // them per CTA)
  float2 ecoef[6];
};
// Host: the stage factors of an x-pass from its phases (FP64 phase, reduced
// mod 2 pi, cos and sin in FP64, rounded to float).
void fill_stage_factors(XPassArgs& a);

struct AxisArgs {
  float2* data;
  int nx, ny, nt;
  long long fstride;
  long long ntiles;
  int xtiles;
  const float4* tw;    // twiddles of the transformed axis (hi/lo pairs)
  const float2* px;    // [nf][nx] propagator factors (t-pass only)
  const float2* py;    // [nf][ny]
  const float2* pt;    // [nf][nt]
  float scale, scale_lo;  // 1/(nx ny nt) = scale + scale_lo (lo = 0 for powers of two)
  int conj_p;             // apply conj(P) (the adjoint of the linear step)
};

// ------------------------------------------------------------ tile shapes
template <int N>
__host__ __device__ constexpr int fft_threads() { return FftPlan<N>::T; }

// x-pass CTA: 128 threads (or one row when a row needs more); rows whose
// threads lie inside one warp synchronise their exchanges with __syncwarp.
template <int N>
__host__ __device__ constexpr int xpass_threads() { return fft_threads<N>() >= 128 ? fft_threads<N>() : 128; }
template <int N>
__host__ __device__ constexpr int xpass_rows() { return xpass_threads<N>() / fft_threads<N>(); }
template <int N>
__host__ __device__ constexpr bool xpass_warp_sync() { return fft_threads<N>() <= 32 && 32 % fft_threads<N>() == 0; }
// shared memory in float2 units: twiddles (N float4), NL coefficients (6 F),
// exchange rows, and a private stash of F-1 fields per thread
template <int N>
__host__ __device__ constexpr int xpass_smem_floats2(int nf) {
  return 6 * nf + nf * xpass_rows<N>() * XchRow::pitch(N);
}
// resident CTAs the x-pass asks the register allocator for: 6 (80 registers)
// where six CTAs' shared memory fits in an SM and rows are at most 256 long
// (no spills there); otherwise 4 (128 registers)
template <int N, int F>
__host__ __device__ constexpr int xpass_min_blocks() {
  return xpass_threads<N>() > 128                                                          ? 1
         : (N <= 256 && 6 * (xpass_smem_floats2<N>(F) * 8 + 1024) <= 228 * 1024) ? 6
                                                                                          : 4;
}

// Strided pencils: tiles of TX neighbouring columns (128-byte rows up to
// N = 1024) times the plan's T threads per pencil.
__host__ __device__ constexpr int col_tile_n(int n) { return n <= 1024 ? 16 : (n <= 2048 ? 8 : 4); }
// columns per tile of a plan's strided-pencil kernels
template <class PL>
struct ColTile {
  static constexpr int value = col_tile_n(PL::N);
};
// (A plan may override its tile width; 8-column tiles for the 512-point tau
// propagator measured slower than 16 on GB300, 575 vs 546 us per OPG launch.)
template <class PL>
__host__ __device__ constexpr int tile_threads() { return PL::T * ColTile<PL>::value; }
template <class PL>
__host__ __device__ constexpr int tiles_per_cta() { return tile_threads<PL>() >= 256 ? 1 : 256 / tile_threads<PL>(); }
// twiddle tables up to 40 KB are copied to shared memory; larger ones are read through L1
template <class PL>
__host__ __device__ constexpr bool tw_in_smem() { return tw_table_size<PL>() * 16 <= 40960; }
template <class PL>
__host__ __device__ constexpr int axis_smem_floats2() {
  return (tw_in_smem<PL>() ? 2 * tw_table_size<PL>() : 0) + tiles_per_cta<PL>() * PL::N * ColTile<PL>::value;
}
// The forward y-pass reads its twiddles through L1 instead of staging them in
// shared memory per CTA: measured on the 3 x 256x256x512 state, 285 -> 253 us
// per launch (the inverse y-pass, 259 -> 266, and the tau propagator,
// 477 -> 485, measured the other way and keep the staging).
template <class PL, bool INV, int AXIS>
__host__ __device__ constexpr bool axis_tw_staged() { return tw_in_smem<PL>() && !(AXIS == 1 && !INV); }
template <class PL, bool INV, int AXIS>
__host__ __device__ constexpr int axis_kernel_smem_floats2() {
  return (axis_tw_staged<PL, INV, AXIS>() ? 2 * tw_table_size<PL>() : 0) +
         tiles_per_cta<PL>() * PL::N * ColTile<PL>::value;
}

// -------------------------------------------------------- nonlinear step
// Right-hand sides of Eqs. CEp/CEs/CEi (3 fields p, s, i) or of the
// degenerate SHG pair (SH, F), already multiplied by the step h, with
//   c[f] = i kappa_f h e^{-/+ i Phi(z)}  (minus for field 0);
// the adjoint's stage recomputation uses this form.
template <int F>
__device__ __forceinline__ void nl_rhs(const float2 (&a)[F], const float2* __restrict__ c,
                                       float2 (&k)[F]) {
  if constexpr (F == 3) {
    k[0] = cmul(c[0], cmul(a[1], a[2]));
    k[1] = cmul(c[1], cmulc(a[0], a[2]));
    k[2] = cmul(c[2], cmulc(a[0], a[1]));
  } else {
    k[0] = cmul(c[0], cmul(a[1], a[1]));
    k[1] = cmul(c[1], cmulc(a[0], a[1]));
  }
}

// Stage right-hand sides in the form used by the forward half steps:
// k_f = i (kappa_f h) m_f with e = e^{+i Phi(z_stage)} and
//   F = 3: m_p = conj(e) A_s A_i,  m_s = e A_p conj(A_i),  m_i = e A_p conj(A_s)
//   F = 2: m_SH = conj(e) A_F^2,   m_F = e A_SH conj(A_F)
// (five complex products per stage for three fields instead of six; the
// factor i kappa_f h goes into the stage updates' FMAs).
template <int F>
__device__ __forceinline__ void nl_m(const float2 (&a)[F], float2 e, float2 (&m)[F]) {
  if constexpr (F == 3) {
    const float2 u = cmul(e, a[0]);
    m[1] = cmulc(u, a[2]);
    m[2] = cmulc(u, a[1]);
    m[0] = cmulc(cmul(a[1], a[2]), e);
  } else {
    const float2 sq = make_float2(fmaf(a[1].x, a[1].x, -a[1].y * a[1].y), (a[1].x + a[1].x) * a[1].y);
    m[0] = cmulc(sq, e);
    m[1] = cmulc(cmul(e, a[0]), a[1]);
  }
}
// a + i c m for a real c
__device__ __forceinline__ float2 add_i_scaled(float2 a, float c, float2 m) {
  return make_float2(fmaf(-c, m.y, a.x), fmaf(c, m.x, a.y));
}

// Classical RK4 over one half step h (Sec. 3.1): e3 holds e^{+i Phi} at the
// start, the midpoint and the end of the interval; kh = kappa h and
// kh2 = kh/2 per field.  Every stage and the final combination use the same
// kh_f, and the 1/6 weight is common to all fields: field-dependent rounding
// of the weights would break the Manley-Rowe balance the exact scheme keeps
// and let the total energy drift step after step.
template <int F>
__device__ __forceinline__ void rk4(float2 (&a)[F], const float2* __restrict__ e3, const float* kh,
                                    const float* kh2) {
  float2 m[F], acc[F], t[F];
  nl_m<F>(a, e3[0], m);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    acc[f] = m[f];
    t[f] = add_i_scaled(a[f], kh2[f], m[f]);
  }
  const float2 emid = e3[1];
  nl_m<F>(t, emid, m);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    acc[f] = make_float2(fmaf(2.f, m[f].x, acc[f].x), fmaf(2.f, m[f].y, acc[f].y));
    t[f] = add_i_scaled(a[f], kh2[f], m[f]);
  }
  nl_m<F>(t, emid, m);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    acc[f] = make_float2(fmaf(2.f, m[f].x, acc[f].x), fmaf(2.f, m[f].y, acc[f].y));
    t[f] = add_i_scaled(a[f], kh[f], m[f]);
  }
  nl_m<F>(t, e3[2], m);
#pragma unroll
  for (int f = 0; f < F; ++f) a[f] = add_i_scaled(a[f], kh[f], cscale(cadd(acc[f], m[f]), 1.f / 6.f));
}

// e^{-i Phi} with Phi in FP64, reduced to [-pi, pi] before the FP32 sincos.
__device__ __forceinline__ float2 phase_minus(double phi) {
  const double two_pi = 6.283185307179586476925286766559;
  double r = phi - two_pi * rint(phi / two_pi);
  float s, c;
  sincosf((float)r, &s, &c);
  return make_float2(c, -s);
}

// Stage phase factors e^{+i Phi}: sets 0..2 = second half of step B at
// z_B + dz/2, z_B + 3dz/4, z_B + dz; sets 3..5 = first half of step A at z_A,
// z_A + dz/4, z_A + dz/2.
template <int F>
__device__ __forceinline__ void nl_coefficients(const XPassArgs& p, float2* coef) {
  const int s = threadIdx.x;
  if (s < 6) {
    double phi;
    if (s < 3) phi = p.phiB + p.dkB * (0.5 * p.dz + 0.25 * p.dz * s);
    else phi = p.phiA + p.dkA * (0.25 * p.dz * (s - 3));
    const float2 em = phase_minus(phi);  // e^{-i Phi}
    coef[s] = make_float2(em.x, -em.y);
  }
}

// ------------------------------------------------------------------ x-pass
// One row (y, tau) of every field per T threads; a CTA of THREADS threads
// handles THREADS/T rows per tile.  Each field of a row has its own padded
// row buffer in shared memory, used both as that field's FFT exchange space
// and to park the field between the transforms: after the inverse transform
// every thread parks its values at the positions it owns (the last pass of a
// Stockham transform reads and writes the same positions per thread), the
// pointwise RK4 pair then reads all F values of each owned point, and the
// forward transform starts from the owned positions again.  No thread ever
// reads a position another thread parked, so parking needs no barrier, and
// the fields and the points are processed in loops rather than unrolled
// (the points two at a time), which keeps the kernel small enough for the
// instruction cache.  Field data
// is read with ld.global.cg (L2), twiddles through L1.
template <int NX, int THREADS>
__host__ __device__ constexpr int xtile_rows() { return THREADS / FftPlan<NX>::T; }
template <int NX, int THREADS>
__host__ __device__ constexpr int xtile_smem_floats2(int nf) {
  return 6 * nf + nf * xtile_rows<NX, THREADS>() * XchRow::pitch(NX);
}

template <int NX, int F, int THREADS, bool MAP = false, bool REC = false>
__device__ __forceinline__ void xpass_tile(const XPassArgs& p, long long tile, const float2* coef, float2* rowbuf) {
  using PL = FftPlan<NX>;
  constexpr int E = PL::E;
  constexpr int T = PL::T;
  constexpr int ROWS = xtile_rows<NX, THREADS>();
  constexpr int PITCH = XchRow::pitch(NX);
  constexpr int RF0 = fft_radix<PL, false>(0);           // forward first radix
  constexpr int RFL = fft_radix<PL, false>(PL::NP - 1);  // forward last radix
  constexpr int SF0 = NX / RF0, SFL = NX / RFL;
  using SY = typename std::conditional<xpass_warp_sync<NX>(), SyncWarp, SyncBlock>::type;
  static_assert(ROWS >= 1 && ROWS * T == THREADS, "CTA must hold whole rows");
  const TwGlobal tw{p.tw};

  const int t = threadIdx.x % T;
  const int rl = threadIdx.x / T;
  const long long row = tile * ROWS + rl;
  const bool act = row < p.rows;
  float2* myrow = rowbuf + rl * PITCH;  // field f at myrow + f ROWS PITCH
  const int mode = p.mode;
  const bool from_k = (mode == XM_INV || mode == XM_NL_MID || mode == XM_NL_LAST);

  // 1. every field: load, inverse transform (from k-space), park
#pragma unroll 1
  for (int f = 0; f < F; ++f) {
    const XchRow xr{myrow + f * ROWS * PITCH};
    const float2* src = p.data + f * p.fstride + (act ? row : 0) * NX;
    float2 v[E];
    if (from_k) {
#pragma unroll
      for (int b = 0; b < E / RFL; ++b)
#pragma unroll
        for (int r = 0; r < RFL; ++r)
          v[b * RFL + r] = act ? __ldcg(src + t + b * T + r * SFL) : make_float2(0.f, 0.f);
      // inverse's output positions t + b T + r NX/RF0 = forward first-pass positions
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

  // 2. the RK4 half steps, point by point over the owned positions
  if (mode == XM_NL_MID || mode == XM_NL_LAST || mode == XM_NL_FIRST) {
    const long long nxy = (long long)p.ny * NX;
    const float2* emap = MAP ? p.emap + (act ? row % p.ny : 0) * NX : nullptr;
    // MAP: the next point's stage-factor tables are requested while this point's
    // RK4 pair runs (with a fan-out map: 656 -> 579 us per OPG launch)
    float2 nm[4];
    if constexpr (MAP) {
#pragma unroll
      for (int q = 0; q < 4; ++q) nm[q] = __ldg(emap + q * nxy + t);
    }
    // two points per iteration: their RK4 chains interleave (measured on GB300:
    // OPG x-pass 549 -> 540 us, with a fan-out map 699 -> 655 us, SFG 94 -> 90 us;
    // four points per iteration, 579 us, overflow the instruction cache)
#pragma unroll 2
    for (int e = 0; e < E; ++e) {
      const int pos = t + (e / RF0) * T + (e % RF0) * SF0;
      const int off = pos + (pos >> 4);  // XchRow padding
      float2 cm[4];
      if constexpr (MAP) {
#pragma unroll
        for (int q = 0; q < 4; ++q) cm[q] = nm[q];
        if (e + 1 < E) {
          const int pn = t + ((e + 1) / RF0) * T + ((e + 1) % RF0) * SF0;
#pragma unroll
          for (int q = 0; q < 4; ++q) nm[q] = __ldg(emap + q * nxy + pn);
        }
      }
      float2 a[F];
#pragma unroll
      for (int f = 0; f < F; ++f) a[f] = myrow[f * ROWS * PITCH + off];
      // MAP: e^{i Phi(x, y, z_s)} = T V^s at this point, for the B and A stages
      if (mode != XM_NL_FIRST) {
        if constexpr (REC) {
          if (p.rec_b && act) {
#pragma unroll
            for (int f = 0; f < F; ++f) p.rec_b[f * p.fstride + row * NX + pos] = a[f];
          }
        }
        if constexpr (MAP) {
          float2 e3[3];
          const float2 v = cm[1];
          e3[0] = cm[0];
          e3[1] = cmul(e3[0], v);
          e3[2] = cmul(e3[1], v);
          rk4<F>(a, e3, p.kh, p.kh2);
        } else {
          rk4<F>(a, coef, p.kh, p.kh2);
        }
      }
      if (mode != XM_NL_LAST) {
        if constexpr (REC) {
          if (p.rec_a && act) {
#pragma unroll
            for (int f = 0; f < F; ++f) p.rec_a[f * p.fstride + row * NX + pos] = a[f];
          }
        }
        if constexpr (MAP) {
          float2 e3[3];
          const float2 v = cm[3];
          e3[0] = cm[2];
          e3[1] = cmul(e3[0], v);
          e3[2] = cmul(e3[1], v);
          rk4<F>(a, e3, p.kh, p.kh2);
        } else {
          rk4<F>(a, coef + 3, p.kh, p.kh2);
        }
      }
#pragma unroll
      for (int f = 0; f < F; ++f) myrow[f * ROWS * PITCH + off] = a[f];
    }
  }

  // 3. every field: unpark, forward transform (or scale), store
  const bool to_x = (mode == XM_INV || mode == XM_NL_LAST);
  const float sc = mode == XM_INV ? p.scale : 1.f;
#pragma unroll 1
  for (int f = 0; f < F; ++f) {
    const XchRow xr{myrow + f * ROWS * PITCH};
    float2* dst = p.data + f * p.fstride + (act ? row : 0) * NX;
    float2 v[E];
#pragma unroll
    for (int b = 0; b < E / RF0; ++b)
#pragma unroll
      for (int r = 0; r < RF0; ++r) v[b * RF0 + r] = xr.ld(t + b * T + r * SF0);
    if (to_x) {
      if (act) {
#pragma unroll
        for (int b = 0; b < E / RF0; ++b)
#pragma unroll
          for (int r = 0; r < RF0; ++r) dst[t + b * T + r * SF0] = cscale(v[b * RF0 + r], sc);
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
    SY::sync();  // the next field's exchanges use another buffer; keep the warp together
  }
}

// MAP: per-point stage phases from a transverse mismatch map (p.emap);
// REC: record the half steps' input states (p.rec_b, p.rec_a)
template <int NX, int F, bool MAP, bool REC = false>
__global__ void __launch_bounds__(xpass_threads<NX>(), xpass_min_blocks<NX, F>())
    xpass_kernel(const XPassArgs p) {
  constexpr int THREADS = xpass_threads<NX>();
  extern __shared__ float4 sm4[];
  float2* coef = reinterpret_cast<float2*>(sm4);
  float2* rowbuf = coef + 6 * F;
  // stage factors from the launch (formed on the host in FP64: a per-CTA FP64
  // phase reduction ahead of this barrier stalled every CTA's first warps)
  if constexpr (!MAP) {
    if (threadIdx.x < 6) coef[threadIdx.x] = p.ecoef[threadIdx.x];
  }
  __syncthreads();
  // rows from the last tau-plane down (see the note on pass order above)
  xpass_tile<NX, F, THREADS, MAP, REC>(p, (long long)gridDim.x - 1 - blockIdx.x, coef, rowbuf);
}

// w (1 + d) for a propagator factor in delta form: the small product w d is
// formed first and w added with one rounding.  (Folding w into the FMA chain,
// e.g. fma(w.x, d.x, fma(-w.y, d.y, w.x)), rounds w.x - w.y d.y before the
// second-order term w.x (cos phi - 1) arrives; for small phases that term is
// below half an ulp and is then always lost, so |1 + d| acts as
// 1 + phi^2 / 2 and the energy grows step after step.)
__device__ __forceinline__ float2 mul_one_plus(float2 w, float2 d) { return cadd(w, cmul(w, d)); }

// ------------------------------------------------- strided-axis passes
// AXIS 1: pencils along y (stride nx), tiles over (f, tau, x-tile).
// AXIS 2: pencils along tau (stride nx ny), tiles over (f, y, x-tile).
// Order across passes: the x-pass walks its rows from the last tau-plane
// down and the y-passes from the first up, so the x-pass starts on planes the
// y-inverse wrote last and the y-forward on planes the x-pass wrote last,
// still in L2 (read there, and overwritten there before they are written
// back).  Measured on the 3 x 256x256x512 state: 1603 -> 1592 ms per
// 1000-step call; a tau-major y order (every field of a plane together)
// made the y-passes 20 us slower and the step 1622 ms.  The tau-propagator
// also walks its tiles from the last down (tau 476 -> 473, y-inverse
// 258 -> 257 us).
template <int N, int AXIS, int TX>
struct AxisTile {
  float2* base;  // element (x, pencil index 0)
  long long stride;
  int f, other, x;
  bool act;
  __device__ __forceinline__ AxisTile(const AxisArgs& p, long long tile, int tx) {
    const int xt = (int)(tile % p.xtiles);
    const long long rest = tile / p.xtiles;
    const int no = AXIS == 1 ? p.nt : p.ny;
    other = (int)(rest % no);
    f = (int)(rest / no);
    x = xt * TX + tx;
    act = tile < p.ntiles && x < p.nx;
    stride = AXIS == 1 ? (long long)p.nx : (long long)p.nx * p.ny;
    const long long off = AXIS == 1 ? (long long)other * p.nx * p.ny + x : (long long)other * p.nx + x;
    base = p.data + (act ? (long long)f * p.fstride + off : 0);
  }
};

// Tiles per CTA of THREADS threads for strided pencils.
template <class PL, int THREADS>
__host__ __device__ constexpr int tiles_per_cta_t() { return THREADS / tile_threads<PL>(); }

template <class PL, bool INV, int AXIS, int THREADS, class TW = TwShared>
__device__ __forceinline__ void axis_tile(const AxisArgs& p, long long cta_tile, const TW& tw, float2* xch) {
  constexpr int N = PL::N, E = PL::E, T = PL::T, TX = ColTile<PL>::value;
  constexpr int TPC = tiles_per_cta_t<PL, THREADS>();
  static_assert(TPC >= 1 && TPC * T * TX == THREADS, "CTA must hold whole tiles");
  constexpr int R0 = fft_radix<PL, INV>(0), RL = fft_radix<PL, INV>(PL::NP - 1);
  constexpr int S0 = N / R0, SL = N / RL;
  const int lt = threadIdx.x % (T * TX), tl = threadIdx.x / (T * TX);
  const int tx = lt % TX, t = lt / TX;
  const AxisTile<N, AXIS, TX> a(p, cta_tile * TPC + tl, tx);
  const XchCol<TX> xc{xch + tl * N * TX, tx};
  float2 v[E];
#pragma unroll
  for (int b = 0; b < E / R0; ++b)
#pragma unroll
    for (int r = 0; r < R0; ++r)
      v[b * R0 + r] = a.act ? __ldcg(a.base + (t + b * T + r * S0) * a.stride) : make_float2(0.f, 0.f);
  fft_run<PL, INV, 0, XchCol<TX>, SyncBlock, TW>(v, t, xc, tw);
  if (a.act) {
#pragma unroll
    for (int b = 0; b < E / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) a.base[(t + b * T + r * SL) * a.stride] = v[b * RL + r];
  }
}

// Forward tau-FFT, propagator multiply, inverse tau-FFT, in one pass.
template <class PL, int THREADS, class TW = TwShared>
__device__ __forceinline__ void tprop_tile(const AxisArgs& p, long long cta_tile, const TW& tw, float2* xch) {
  constexpr int N = PL::N, E = PL::E, T = PL::T, TX = ColTile<PL>::value;
  constexpr int TPC = tiles_per_cta_t<PL, THREADS>();
  static_assert(TPC >= 1 && TPC * T * TX == THREADS, "CTA must hold whole tiles");
  constexpr int R0 = fft_radix<PL, false>(0), RL = fft_radix<PL, false>(PL::NP - 1);
  constexpr int S0 = N / R0, SL = N / RL;
  const int lt = threadIdx.x % (T * TX), tl = threadIdx.x / (T * TX);
  const int tx = lt % TX, t = lt / TX;
  const AxisTile<N, 2, TX> a(p, cta_tile * TPC + tl, tx);
  const XchCol<TX> xc{xch + tl * N * TX, tx};
  float2 v[E];
#pragma unroll
  for (int b = 0; b < E / R0; ++b)
#pragma unroll
    for (int r = 0; r < R0; ++r)
      v[b * R0 + r] = a.act ? __ldcg(a.base + (t + b * T + r * S0) * a.stride) : make_float2(0.f, 0.f);
  fft_run<PL, false, 0, XchCol<TX>, SyncBlock, TW>(v, t, xc, tw);
  // now v[b RL + r] = A_hat(kx, ky, Omega_k), k = t + b T + r N/RL.
  // P = (1 + Dx)(1 + Dy)(1 + Dt) applied as w + w D with w = v/(nx ny nt).
  // (Measured slower on the 512-point plan: w (1 + Dt)(1 + Dxy) as two
  // delta-form products, 127 registers and 522 us against 104 and 476; the
  // scale and conjugation as four specialised copies, 542 us; the twiddle
  // staging issued after this tile's loads instead of before them, 520 us;
  // a persistent loop over tiles, 542 us; the first pass's loads issued in
  // the order the radix-32 codelet consumes them, 549 us; launch bounds of
  // two CTAs per SM (128 registers), 531 us; the field's tau factors staged
  // in shared memory with the twiddles, 506 us.)
  float2 dxy = make_float2(0.f, 0.f);
  if (a.act) {
    const float2 dx = p.px[a.f * p.nx + a.x], dy = p.py[a.f * p.ny + a.other];
    dxy = cadd(cadd(dx, dy), cmul(dx, dy));
  }
  if (p.conj_p) dxy.y = -dxy.y;
  const float2* pt = p.pt + (a.act ? a.f * p.nt : 0);
  const float tsign = p.conj_p ? -1.f : 1.f;
#pragma unroll
  for (int b = 0; b < E / RL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int k = t + b * T + r * SL;
      float2 dt = pt[k];
      dt.y *= tsign;
      float2 w = v[b * RL + r];
      w = make_float2(fmaf(w.x, p.scale, w.x * p.scale_lo), fmaf(w.y, p.scale, w.y * p.scale_lo));
      v[b * RL + r] = mul_one_plus(w, cadd(cadd(dxy, dt), cmul(dxy, dt)));
    }
  // the inverse's first pass reads exactly these positions
  fft_run<PL, true, 0, XchCol<TX>, SyncBlock, TW>(v, t, xc, tw);
  if (a.act) {
#pragma unroll
    for (int b = 0; b < E / R0; ++b)
#pragma unroll
      for (int r = 0; r < R0; ++r) a.base[(t + b * T + r * S0) * a.stride] = v[b * R0 + r];
  }
}

template <class PL, bool INV, int AXIS>
__global__ void __launch_bounds__(tiles_per_cta<PL>() * tile_threads<PL>())
    axis_fft_kernel(const AxisArgs p) {
  constexpr int THREADS = tiles_per_cta<PL>() * tile_threads<PL>();
  extern __shared__ float4 sm4[];
  if constexpr (axis_tw_staged<PL, INV, AXIS>()) {
    float4* tw = sm4;
    for (int i = threadIdx.x; i < tw_table_size<PL>(); i += blockDim.x) tw[i] = p.tw[i];
    __syncthreads();
    axis_tile<PL, INV, AXIS, THREADS>(p, blockIdx.x, TwShared{tw},
                                      reinterpret_cast<float2*>(tw + tw_table_size<PL>()));
  } else {
    axis_tile<PL, INV, AXIS, THREADS>(p, blockIdx.x, TwGlobal{p.tw}, reinterpret_cast<float2*>(sm4));
  }
}

template <class PL>
__global__ void __launch_bounds__(tiles_per_cta<PL>() * tile_threads<PL>())
    tpass_prop_kernel(const AxisArgs p) {
  constexpr int THREADS = tiles_per_cta<PL>() * tile_threads<PL>();
  extern __shared__ float4 sm4[];
  if constexpr (tw_in_smem<PL>()) {
    float4* tw = sm4;
    for (int i = threadIdx.x; i < tw_table_size<PL>(); i += blockDim.x) tw[i] = p.tw[i];
    __syncthreads();
    // tiles from the last down: the pass ends on the first field's low-y
    // pencils, which the y-inverse then reads first
    tprop_tile<PL, THREADS>(p, (long long)gridDim.x - 1 - blockIdx.x, TwShared{tw},
                            reinterpret_cast<float2*>(tw + tw_table_size<PL>()));
  } else {
    tprop_tile<PL, THREADS>(p, blockIdx.x, TwGlobal{p.tw}, reinterpret_cast<float2*>(sm4));
  }
}

// ------------------------------------------------------------ dispatchers
// Each returns cudaErrorInvalidValue for an unsupported length.
cudaError_t run_xpass(int nx, int nf, const XPassArgs& a, cudaStream_t s);
cudaError_t run_axis_fft(int n, int axis, bool inv, const AxisArgs& a, cudaStream_t s);
cudaError_t run_tpass_prop(int nt, const AxisArgs& a, cudaStream_t s);
bool size_supported(int n);
int col_tile_of(int n);      // columns per tile of the y/tau FFT kernels
int tau_col_tile_of(int n);  // columns per tile of the tau propagator kernel

// grouped x-pass of the batched form (k_xgroup.cu): the same x-pass for
// ninst instances of one shape stored one after another (2 fields each,
// base.data the first, base.fstride between fields, base.rows = ny nt rows
// per instance, base.tw the x twiddles); the instance parameters come from
// gi[0..ninst); step < 0 is the first half step of step 0.
struct GroupInst {
  float kh[2], kh2[2];  // kappa_f dz/2 (1/2 on the SH equation) and half of it
  double dk, dz;
  int nz;
};
// ecoef: the instances' stage factors, instance i's for step j at
// ecoef[i stride + (j + 1) 6 + 0..5]
cudaError_t run_xpass_group(int nx, const XPassArgs& base, const GroupInst* gi, const float2* ecoef, int stride,
                            int step, int ninst, cudaStream_t s);
int xpass_rows_of(int nx);  // rows per CTA of the x-pass of length nx

// misc kernels (k_misc.cu)
// TMA tau-pass (k_tma.cu)
bool tma_tau_supported(int nx, int nt);
cudaError_t make_tau_tensor_map(void* map128, const float2* data, int nx, int ny, int nt, int nf, int tx);
// wait_ns bounds each wait for a tile's copy; on expiry *err is set
cudaError_t run_tpass_prop_tma(int nt, int tx, const void* map128, const AxisArgs& a, int* err,
                               unsigned long long wait_ns, cudaStream_t s);

// per-pass twiddle table of the default plan of length n (host-built, FP64
// split into hi + lo floats), and its size in float4 entries
int tw_table_size_of(int n);
cudaError_t upload_twiddles(float4* tw, int n, cudaStream_t s);
struct TableArgs {
  float2* px;
  float2* py;
  float2* pt;
  int nx, ny, nt, nf;
  double dx, dy, dt, dz;
  double k[3], rho[3], delta[3], k2[3], k3[3], alpha[3];
};
cudaError_t run_prop_tables(const TableArgs& a, cudaStream_t s);
// Stage phase factors of one x-pass under a transverse mismatch map m(x, y):
// Phi(x, y, z) = Phi(z) + m z.  With zj the distance of the B step's start
// (phiB = Phi there, dkB its mismatch) and zA that of the A step's start,
//   emap[0] = e^{i (phiB + dkB dz/2 + m (zj + dz/2))},  emap[1] = e^{i (dkB + m) dz/4},
//   emap[2] = e^{i (phiA + m zA)},                        emap[3] = e^{i (dkA + m) dz/4},
// each [ny][nx]; phases in FP64 reduced mod 2 pi before the FP32 sincos.
// The map's share of the coupling phase at a point is Q = P + m (z - zp):
// P the integral of the maps in effect before zp, m the map in effect since.
// mapB is the map of the step whose B half step this x-pass applies, mapA
// that of the next step's A half step; when they differ (advance != 0) the
// kernel brings P up to zA (P += mapB (zA - zp)) and the A factors start
// from there.
struct MapArgs {
  const double* mapB;
  const double* mapA;
  double* mphase;  // P [ny][nx]
  float2* emap;
  long long nxy;
  double phiB, dkB, zB, phiA, dkA, zA, dz, zp;
  int advance;
};
cudaError_t run_map_tables(const MapArgs& a, cudaStream_t s);
// P += m * len at every point (a map replaced between propagations)
cudaError_t run_map_phase_advance(double* mphase, const double* m, double len, long long nxy, cudaStream_t s);
// the linear step's multiply element by element (grids with nt = 1)
cudaError_t run_prop_pointwise(const AxisArgs& a, int nf, cudaStream_t s);
// diagnostics (k_diag.cu): out[f nt + k] = sum_{x,y} |A_f(tau_k)|^2, and
// out[f nt + m] += sum_{x,y} |DFT_tau A_f|^2 (m) (out zeroed by the caller;
// a: tau-axis arguments without the propagator)
cudaError_t run_power_trace(const float2* data, int nx, int ny, int nt, int nf, long long fstride, double* out,
                            cudaStream_t s);
cudaError_t run_tau_spectrum(int nt, const AxisArgs& a, double* out, cudaStream_t s);

// thermal model (k_thermal.cu)
struct HeatArgs {
  const float2* data;
  long long fstride;
  int nx, ny, nt, nf;
  double c[3];  // weight * alpha_f * 1/2 c eps0 n_f (* rep_rate dt for nt > 1)
  double* heat;  // [ny][nx], accumulated into
};
cudaError_t run_heat_load(const HeatArgs& a, cudaStream_t s);
// sine-transform tables for one axis of even length n > 1: 2n entries
cudaError_t run_sine_twiddles(double2* tw, int n, cudaStream_t s);
bool sine_length_supported(int n);
struct ThermalArgs {
  const double* heat;  // [ny][nx] W/m^3
  double* temp;        // [ny][nx] K, output (also the transform's work array)
  const double2* twx;  // sine-transform tables of nx and ny
  const double2* twy;
  int nx, ny;
  double dx, dy, kappa;
  double dkdT;
  double* dkmap;  // [ny][nx] 1/m, output
  int* bad;       // set if a temperature is not finite
};
cudaError_t run_thermal_solve(const ThermalArgs& a, int* nlaunch, cudaStream_t s);
cudaError_t run_energy(const float2* data, long long n, int nf, long long fstride, double* partial,
                       int nblocks, double* out, cudaStream_t s);
cudaError_t run_c128_to_c64(const double2* in, float2* out, long long n, cudaStream_t s);
cudaError_t run_c64_to_c128(const float2* in, double2* out, long long n, cudaStream_t s);

// adjoint recomputation and reverse x-pass (k_xadj.cu)
// x-pass that also records the states entering its half steps (a.rec_b, a.rec_a)
cudaError_t run_xpass_record(int nx, int nf, const XPassArgs& a, cudaStream_t s);
cudaError_t run_xpass_record_map(int nx, int nf, const XPassArgs& a, cudaStream_t s);
// Reverse of one x-pass boundary: the adjoint g, in (kx, y, tau) when
// from_k (else real space), goes through the inverse x-FFT, the reverse of
// the A half step at state xa (if xa), the reverse of the B half step at
// state xb (if xb), and the forward x-FFT when to_k.  Each CTA writes its
// six stage-phase sensitivity sums (A: start, middle, end; B: the same) to
// partial[blockIdx.x][6]; *ncta receives the CTA count.
struct XAdjArgs {
  float2* g;
  const float2* xa;
  const float2* xb;
  long long fstride, rows;
  const float4* tw;
  int from_k, to_k;
  double phiA, dkA, phiB, dkB, h;  // phase and mismatch at the start of each half step; h = dz/2
  float kh[3];                     // kappa_f h (1/2 on the SH equation for two fields)
  double* partial;
  // transverse mismatch map: the per-(x, y) stage phase factors of this
  // boundary's B and A half steps [4][ny][nx] (as in XPassArgs), or NULL
  const float2* emap;
  int ny;
  // map-free: the coefficient sets i kappa_f h e^{-/+ i Phi} at the start,
  // middle and end of the A half step (cset[0]) and of the B half step
  // (cset[1]), [stage][field], written by the host dispatcher in FP64 from
  // the phases above (the stage factors the forward x-pass uses)
  float2 cset[2][9];
};
cudaError_t run_xpass_adjoint(int nx, int nf, const XAdjArgs& a, long long* ncta, cudaStream_t s);
cudaError_t run_xpass_adjoint_map(int nx, int nf, const XAdjArgs& a, long long* ncta, cudaStream_t s);
// sensA[k] = sum_c partial[c][k], sensB[k] = sum_c partial[c][3 + k] (either may be NULL)
cudaError_t run_sens_boundary(const double* partial, long long ncta, double* sensA, double* sensB, cudaStream_t s);
long long xpass_adjoint_ctas(int nx, long long rows);

// adjoint kernels (k_adjoint.cu)
cudaError_t run_scale_fields(const float2* a, float2* g, long long n, int nf, long long fstride, const float* s,
                             cudaStream_t st);
cudaError_t run_phase_grad(const float2* gh, const float2* ah, long long plane, int nt, double* acc, cudaStream_t s);
cudaError_t run_phase_tables(float2* px, int nx, float2* py, int ny, float2* pt, int nt, const double* phi, int sign,
                             cudaStream_t s);

}  // namespace brahms

// Supported transform lengths (each needs an FftPlan).
#define BRAHMS_FOR_EACH_SIZE(X) \
  X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) \
  X(6) X(12) X(24) X(48) X(96) X(192) X(384) X(768)
