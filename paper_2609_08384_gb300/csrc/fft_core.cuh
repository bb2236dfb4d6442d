// Register-resident mixed-radix Stockham FFT building blocks for sm_103a.
//
// A pencil of length N is owned by T = N/E threads; each thread keeps E
// complex values in registers.  One Stockham pass of radix R (Govindaraju et
// al., "High performance discrete Fourier transforms on graphics processors",
// SC'08, autosort formulation) reads the R inputs j + r N/R of butterfly j,
// multiplies by W_N^{r (j mod Ns) N/(Ns R)}, applies a radix-R DFT and writes
// the results to (j/Ns) Ns R + (j mod Ns) + r Ns.  Between passes the values
// are exchanged through shared memory; the first pass reads its inputs
// straight from global memory and the last pass leaves the outputs in
// registers at positions j + r N/R_last, so a kernel stores them with
// coalesced writes and never stages the whole pencil twice.
//
// The forward transform is unnormalised with e^{-2 pi i m n / N}; the inverse
// uses e^{+...} and the radix order reversed, so that the inverse's first
// pass reads exactly the positions the forward's last pass produced.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace brahms {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward sign) or +i (inverse sign)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// Irrational codelet constants as hi + lo float pairs.  Rounded to one float
// each, cos(pi/4), cos(pi/8) and sin(pi/8) all have |w| slightly below 1
// (|w|^2 - 1 = -3.4e-8 for the pi/4 pair, -5.7e-8 for the pi/8 pair), and
// because a z-step applies the same factors again and again the field energy
// would drift by about -2e-7 per step.  Multiplying by hi and lo (one extra
// FMA) makes each product correctly rounded, so rounding errors are unbiased.
constexpr double kS2d = 0.70710678118654752440084436210485;   // cos(pi/4)
constexpr double kC16d = 0.92387953251128675612818318939679;  // cos(pi/8)
constexpr double kS16d = 0.38268343236508977172845998403040;  // sin(pi/8)
constexpr double kS3d = 0.86602540378443864676372317075294;   // sin(pi/3)
constexpr float kS2 = (float)kS2d, kS2lo = (float)(kS2d - (double)(float)kS2d);
constexpr float kC16 = (float)kC16d, kC16lo = (float)(kC16d - (double)(float)kC16d);
constexpr float kS16 = (float)kS16d, kS16lo = (float)(kS16d - (double)(float)kS16d);
constexpr float kS3 = (float)kS3d, kS3lo = (float)(kS3d - (double)(float)kS3d);

// u * c with c = hi + lo
__device__ __forceinline__ float xmul(float u, float hi, float lo) { return fmaf(u, hi, u * lo); }
// a * (c -/+ i s) with c = ch + cl, s = sh + sl (forward uses minus)
template <bool INV>
__device__ __forceinline__ float2 twx(float2 a, float ch, float cl, float sh, float sl) {
  if (INV)
    return make_float2(fmaf(a.x, ch, fmaf(-a.y, sh, fmaf(a.x, cl, -a.y * sl))),
                       fmaf(a.y, ch, fmaf(a.x, sh, fmaf(a.y, cl, a.x * sl))));
  return make_float2(fmaf(a.x, ch, fmaf(a.y, sh, fmaf(a.x, cl, a.y * sl))),
                     fmaf(a.y, ch, fmaf(-a.x, sh, fmaf(a.y, cl, -a.x * sl))));
}
// a * W8^1 (forward: (1 - i)/sqrt 2; inverse: (1 + i)/sqrt 2)
template <bool INV>
__device__ __forceinline__ float2 w8_1(float2 a) {
  return INV ? make_float2(xmul(a.x - a.y, kS2, kS2lo), xmul(a.x + a.y, kS2, kS2lo))
             : make_float2(xmul(a.x + a.y, kS2, kS2lo), xmul(a.y - a.x, kS2, kS2lo));
}
// a * W8^3 (forward: (-1 - i)/sqrt 2; inverse: (-1 + i)/sqrt 2)
template <bool INV>
__device__ __forceinline__ float2 w8_3(float2 a) {
  return INV ? make_float2(-xmul(a.x + a.y, kS2, kS2lo), xmul(a.x - a.y, kS2, kS2lo))
             : make_float2(xmul(a.y - a.x, kS2, kS2lo), -xmul(a.x + a.y, kS2, kS2lo));
}

// ---------------------------------------------------------------- codelets
template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  float2 a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = rot90<INV>(csub(v1, v3));
  v0 = cadd(a, c);
  v2 = csub(a, c);
  v1 = cadd(b, d);
  v3 = csub(b, d);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2& v0, float2& v1, float2& v2) {
  float2 s = cadd(v1, v2);
  float2 t = make_float2(fmaf(-0.5f, s.x, v0.x), fmaf(-0.5f, s.y, v0.y));
  const float2 d = csub(v1, v2);
  float2 u = rot90<INV>(make_float2(xmul(d.x, kS3, kS3lo), xmul(d.y, kS3, kS3lo)));
  v0 = cadd(v0, s);
  v1 = cadd(t, u);
  v2 = csub(t, u);
}

// radix 8 = 2 x 4: n = 4 n1 + n2, k = k1 + 2 k2
template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  float2 y0[4], y1[4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    y0[n2] = cadd(v[n2], v[n2 + 4]);
    y1[n2] = csub(v[n2], v[n2 + 4]);
  }
  y1[1] = w8_1<INV>(y1[1]);
  y1[2] = rot90<INV>(y1[2]);
  y1[3] = w8_3<INV>(y1[3]);
  dft4<INV>(y0[0], y0[1], y0[2], y0[3]);
  dft4<INV>(y1[0], y1[1], y1[2], y1[3]);
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    v[2 * k2] = y0[k2];
    v[2 * k2 + 1] = y1[k2];
  }
}

// multiply by W16^e, e in [0, 9]
template <bool INV, int E>
__device__ __forceinline__ float2 w16(float2 a) {
  if constexpr (E == 0) return a;
  else if constexpr (E == 1) return twx<INV>(a, kC16, kC16lo, kS16, kS16lo);
  else if constexpr (E == 2) return w8_1<INV>(a);
  else if constexpr (E == 3) return twx<INV>(a, kS16, kS16lo, kC16, kC16lo);
  else if constexpr (E == 4) return rot90<INV>(a);
  else if constexpr (E == 6) return w8_3<INV>(a);
  else if constexpr (E == 9) return twx<INV>(a, -kC16, -kC16lo, -kS16, -kS16lo);
  else return a;
}

// radix 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  float2 y[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 a0 = v[n2], a1 = v[4 + n2], a2 = v[8 + n2], a3 = v[12 + n2];
    dft4<INV>(a0, a1, a2, a3);
    y[n2][0] = a0;
    y[n2][1] = a1;
    y[n2][2] = a2;
    y[n2][3] = a3;
  }
  y[1][1] = w16<INV, 1>(y[1][1]);
  y[1][2] = w16<INV, 2>(y[1][2]);
  y[1][3] = w16<INV, 3>(y[1][3]);
  y[2][1] = w16<INV, 2>(y[2][1]);
  y[2][2] = w16<INV, 4>(y[2][2]);
  y[2][3] = w16<INV, 6>(y[2][3]);
  y[3][1] = w16<INV, 3>(y[3][1]);
  y[3][2] = w16<INV, 6>(y[3][2]);
  y[3][3] = w16<INV, 9>(y[3][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 b0 = y[0][k1], b1 = y[1][k1], b2 = y[2][k1], b3 = y[3][k1];
    dft4<INV>(b0, b1, b2, b3);
    v[k1] = b0;
    v[k1 + 4] = b1;
    v[k1 + 8] = b2;
    v[k1 + 12] = b3;
  }
}

// cos(pi k / 16) for any integer k, in double (compile time): the first
// quadrant's values, the rest by symmetry.
__host__ __device__ constexpr double cos_pi16_q(int k) {
  return k == 0 ? 1.0
       : k == 1 ? 0.98078528040323044912618223613424
       : k == 2 ? 0.92387953251128675612818318939679
       : k == 3 ? 0.83146961230254523707878837761791
       : k == 4 ? 0.70710678118654752440084436210485
       : k == 5 ? 0.55557023301960222474283081394853
       : k == 6 ? 0.38268343236508977172845998403040
       : k == 7 ? 0.19509032201612826784828486847702
                : 0.0;
}
__host__ __device__ constexpr double cos_pi16(int k) {
  return (k % 32 + 32) % 32 > 16 ? cos_pi16(32 - (k % 32 + 32) % 32)
       : (k % 32 + 32) % 32 > 8  ? -cos_pi16_q(16 - (k % 32 + 32) % 32)
                                 : cos_pi16_q((k % 32 + 32) % 32);
}
__host__ __device__ constexpr double sin_pi16(int k) { return cos_pi16(8 - k); }
__host__ __device__ constexpr float hi_of(double v) { return (float)v; }
__host__ __device__ constexpr float lo_of(double v) { return (float)(v - (double)(float)v); }

// multiply by W32^e = e^{-/+ 2 pi i e / 32}: the exact cases (multiples of
// 8) as swaps and signs, the others through W16 or as hi + lo products
template <bool INV, int E>
__device__ __forceinline__ float2 w32(float2 a) {
  if constexpr (E % 2 == 0 && (E / 2 <= 4 || E / 2 == 6 || E / 2 == 9)) return w16<INV, E / 2>(a);
  else if constexpr (E == 16) return make_float2(-a.x, -a.y);
  else {
    constexpr double c = cos_pi16(E), s = sin_pi16(E);
    return twx<INV>(a, hi_of(c), lo_of(c), hi_of(s), lo_of(s));
  }
}

// radix 32 = 8 x 4: n = 4 n1 + n2 (n1 < 8, n2 < 4), k = k1 + 8 k2; eight-point
// transforms over n1, twiddles W32^{n2 k1}, four-point transforms over n2
template <bool INV>
__device__ __forceinline__ void dft32(float2* v) {
  float2 y[4][8];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) y[n2][n1] = v[4 * n1 + n2];
    dft8<INV>(y[n2]);
  }
#define BRAHMS_W32_ROW(N2)                   \
  y[N2][1] = w32<INV, N2 * 1>(y[N2][1]);     \
  y[N2][2] = w32<INV, N2 * 2>(y[N2][2]);     \
  y[N2][3] = w32<INV, N2 * 3>(y[N2][3]);     \
  y[N2][4] = w32<INV, N2 * 4>(y[N2][4]);     \
  y[N2][5] = w32<INV, N2 * 5>(y[N2][5]);     \
  y[N2][6] = w32<INV, N2 * 6>(y[N2][6]);     \
  y[N2][7] = w32<INV, N2 * 7>(y[N2][7]);
  BRAHMS_W32_ROW(1)
  BRAHMS_W32_ROW(2)
  BRAHMS_W32_ROW(3)
#undef BRAHMS_W32_ROW
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    float2 b0 = y[0][k1], b1 = y[1][k1], b2 = y[2][k1], b3 = y[3][k1];
    dft4<INV>(b0, b1, b2, b3);
    v[k1] = b0;
    v[k1 + 8] = b1;
    v[k1 + 16] = b2;
    v[k1 + 24] = b3;
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
  else if constexpr (R == 32) dft32<INV>(v);
  else static_assert(R == 2, "unsupported radix");
}

// ------------------------------------------------------------------- plans
// A plan: length N, registers per thread E (a multiple of every radix), and
// the forward radix sequence.  Kernels pick a plan per length.
template <int N_, int E_, int NP_, int R0_, int R1_ = 0, int R2_ = 0, int R3_ = 0>
struct Plan {
  static constexpr int N = N_;
  static constexpr int E = E_;
  static constexpr int NP = NP_;
  static constexpr int T = N_ / E_;  // threads per pencil
  __host__ __device__ static constexpr int r(int p) { return p == 0 ? R0_ : p == 1 ? R1_ : p == 2 ? R2_ : R3_; }
};

// default plans (x- and y-passes)
template <int N>
struct FftPlan;
template <> struct FftPlan<2> : Plan<2, 2, 1, 2> {};
template <> struct FftPlan<4> : Plan<4, 4, 1, 4> {};
template <> struct FftPlan<8> : Plan<8, 8, 1, 8> {};
template <> struct FftPlan<16> : Plan<16, 16, 1, 16> {};
template <> struct FftPlan<32> : Plan<32, 8, 2, 4, 8> {};
template <> struct FftPlan<64> : Plan<64, 8, 2, 8, 8> {};
template <> struct FftPlan<128> : Plan<128, 16, 2, 16, 8> {};
template <> struct FftPlan<256> : Plan<256, 16, 2, 16, 16> {};
// 512 = 32 x 16 (two passes, one exchange): measured on GB300 for the tau
// propagator of the 3 x 256x256x512 state, 473 us per launch against 546 for
// 8 x 8 x 8 and 610 for 16 x 32
template <> struct FftPlan<512> : Plan<512, 32, 2, 32, 16> {};
template <> struct FftPlan<1024> : Plan<1024, 16, 3, 16, 8, 8> {};
template <> struct FftPlan<2048> : Plan<2048, 16, 3, 16, 16, 8> {};
template <> struct FftPlan<4096> : Plan<4096, 16, 3, 16, 16, 16> {};
template <> struct FftPlan<6> : Plan<6, 6, 2, 3, 2> {};
template <> struct FftPlan<12> : Plan<12, 12, 2, 3, 4> {};
template <> struct FftPlan<24> : Plan<24, 12, 3, 3, 2, 4> {};
template <> struct FftPlan<48> : Plan<48, 12, 3, 3, 4, 4> {};
template <> struct FftPlan<96> : Plan<96, 12, 4, 3, 4, 4, 2> {};
template <> struct FftPlan<192> : Plan<192, 12, 4, 3, 4, 4, 4> {};
template <> struct FftPlan<384> : Plan<384, 24, 4, 3, 8, 4, 4> {};
template <> struct FftPlan<768> : Plan<768, 24, 4, 3, 4, 8, 8> {};

// tau-pass plans (a 512-point plan with 8 values per thread and 1024-thread
// tiles measured slower on GB300 than the default, 742 vs 709 us per OPG
// launch; the tau pass shares the default plans and their twiddle tables)
template <int N>
struct TauPlan : FftPlan<N> {};

template <class PL, bool INV>
__host__ __device__ constexpr int fft_radix(int p) {
  return INV ? PL::r(PL::NP - 1 - p) : PL::r(p);
}
template <class PL, bool INV>
__host__ __device__ constexpr int fft_ns(int p) {
  int s = 1;
  for (int q = 0; q < p; ++q) s *= fft_radix<PL, INV>(q);
  return s;
}

// ---------------------------------------------------------------- exchange
// Contiguous pencil (one row of x): one padding slot per 16 entries.
struct XchRow {
  static constexpr bool kSplit = false;
  float2* base;
  __device__ __forceinline__ void st(int pos, float2 v) const { base[pos + (pos >> 4)] = v; }
  __device__ __forceinline__ float2 ld(int pos) const { return base[pos + (pos >> 4)]; }
  __host__ __device__ static constexpr int pitch(int n) { return n + n / 16 + 1; }
};
// Strided pencils: TX neighbouring columns, column index fastest.
template <int TX>
struct XchCol {
  static constexpr bool kSplit = false;
  float2* base;
  int tx;
  __device__ __forceinline__ void st(int pos, float2 v) const { base[pos * TX + tx] = v; }
  __device__ __forceinline__ float2 ld(int pos) const { return base[pos * TX + tx]; }
};
// The same layout for one real component at a time: the exchange runs in two
// rounds (real parts, then imaginary parts) through half the shared memory.
template <int TX>
struct XchColSplit {
  static constexpr bool kSplit = true;
  float* base;
  int tx;
  __device__ __forceinline__ void st(int pos, float v) const { base[pos * TX + tx] = v; }
  __device__ __forceinline__ float ld(int pos) const { return base[pos * TX + tx]; }
};

// Twiddle tables hold W = (c, s) as hi + lo float pairs, float4 (ch, sh, cl,
// sl): a product with the table is then correctly rounded, so the FFT carries
// no systematic modulus error from rounded twiddles.
__device__ __forceinline__ float2 tw_mul(float2 a, float4 w) { return twx<true>(a, w.x, w.z, w.y, w.w); }

// Per-pass layout: pass P >= 1 of a direction with radix R and stride NS owns
// the R x NS block [r][m] = exp(-/+ 2 pi i r m / (NS R)) (inverse entries are
// stored conjugated), so the threads of a warp, whose butterflies have
// consecutive m, read consecutive entries.  Forward blocks come first.
template <class PL, bool INV>
__host__ __device__ constexpr int tw_dir_size() {
  int s = 0, ns = 1;
  for (int q = 0; q < PL::NP; ++q) {
    const int r = INV ? PL::r(PL::NP - 1 - q) : PL::r(q);
    if (q > 0) s += r * ns;
    ns *= r;
  }
  return s;
}
template <class PL, bool INV>
__host__ __device__ constexpr int tw_pass_off(int P) {
  int o = INV ? tw_dir_size<PL, false>() : 0, ns = 1;
  for (int q = 0; q < P; ++q) {
    const int r = INV ? PL::r(PL::NP - 1 - q) : PL::r(q);
    if (q > 0) o += r * ns;
    ns *= r;
  }
  return o;
}
template <class PL>
__host__ __device__ constexpr int tw_table_size() {
  return tw_dir_size<PL, false>() + tw_dir_size<PL, true>() > 0 ? tw_dir_size<PL, false>() + tw_dir_size<PL, true>()
                                                                  : 1;
}

// twiddle access from shared memory or, read-only, through L1
struct TwShared {
  const float4* p;
  __device__ __forceinline__ float4 operator()(int i) const { return p[i]; }
};
struct TwGlobal {
  const float4* p;
  __device__ __forceinline__ float4 operator()(int i) const { return __ldg(p + i); }
};

// Barrier used around shared-memory exchanges: the whole CTA, or only the
// warp when every pencil's threads lie inside one warp.
struct SyncBlock {
  __device__ __forceinline__ static void sync() { __syncthreads(); }
};
struct SyncWarp {
  __device__ __forceinline__ static void sync() { __syncwarp(); }
};

// Passes P..NP-1 of a length-N transform on the registers v (see header).
// Every thread that shares a barrier of type S must call this.
template <class PL, bool INV, int P, class X, class S = SyncBlock, class TW = TwShared>
__device__ __forceinline__ void fft_run(float2 (&v)[PL::E], int t, const X& x, const TW& tw) {
  constexpr int N = PL::N;
  constexpr int NP = PL::NP;
  constexpr int E = PL::E;
  constexpr int T = PL::T;
  constexpr int R = fft_radix<PL, INV>(P);
  constexpr int NS = fft_ns<PL, INV>(P);
  constexpr int B = E / R;
  static_assert(E % R == 0, "E must be a multiple of every radix");
  if constexpr (NS > 1) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * T;
      const int m = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        v[b * R + r] = tw_mul(v[b * R + r], tw(tw_pass_off<PL, INV>(P) + r * NS + m));
      }
    }
  }
#pragma unroll
  for (int b = 0; b < B; ++b) dft<R, INV>(&v[b * R]);
  if constexpr (P + 1 < NP) {
    constexpr int R2 = fft_radix<PL, INV>(P + 1);
    constexpr int B2 = E / R2;
    if constexpr (X::kSplit) {
      // real parts, then imaginary parts, through the same buffer
      float re[E];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        S::sync();  // earlier readers of the exchange buffer are done
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int j = t + b * T;
          const int m = j % NS;
          const int d = (j / NS) * NS * R + m;
#pragma unroll
          for (int r = 0; r < R; ++r) x.st(d + r * NS, c == 0 ? v[b * R + r].x : v[b * R + r].y);
        }
        S::sync();
#pragma unroll
        for (int b = 0; b < B2; ++b) {
          const int j = t + b * T;
#pragma unroll
          for (int r = 0; r < R2; ++r) {
            const float u = x.ld(j + r * (N / R2));
            if (c == 0)
              re[b * R2 + r] = u;
            else
              v[b * R2 + r] = make_float2(re[b * R2 + r], u);
          }
        }
      }
    } else {
      S::sync();  // earlier readers of the exchange buffer are done
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int j = t + b * T;
        const int m = j % NS;
        const int d = (j / NS) * NS * R + m;
#pragma unroll
        for (int r = 0; r < R; ++r) x.st(d + r * NS, v[b * R + r]);
      }
      S::sync();
#pragma unroll
      for (int b = 0; b < B2; ++b) {
        const int j = t + b * T;
#pragma unroll
        for (int r = 0; r < R2; ++r) v[b * R2 + r] = x.ld(j + r * (N / R2));
      }
    }
    fft_run<PL, INV, P + 1, X, S, TW>(v, t, x, tw);
  }
}

}  // namespace brahms
