// Reverse mode of the RK4 half step (Sec. 3.1) at one grid point, shared by
// the stand-alone VJP kernel and the fused adjoint x-pass.
//
// Complex gradients follow G_z = dJ/dRe z + i dJ/dIm z.  For y = f(x):
//   G_x = sum_y [ conj(G_y) dy/dconj(x) + G_y conj(dy/dx) ].
// The stages are recomputed in registers from the state at the start of the
// half step; the mismatch phase sensitivity at a stage is
//   dJ/dPhi = sum_f Re( conj(G_k_f) dk_f/dPhi ),  dk_0/dPhi = -i k_0,
//   dk_f/dPhi = +i k_f (f >= 1).
#pragma once

#include "kernels.cuh"

namespace brahms {

__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// Im(conj(a) b)
__device__ __forceinline__ float im_cb(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }

// gu += adjoint of k = f(u) (coefficients c) applied to gk
template <int F>
__device__ __forceinline__ void rhs_vjp(const float2* __restrict__ c, const float2 (&u)[F], const float2 (&gk)[F],
                                        float2 (&gu)[F]) {
  if constexpr (F == 3) {
    gu[0] = cadd(gu[0], cadd(cmul(gk[1], cmul(cconj(c[1]), u[2])), cmul(gk[2], cmul(cconj(c[2]), u[1]))));
    gu[1] = cadd(gu[1], cadd(cmul(gk[0], cmul(cconj(c[0]), cconj(u[2]))), cmul(cconj(gk[2]), cmul(c[2], u[0]))));
    gu[2] = cadd(gu[2], cadd(cmul(gk[0], cmul(cconj(c[0]), cconj(u[1]))), cmul(cconj(gk[1]), cmul(c[1], u[0]))));
  } else {
    gu[0] = cadd(gu[0], cmul(gk[1], cmul(cconj(c[1]), u[1])));
    const float2 t = cmul(gk[0], cmul(cconj(c[0]), cconj(u[1])));
    gu[1] = cadd(gu[1], cadd(cadd(t, t), cmul(cconj(gk[1]), cmul(c[1], u[0]))));
  }
}

// sum_f Re(conj(gk_f) dk_f/dPhi)
template <int F>
__device__ __forceinline__ float phase_sens(const float2 (&gk)[F], const float2 (&k)[F]) {
  float s = im_cb(gk[0], k[0]);  // Re(conj(g)(-i k)) = Im(conj(g) k)
#pragma unroll
  for (int f = 1; f < F; ++f) s -= im_cb(gk[f], k[f]);
  return s;
}

// One RK4 half step in reverse at a point: x is the forward state at the
// start of the half step, c the coefficient sets i kappa h e^{-/+ i Phi} at
// the start, middle and end ([3][F]); g enters as the gradient with respect
// to the end state and leaves as the gradient with respect to x.  s0, s1, s2
// gain the sensitivities to the stage phases at the start, the midpoint
// (both middle stages) and the end.
template <int F>
__device__ __forceinline__ void rk4_vjp_point(const float2 (&x)[F], float2 (&g)[F], const float2* __restrict__ c,
                                              float& s0, float& s1, float& s2) {
  float2 u2[F], u3[F], u4[F], k1[F], k2[F], k3[F], k4[F];
  nl_rhs<F>(x, c, k1);
#pragma unroll
  for (int f = 0; f < F; ++f) u2[f] = make_float2(fmaf(0.5f, k1[f].x, x[f].x), fmaf(0.5f, k1[f].y, x[f].y));
  nl_rhs<F>(u2, c + F, k2);
#pragma unroll
  for (int f = 0; f < F; ++f) u3[f] = make_float2(fmaf(0.5f, k2[f].x, x[f].x), fmaf(0.5f, k2[f].y, x[f].y));
  nl_rhs<F>(u3, c + F, k3);
#pragma unroll
  for (int f = 0; f < F; ++f) u4[f] = cadd(x[f], k3[f]);
  nl_rhs<F>(u4, c + 2 * F, k4);
  // y = x + (k1 + 2 k2 + 2 k3 + k4)/6
  float2 gx[F], g1[F], g2[F], g3[F], g4[F], gu[F];
#pragma unroll
  for (int f = 0; f < F; ++f) {
    gx[f] = g[f];
    g1[f] = cscale(g[f], 1.f / 6.f);
    g2[f] = cscale(g[f], 1.f / 3.f);
    g3[f] = g2[f];
    g4[f] = g1[f];
    gu[f] = make_float2(0.f, 0.f);
  }
  // stage 4: u4 = x + k3
  rhs_vjp<F>(c + 2 * F, u4, g4, gu);
  s2 += phase_sens<F>(g4, k4);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    gx[f] = cadd(gx[f], gu[f]);
    g3[f] = cadd(g3[f], gu[f]);
    gu[f] = make_float2(0.f, 0.f);
  }
  // stage 3: u3 = x + k2/2
  rhs_vjp<F>(c + F, u3, g3, gu);
  s1 += phase_sens<F>(g3, k3);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    gx[f] = cadd(gx[f], gu[f]);
    g2[f] = make_float2(fmaf(0.5f, gu[f].x, g2[f].x), fmaf(0.5f, gu[f].y, g2[f].y));
    gu[f] = make_float2(0.f, 0.f);
  }
  // stage 2: u2 = x + k1/2
  rhs_vjp<F>(c + F, u2, g2, gu);
  s1 += phase_sens<F>(g2, k2);
#pragma unroll
  for (int f = 0; f < F; ++f) {
    gx[f] = cadd(gx[f], gu[f]);
    g1[f] = make_float2(fmaf(0.5f, gu[f].x, g1[f].x), fmaf(0.5f, gu[f].y, g1[f].y));
    gu[f] = make_float2(0.f, 0.f);
  }
  // stage 1: u1 = x
  rhs_vjp<F>(c, x, g1, gu);
  s0 += phase_sens<F>(g1, k1);
#pragma unroll
  for (int f = 0; f < F; ++f) g[f] = cadd(gx[f], gu[f]);
}

// Coefficient sets c = i kappa_f h e^{-/+ i Phi} (minus for field 0) at the
// start, middle and end of a half step from phase phi_a with mismatch dk
// (thread s < 3 writes set s).
template <int F>
__device__ __forceinline__ void vjp_coef_sets(double phi_a, double dk, double h, const float* kh, float2* c) {
  const int s = threadIdx.x;
  if (s < 3) {
    const double phi = phi_a + dk * (0.5 * h * s);
    const float2 em = phase_minus(phi);
#pragma unroll
    for (int f = 0; f < F; ++f) {
      const float k = kh[f];
      c[s * F + f] = f == 0 ? make_float2(-em.y * k, em.x * k) : make_float2(em.y * k, em.x * k);
    }
  }
}

}  // namespace brahms
