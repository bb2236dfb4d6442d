// Kernels of the discrete adjoint of the split step.
//
// Complex gradients follow G_z = dJ/dRe z + i dJ/dIm z.  For y = f(x):
//   G_x = sum_y [ conj(G_y) dy/dconj(x) + G_y conj(dy/dx) ].
// The RK4 half step is reversed stage by stage after recomputing its stages
// in registers; the mismatch phase sensitivity at a stage is
//   dJ/dPhi = sum_f Re( conj(G_k_f) dk_f/dPhi ),  dk_0/dPhi = -i k_0,
//   dk_f/dPhi = +i k_f (f >= 1),
// accumulated per block in FP64.
#include "kernels.cuh"

namespace brahms {

struct VjpArgs {
  const float2* x;  // forward state at the start of the half step, [F][n]
  float2* g;        // adjoint, in place, [F][n]
  long long n, fstride;
  double phi_a, dk, h;
  float kh[3];      // kappa_f * h (1/2 on the SH equation for two fields)
  double* partial;  // [gridDim.x][3]
};

// coefficient sets (i kappa h e^{-/+ i Phi}) at the start, middle, end
template <int F>
__device__ __forceinline__ void vjp_coefficients(const VjpArgs& p, float2* c) {
  const int s = threadIdx.x;
  if (s < 3) {
    const double phi = p.phi_a + p.dk * (0.5 * p.h * s);
    const float2 em = phase_minus(phi);
#pragma unroll
    for (int f = 0; f < F; ++f) {
      const float kh = p.kh[f];
      c[s * F + f] = f == 0 ? make_float2(-em.y * kh, em.x * kh) : make_float2(em.y * kh, em.x * kh);
    }
  }
}

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

template <int F>
__global__ void __launch_bounds__(256) rk4_vjp_kernel(const VjpArgs p) {
  __shared__ float2 c[3 * F];
  __shared__ double red[8][3];
  vjp_coefficients<F>(p, c);
  __syncthreads();
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += (long long)gridDim.x * blockDim.x) {
    float2 u1[F], u2[F], u3[F], u4[F], k1[F], k2[F], k3[F], k4[F], gy[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      u1[f] = __ldcg(p.x + f * p.fstride + i);
      gy[f] = __ldcg(p.g + f * p.fstride + i);
    }
    // forward stages (k scaled by h), as in rk4()
    nl_rhs<F>(u1, c, k1);
#pragma unroll
    for (int f = 0; f < F; ++f) u2[f] = make_float2(fmaf(0.5f, k1[f].x, u1[f].x), fmaf(0.5f, k1[f].y, u1[f].y));
    nl_rhs<F>(u2, c + F, k2);
#pragma unroll
    for (int f = 0; f < F; ++f) u3[f] = make_float2(fmaf(0.5f, k2[f].x, u1[f].x), fmaf(0.5f, k2[f].y, u1[f].y));
    nl_rhs<F>(u3, c + F, k3);
#pragma unroll
    for (int f = 0; f < F; ++f) u4[f] = cadd(u1[f], k3[f]);
    nl_rhs<F>(u4, c + 2 * F, k4);
    // y = u1 + (k1 + 2 k2 + 2 k3 + k4)/6
    float2 gx[F], g1[F], g2[F], g3[F], g4[F], gu[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      gx[f] = gy[f];
      g1[f] = cscale(gy[f], 1.f / 6.f);
      g2[f] = cscale(gy[f], 1.f / 3.f);
      g3[f] = g2[f];
      g4[f] = g1[f];
      gu[f] = make_float2(0.f, 0.f);
    }
    // stage 4: u4 = u1 + k3
    rhs_vjp<F>(c + 2 * F, u4, g4, gu);
    s2 += (double)phase_sens<F>(g4, k4);
#pragma unroll
    for (int f = 0; f < F; ++f) {
      gx[f] = cadd(gx[f], gu[f]);
      g3[f] = cadd(g3[f], gu[f]);
      gu[f] = make_float2(0.f, 0.f);
    }
    // stage 3: u3 = u1 + k2/2
    rhs_vjp<F>(c + F, u3, g3, gu);
    s1 += (double)phase_sens<F>(g3, k3);
#pragma unroll
    for (int f = 0; f < F; ++f) {
      gx[f] = cadd(gx[f], gu[f]);
      g2[f] = make_float2(fmaf(0.5f, gu[f].x, g2[f].x), fmaf(0.5f, gu[f].y, g2[f].y));
      gu[f] = make_float2(0.f, 0.f);
    }
    // stage 2: u2 = u1 + k1/2
    rhs_vjp<F>(c + F, u2, g2, gu);
    s1 += (double)phase_sens<F>(g2, k2);
#pragma unroll
    for (int f = 0; f < F; ++f) {
      gx[f] = cadd(gx[f], gu[f]);
      g1[f] = make_float2(fmaf(0.5f, gu[f].x, g1[f].x), fmaf(0.5f, gu[f].y, g1[f].y));
      gu[f] = make_float2(0.f, 0.f);
    }
    // stage 1: u1 = x
    rhs_vjp<F>(c, u1, g1, gu);
    s0 += (double)phase_sens<F>(g1, k1);
#pragma unroll
    for (int f = 0; f < F; ++f) p.g[f * p.fstride + i] = cadd(gx[f], gu[f]);
  }
  // block reduction (fixed order: deterministic)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = s0;
    red[threadIdx.x >> 5][1] = s1;
    red[threadIdx.x >> 5][2] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
    p.partial[blockIdx.x * 3 + threadIdx.x] = t;
  }
}

cudaError_t run_rk4_vjp(int nf, const float2* x, float2* g, long long n, long long fstride, double phi_a, double dk,
                        double h, const float* kh, double* partial, int nblocks, cudaStream_t s) {
  VjpArgs a{};
  a.x = x;
  a.g = g;
  a.n = n;
  a.fstride = fstride;
  a.phi_a = phi_a;
  a.dk = dk;
  a.h = h;
  for (int f = 0; f < nf; ++f) a.kh[f] = kh[f];
  a.partial = partial;
  if (nf == 3) rk4_vjp_kernel<3><<<nblocks, 256, 0, s>>>(a);
  else rk4_vjp_kernel<2><<<nblocks, 256, 0, s>>>(a);
  return cudaPeekAtLastError();
}

// g_f = s_f a_f
__global__ void scale_fields_kernel(const float2* __restrict__ a, float2* __restrict__ g, long long n, int nf,
                                    long long fstride, float s0, float s1, float s2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll 3
    for (int f = 0; f < nf; ++f) {
      const float s = f == 0 ? s0 : (f == 1 ? s1 : s2);
      g[f * fstride + i] = cscale(__ldcg(a + f * fstride + i), s);
    }
  }
}

cudaError_t run_scale_fields(const float2* a, float2* g, long long n, int nf, long long fstride, const float* s,
                             cudaStream_t st) {
  scale_fields_kernel<<<152 * 4, 256, 0, st>>>(a, g, n, nf, fstride, s[0], nf > 1 ? s[1] : 0.f,
                                               nf > 2 ? s[2] : 0.f);
  return cudaPeekAtLastError();
}

// acc[m] = sum over the (x, y) plane of Im(conj(G_hat) A_hat) at tau-bin m
__global__ void __launch_bounds__(256) phase_grad_kernel(const float2* __restrict__ gh, const float2* __restrict__ ah,
                                                         long long plane, double* acc) {
  const float2* g = gh + (long long)blockIdx.x * plane;
  const float2* a = ah + (long long)blockIdx.x * plane;
  double s = 0.0;
  for (long long q = threadIdx.x; q < plane; q += blockDim.x) s += (double)im_cb(__ldcg(g + q), __ldcg(a + q));
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    acc[blockIdx.x] = t;
  }
}

cudaError_t run_phase_grad(const float2* gh, const float2* ah, long long plane, int nt, double* acc, cudaStream_t s) {
  phase_grad_kernel<<<nt, 256, 0, s>>>(gh, ah, plane, acc);
  return cudaPeekAtLastError();
}

// sens[j][k] = sum_b partial[j][b][k] (k < 6: half A stages, half B stages)
__global__ void sens_reduce_kernel(const double* __restrict__ partial, int nblocks, double* sens) {
  const int j = blockIdx.x;
  if (threadIdx.x < 6) {
    const int half = threadIdx.x / 3, k = threadIdx.x % 3;
    const double* p = partial + ((long long)j * 2 + half) * nblocks * 3;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += p[b * 3 + k];
    sens[j * 6 + threadIdx.x] = t;
  }
}

cudaError_t run_sens_reduce(const double* partial, int nblocks, int nz, double* sens, cudaStream_t s) {
  sens_reduce_kernel<<<nz, 32, 0, s>>>(partial, nblocks, sens);
  return cudaPeekAtLastError();
}

// Spectral-phase propagator tables in delta form: px = py = 0 (identity),
// pt[m] = e^{i sign phi[(m + nt/2) mod nt]} - 1 for the centred phase vector.
__global__ void phase_tables_kernel(float2* px, int nx, float2* py, int ny, float2* pt, int nt, const double* phi,
                                    int sign) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx) px[i] = make_float2(0.f, 0.f);
  if (i < ny) py[i] = make_float2(0.f, 0.f);
  if (i < nt) {
    const double r = sign * phi[(i + nt / 2) % nt];
    const double two_pi = 6.283185307179586476925286766559;
    const double rr = r - two_pi * rint(r / two_pi);
    const float sh = sinf((float)(0.5 * rr));
    pt[i] = make_float2(-2.f * sh * sh, sinf((float)rr));
  }
}

cudaError_t run_phase_tables(float2* px, int nx, float2* py, int ny, float2* pt, int nt, const double* phi, int sign,
                             cudaStream_t s) {
  const int n = nx > ny ? (nx > nt ? nx : nt) : (ny > nt ? ny : nt);
  phase_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(px, nx, py, ny, pt, nt, phi, sign);
  return cudaPeekAtLastError();
}

}  // namespace brahms
