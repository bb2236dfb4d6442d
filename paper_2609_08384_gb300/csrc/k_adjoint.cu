// Kernels of the discrete adjoint of the split step besides the reverse
// x-pass: field scaling, the spectral-phase gradient and the spectral-phase
// tables.
#include "vjp.cuh"

namespace brahms {

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
