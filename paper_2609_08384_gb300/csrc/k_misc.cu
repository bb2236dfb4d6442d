// Set-up tables, the energy reduction and dtype conversions.
#include "kernels.cuh"
#include "map_seg.h"

namespace brahms {

// 2 pi * numpy.fft.fftfreq(n, d)[m]; the Nyquist bin is negative.
__device__ __forceinline__ double ang_freq(int m, int n, double d) {
  const int mm = (m < (n + 1) / 2) ? m : m - n;
  return 6.283185307179586476925286766559 * (double)mm / ((double)n * d);
}

// amp * exp(i phi) - 1 ("delta form").  The phase argument is formed and
// reduced to [-pi, pi] in FP64, then evaluated with FP32 sines:
//   amp cos(phi) - 1 = (amp - 1) - 2 amp sin^2(phi/2),   amp sin(phi).
// Stored this way, a factor with a small phase keeps |1 + D| = amp to FP32
// relative precision of the small part, so repeated application does not
// bias the field energy.
__device__ __forceinline__ float2 delta_phase(double phi, double amp_m1) {
  const double two_pi = 6.283185307179586476925286766559;
  const double r = phi - two_pi * rint(phi / two_pi);
  const float sh = sinf((float)(0.5 * r));
  const float s = sinf((float)r);
  const float am1 = (float)amp_m1;
  const float amp = (float)(1.0 + amp_m1);
  return make_float2(fmaf(-2.f * amp * sh, sh, am1), amp * s);
}

// Separable factors of the linear propagator over dz (Eqs. dispOp, diffOp,
// with d/dx -> i kx, d/dtau -> i Omega, diffraction +(i/2k) Laplacian and the
// unitary third-order term), each stored as D = P - 1:
//   Px = exp(-i dz [kx^2/(2k) + tan(rho) kx])
//   Py = exp(-i dz ky^2/(2k))
//   Pt = exp(dz [-alpha/2 - i delta Omega + i k2/2 Omega^2 - i k3/6 Omega^3])
__global__ void prop_tables_kernel(const TableArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = a.nx + a.ny + a.nt;
  if (i >= per * a.nf) return;
  const int f = i / per;
  int m = i % per;
  if (m < a.nx) {
    const double kx = ang_freq(m, a.nx, a.dx);
    const double ph = -a.dz * (kx * kx / (2.0 * a.k[f]) + tan(a.rho[f]) * kx);
    a.px[f * a.nx + m] = delta_phase(ph, 0.0);
    return;
  }
  m -= a.nx;
  if (m < a.ny) {
    const double ky = ang_freq(m, a.ny, a.dy);
    a.py[f * a.ny + m] = delta_phase(-a.dz * ky * ky / (2.0 * a.k[f]), 0.0);
    return;
  }
  m -= a.ny;
  const double om = ang_freq(m, a.nt, a.dt);
  const double ph = a.dz * (-a.delta[f] * om + 0.5 * a.k2[f] * om * om - a.k3[f] / 6.0 * om * om * om);
  a.pt[f * a.nt + m] = delta_phase(ph, expm1(-0.5 * a.alpha[f] * a.dz));
}

// ---------------------------------------------- mismatch-map tables
__device__ __forceinline__ float2 phase_plus(double phi) {
  const float2 em = phase_minus(phi);
  return make_float2(em.x, -em.y);
}

__global__ void map_tables_kernel(const MapArgs a) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.nxy;
       i += (long long)gridDim.x * blockDim.x) {
    const double mb = a.mapB[i], ma = a.mapA[i];
    const double p = a.mphase[i];
    a.emap[i] = phase_plus(a.phiB + a.dkB * 0.5 * a.dz + p + mb * (a.zB - a.zp + 0.5 * a.dz));
    a.emap[a.nxy + i] = phase_plus((a.dkB + mb) * 0.25 * a.dz);
    double pa = p, zpa = a.zp;
    if (a.advance) {
      pa = p + mb * (a.zA - a.zp);
      zpa = a.zA;
      a.mphase[i] = pa;
    }
    a.emap[2 * a.nxy + i] = phase_plus(a.phiA + pa + ma * (a.zA - zpa));
    a.emap[3 * a.nxy + i] = phase_plus((a.dkA + ma) * 0.25 * a.dz);
  }
}

cudaError_t run_map_tables(const MapArgs& a, cudaStream_t s) {
  long long g = (a.nxy + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  map_tables_kernel<<<(unsigned)g, 256, 0, s>>>(a);
  return cudaPeekAtLastError();
}

__global__ void map_phase_advance_kernel(double* mphase, const double* m, double len, long long nxy) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nxy; i += (long long)gridDim.x * blockDim.x)
    mphase[i] += m[i] * len;
}

cudaError_t run_map_phase_advance(double* mphase, const double* m, double len, long long nxy, cudaStream_t s) {
  long long g = (nxy + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  map_phase_advance_kernel<<<(unsigned)g, 256, 0, s>>>(mphase, m, len, nxy);
  return cudaPeekAtLastError();
}

// B: the second half of step jB (starting at its midpoint), A: the first half
// of step jA; the same four tables as map_tables_kernel.
__global__ void map_tables_seg_kernel(const MapSegArgs a) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.nxy;
       i += (long long)gridDim.x * blockDim.x) {
    double qb = 0.0, qa = 0.0;
    for (int s = 0; s < a.nseg; ++s) {
      const double m = a.maps[s * a.nxy + i];
      qb += a.cB[s] * m;
      qa += a.cA[s] * m;
    }
    const double mb = a.maps[a.sB * a.nxy + i], ma = a.maps[a.sA * a.nxy + i];
    a.emap[i] = phase_plus(a.phiB + a.dkB * 0.5 * a.dz + qb + mb * (0.5 * a.dz));
    a.emap[a.nxy + i] = phase_plus((a.dkB + mb) * 0.25 * a.dz);
    a.emap[2 * a.nxy + i] = phase_plus(a.phiA + qa);
    a.emap[3 * a.nxy + i] = phase_plus((a.dkA + ma) * 0.25 * a.dz);
  }
}

cudaError_t run_map_tables_seg(const MapSegArgs& a, cudaStream_t s) {
  if (a.nseg < 1 || a.nseg > kMapSegMax) return cudaErrorInvalidValue;
  long long g = (a.nxy + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  map_tables_seg_kernel<<<(unsigned)g, 256, 0, s>>>(a);
  return cudaPeekAtLastError();
}

cudaError_t run_prop_tables(const TableArgs& a, cudaStream_t s) {
  const int n = (a.nx + a.ny + a.nt) * a.nf;
  prop_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(a);
  return cudaPeekAtLastError();
}

// ------------------------------------------------------------- energy
// Per-field sum of |A|^2: two complex values per 16-byte load, squares
// summed in FP32 over eight points (round-to-nearest, unbiased) and added to
// an FP64 accumulator, so the FP64 work is one add per eight points.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) energy_partial_kernel(const float2* __restrict__ data, long long n,
                                                             long long fstride, double* partial) {
  const float2* a = data + blockIdx.y * fstride;
  double s = 0.0;
  // pairs (every length is even, so a field starts on a 16-byte boundary)
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const long long n2 = n / 2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // four independent pairs per round: the loads overlap, one FP64 add per eight points
  for (; i + 3 * stride < n2; i += 4 * stride) {
    const float4 v0 = __ldcg(a4 + i), v1 = __ldcg(a4 + i + stride), v2 = __ldcg(a4 + i + 2 * stride),
                 v3 = __ldcg(a4 + i + 3 * stride);
    const float q0 = fmaf(v0.x, v0.x, fmaf(v0.y, v0.y, fmaf(v0.z, v0.z, v0.w * v0.w)));
    const float q1 = fmaf(v1.x, v1.x, fmaf(v1.y, v1.y, fmaf(v1.z, v1.z, v1.w * v1.w)));
    const float q2 = fmaf(v2.x, v2.x, fmaf(v2.y, v2.y, fmaf(v2.z, v2.z, v2.w * v2.w)));
    const float q3 = fmaf(v3.x, v3.x, fmaf(v3.y, v3.y, fmaf(v3.z, v3.z, v3.w * v3.w)));
    s += (double)((q0 + q1) + (q2 + q3));
  }
  for (; i < n2; i += stride) {
    const float4 v = __ldcg(a4 + i);
    s += (double)fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w)));
  }
  if (n & 1) {  // odd length (not produced by the supported grids): the last point
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const float2 v = a[n - 1];
      s += (double)fmaf(v.x, v.x, v.y * v.y);
    }
  }
  __shared__ double red[8];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(256) energy_final_kernel(const double* partial, int nblocks, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partial[blockIdx.x * nblocks + i];
  __shared__ double red[8];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

cudaError_t run_energy(const float2* data, long long n, int nf, long long fstride, double* partial,
                       int nblocks, double* out, cudaStream_t s) {
  energy_partial_kernel<<<dim3(nblocks, nf), 256, 0, s>>>(data, n, fstride, partial);
  energy_final_kernel<<<nf, 256, 0, s>>>(partial, nblocks, out);
  return cudaPeekAtLastError();
}

// ---------------------------------------------------------- conversions
__global__ void c128_to_c64_kernel(const double2* __restrict__ in, float2* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void c64_to_c128_kernel(const float2* __restrict__ in, double2* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    out[i] = make_double2((double)v.x, (double)v.y);
  }
}

static int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g > 152 * 16 ? 152 * 16 : (g < 1 ? 1 : g));
}

// ------------------------------------------------ pointwise linear step
// The linear step of a grid without a tau extent (nt = 1, a cw field, or
// any grid whose tau-transform is the identity): the multiply
// P = (1 + Dx)(1 + Dy)(1 + Dt) / N of the tau-pass, element by element, with
// the tau-pass's arithmetic, on the (kx, ky)-domain state.
__global__ void prop_pointwise_kernel(const AxisArgs p, int nf) {
  const long long plane = (long long)p.nx * p.ny;
  const long long per_field = plane * p.nt;
  const long long n = per_field * nf;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i / per_field);
    const long long r = i - (long long)f * per_field;
    const int x = (int)(r % p.nx);
    const int y = (int)((r / p.nx) % p.ny);
    const int t = (int)(r / plane);
    const float2 dx = p.px[f * p.nx + x], dy = p.py[f * p.ny + y];
    float2 dxy = cadd(cadd(dx, dy), cmul(dx, dy));
    float2 dt = p.pt[f * p.nt + t];
    if (p.conj_p) {
      dxy.y = -dxy.y;
      dt.y = -dt.y;
    }
    float2* q = p.data + (long long)f * p.fstride + r;
    float2 w = *q;
    w = make_float2(fmaf(w.x, p.scale, w.x * p.scale_lo), fmaf(w.y, p.scale, w.y * p.scale_lo));
    *q = mul_one_plus(w, cadd(cadd(dxy, dt), cmul(dxy, dt)));
  }
}

cudaError_t run_prop_pointwise(const AxisArgs& a, int nf, cudaStream_t s) {
  prop_pointwise_kernel<<<grid_for((long long)a.nx * a.ny * a.nt * nf), 256, 0, s>>>(a, nf);
  return cudaPeekAtLastError();
}

cudaError_t run_c128_to_c64(const double2* in, float2* out, long long n, cudaStream_t s) {
  c128_to_c64_kernel<<<grid_for(n), 256, 0, s>>>(in, out, n);
  return cudaPeekAtLastError();
}
cudaError_t run_c64_to_c128(const float2* in, double2* out, long long n, cudaStream_t s) {
  c64_to_c128_kernel<<<grid_for(n), 256, 0, s>>>(in, out, n);
  return cudaPeekAtLastError();
}

}  // namespace brahms
