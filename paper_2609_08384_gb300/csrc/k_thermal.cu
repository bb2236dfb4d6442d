// Thermal model (Sec. 4.1: steady-state heat equation on the fields' grid and the
// temperature dependence of the phase mismatch).
//
// heat_load_kernel   Q(x, y) += sum_f c_f sum_tau |A_f|^2: one pass over the
//                    state, 64 x-points by 8 tau-lanes per CTA, FP32 squares of
//                    eight tau samples summed pairwise, then into FP64; lanes
//                    reduced in a fixed order (deterministic).
// sine_lines_kernel  the transverse Poisson solve's transforms.  With T = 0
//                    half a cell outside the window, sin(pi k (j + 1/2) / n),
//                    k = 1..n, are the eigenvectors of the 3-point second
//                    difference, with eigenvalues -4 sin^2(pi k / (2n)) / d^2;
//                    analysis along x and y, a division by the eigenvalues
//                    and synthesis solve the 5-point system exactly.  A line's
//                    analysis is a real-input sine transform computed through
//                    one complex FFT of n/2 points (Makhoul's packing of a
//                    real sequence for the cosine transform, IEEE Trans. ASSP
//                    28 (1980), with the sine transform read off the cosine
//                    transform of the sign-alternated line), and its
//                    synthesis undoes those steps one by one.  The FFT is an
//                    in-place Stockham FFT in FP64 shared memory, radix 2 and
//                    3, with one barrier between the reads and the writes of
//                    every stage.
#include "kernels.cuh"
#include "launch_cfg.h"

namespace brahms {

namespace {

constexpr int kHeatX = 64;    // x-points per CTA (32 pairs)
constexpr int kHeatLanes = 8;  // tau-lanes per CTA
constexpr int kHeatU = 8;      // tau samples per thread and iteration
constexpr int kSineThreads = 256;
constexpr int kSineMaxB2 = 8;  // radix-2 butterflies per thread: m / 2 <= 8 * 256, m <= 4096
constexpr int kSineMaxB3 = 2;  // radix-3 butterflies per thread: m / 3 <= 2 * 256
constexpr int kSineMaxStages = 16;

struct SineArgs {
  double* d;
  const double2* tw;  // 2n entries: e^{-i pi j / n} (j < n), then e^{-i pi k / (2n)} (k < n)
  long long elem;     // stride between the entries of a line
  long long pitch;    // stride between lines
  int n;              // line length (even); the FFT has m = n / 2 points
  int nst;
  int rad[kSineMaxStages];
};

__device__ __forceinline__ double2 z_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// e^{-+2 pi i e / m}, 0 <= e < m, m = n / 2, from the table of e^{-i pi j / n}
// (the entry 4 e for e < m / 2, and its negative above)
__device__ __forceinline__ double2 sine_tw(const double2* tw, int m, int e, bool inv) {
  const int h = m >> 1;
  double2 w = e < h ? tw[4 * e] : make_double2(-tw[4 * (e - h)].x, -tw[4 * (e - h)].y);
  if (inv) w.y = -w.y;
  return w;
}

// unnormalised DFT of buf[0..m) in place: sign -1 (forward) or +1 (inv)
__device__ void fft64_inplace(double2* buf, const SineArgs& a, int m, bool inv) {
  int ns = 1;
  for (int s = 0; s < a.nst; ++s) {
    const int R = a.rad[s];
    const int nb = m / R;
    const int step = m / (ns * R);
    if (R == 2) {
      double2 v[kSineMaxB2][2];
#pragma unroll
      for (int b = 0; b < kSineMaxB2; ++b) {
        const int j = threadIdx.x + b * kSineThreads;
        if (j < nb) {
          const int k = j % ns;
          v[b][0] = buf[j];
          v[b][1] = z_mul(buf[j + nb], sine_tw(a.tw, m, k * step, inv));
        }
      }
      __syncthreads();
#pragma unroll
      for (int b = 0; b < kSineMaxB2; ++b) {
        const int j = threadIdx.x + b * kSineThreads;
        if (j < nb) {
          const int k = j % ns;
          const int base = (j / ns) * ns * 2 + k;
          buf[base] = make_double2(v[b][0].x + v[b][1].x, v[b][0].y + v[b][1].y);
          buf[base + ns] = make_double2(v[b][0].x - v[b][1].x, v[b][0].y - v[b][1].y);
        }
      }
    } else {
      double2 v[kSineMaxB3][3];
#pragma unroll
      for (int b = 0; b < kSineMaxB3; ++b) {
        const int j = threadIdx.x + b * kSineThreads;
        if (j < nb) {
          const int k = j % ns;
          v[b][0] = buf[j];
          v[b][1] = z_mul(buf[j + nb], sine_tw(a.tw, m, k * step, inv));
          v[b][2] = z_mul(buf[j + 2 * nb], sine_tw(a.tw, m, 2 * k * step, inv));
        }
      }
      __syncthreads();
      // X1,2 = x0 - (x1 + x2) / 2 -+ i s (sqrt(3) / 2) (x1 - x2), s = +1 forward, -1 inverse
      const double h3 = inv ? -0.86602540378443864676 : 0.86602540378443864676;
#pragma unroll
      for (int b = 0; b < kSineMaxB3; ++b) {
        const int j = threadIdx.x + b * kSineThreads;
        if (j < nb) {
          const int k = j % ns;
          const int base = (j / ns) * ns * 3 + k;
          const double2 x0 = v[b][0], x1 = v[b][1], x2 = v[b][2];
          const double2 t1 = make_double2(x1.x + x2.x, x1.y + x2.y);
          const double2 t2 = make_double2(x0.x - 0.5 * t1.x, x0.y - 0.5 * t1.y);
          const double2 t3 = make_double2(h3 * (x1.x - x2.x), h3 * (x1.y - x2.y));
          buf[base] = make_double2(x0.x + t1.x, x0.y + t1.y);
          buf[base + ns] = make_double2(t2.x + t3.y, t2.y - t3.x);
          buf[base + 2 * ns] = make_double2(t2.x - t3.y, t2.y + t3.x);
        }
      }
    }
    __syncthreads();
    ns *= R;
  }
}

// SYNTH false: S_k = sum_j x_j sin(pi k (j + 1/2) / n), k = 1..n, stored at k - 1.
// SYNTH true:  x_j = sum_k (a_k / nu_k) sin(pi k (j + 1/2) / n), a_k read at k - 1,
//              nu_k = n / 2 (k < n) or n (k = n): the inverse of the analysis.
//
// Analysis.  With x'_j = (-1)^j x_j, S_k = C_{n-k} (k < n) and S_n = C_0, C the
// cosine transform C_k = sum_j x'_j cos(pi k (2j + 1) / (2n)).  Packing
// v_j = x'_{2j}, v_{n-1-j} = x'_{2j+1} (j < n/2) gives C_k = Re(w_k V_k), V the
// n-point DFT of v and w_k = e^{-i pi k / (2n)}; V of the real v comes from the
// n/2-point DFT Z of z_q = v_{2q} + i v_{2q+1}:
//   V_k = E_k + e^{-2 pi i k / n} O_k,  E_k = (Z_k + conj Z_{m-k}) / 2,
//   O_k = (Z_k - conj Z_{m-k}) / (2i),  k = 0..m (indices of Z mod m),
// and with V_{n-k} = conj V_k, C_{n-k} = -Im(w_k V_k).
// Synthesis runs the steps backwards: V_k = conj(w_k) (C_k - i C_{n-k}),
// Z_q = E_q + i O_q with E_q = (V_q + conj V_{m-q}) / 2 and
// O_q = e^{2 pi i q / n} (V_q - conj V_{m-q}) / 2, the inverse n/2-point DFT, and
// the unpacking.
template <bool SYNTH>
__global__ void __launch_bounds__(kSineThreads) sine_lines_kernel(const SineArgs a) {
  extern __shared__ double2 zbuf[];
  const int n = a.n, m = n / 2;
  const double2* th = a.tw + n;  // e^{-i pi k / (2n)}
  double* p = a.d + (long long)blockIdx.x * a.pitch;
  if (!SYNTH) {
    // z_q = v_{2q} + i v_{2q+1}, v_i = x'_{2i} (i < m) or x'_{2n-1-2i} (i >= m)
    for (int q = threadIdx.x; q < m; q += kSineThreads) {
      double c[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * q + h;
        const int jj = i < m ? 2 * i : 2 * n - 1 - 2 * i;
        const double x = p[(long long)jj * a.elem];
        c[h] = (jj & 1) ? -x : x;
      }
      zbuf[q] = make_double2(c[0], c[1]);
    }
  } else {
    // Z_q from the coefficients: C_k = a[n-1-k] (k >= 1), C_0 = a[n-1]
    for (int q = threadIdx.x; q < m; q += kSineThreads) {
      double2 v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = h == 0 ? q : m - q;
        const double ck = k == 0 ? p[(long long)(n - 1) * a.elem] : p[(long long)(n - 1 - k) * a.elem];
        const double cn = k == 0 ? 0.0 : p[(long long)(k - 1) * a.elem];
        const double2 w = th[k];  // V_k = conj(w_k) (C_k - i C_{n-k})
        v[h] = make_double2(w.x * ck - w.y * cn, -w.y * ck - w.x * cn);
      }
      const double2 vq = v[0], vc = make_double2(v[1].x, -v[1].y);  // V_q, conj V_{m-q}
      const double2 e = make_double2(0.5 * (vq.x + vc.x), 0.5 * (vq.y + vc.y));
      const double2 d = make_double2(0.5 * (vq.x - vc.x), 0.5 * (vq.y - vc.y));
      const double2 wq = a.tw[2 * q];  // e^{-2 pi i q / n}; O_q = conj(wq) d
      const double2 o = make_double2(wq.x * d.x + wq.y * d.y, wq.x * d.y - wq.y * d.x);
      zbuf[q] = make_double2(e.x - o.y, e.y + o.x);  // E + i O
    }
  }
  __syncthreads();
  fft64_inplace(zbuf, a, m, SYNTH);
  if (!SYNTH) {
    for (int k = threadIdx.x; k <= m; k += kSineThreads) {
      const double2 zk = zbuf[k % m], zr = zbuf[(m - k) % m];
      const double2 zc = make_double2(zr.x, -zr.y);
      const double2 e = make_double2(0.5 * (zk.x + zc.x), 0.5 * (zk.y + zc.y));
      const double2 o = make_double2(0.5 * (zk.y - zc.y), -0.5 * (zk.x - zc.x));  // (Z_k - conj Z_{m-k}) / (2i)
      const double2 wk = k < m ? a.tw[2 * k] : make_double2(-1.0, 0.0);        // e^{-2 pi i k / n}
      const double2 vk = make_double2(e.x + wk.x * o.x - wk.y * o.y, e.y + wk.x * o.y + wk.y * o.x);
      const double2 w = th[k];
      const double ur = w.x * vk.x - w.y * vk.y, ui = w.x * vk.y + w.y * vk.x;  // w_k V_k
      if (k < m) p[(long long)(k == 0 ? n - 1 : n - 1 - k) * a.elem] = ur;        // C_k
      if (k >= 1) p[(long long)(k - 1) * a.elem] = -ui;                           // C_{n-k}
    }
  } else {
    const double inv_m = 1.0 / (double)m;
    for (int j = threadIdx.x; j < n; j += kSineThreads) {
      // x_j = (-1)^j x'_j, x'_{2i} = v_i, x'_{2i+1} = v_{n-1-i}, v_i from z_{i/2}
      const int i = (j & 1) ? n - 1 - (j >> 1) : (j >> 1);
      const double2 zq = zbuf[i >> 1];
      const double v = ((i & 1) ? zq.y : zq.x) * inv_m;
      p[(long long)j * a.elem] = (j & 1) ? -v : v;
    }
  }
}

// tw[j] = e^{-i pi j / n} and tw[n + j] = e^{-i pi j / (2n)}, j < n
__global__ void sine_twiddles_kernel(double2* tw, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 2 * n) return;
  double sn, cs;
  if (j < n)
    sincospi(-(double)j / (double)n, &sn, &cs);
  else
    sincospi(-(double)(j - n) / (2.0 * n), &sn, &cs);
  tw[j] = make_double2(cs, sn);
}

// T-hat /= kappa mu_pq, mu_pq = 4 sin^2(pi (p+1) / (2 nx)) / dx^2 + (same in y)
__global__ void thermal_divide_kernel(double* d, int nx, int ny, double dx, double dy, double kappa) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nx * ny) return;
  const int p = (int)(i % nx), q = (int)(i / nx);
  const double sx = sinpi((double)(p + 1) / (2.0 * nx));
  double mu = 4.0 * sx * sx / (dx * dx);
  if (ny > 1) {
    const double sy = sinpi((double)(q + 1) / (2.0 * ny));
    mu += 4.0 * sy * sy / (dy * dy);
  }
  d[i] /= kappa * mu;
}

__global__ void thermal_map_kernel(const double* __restrict__ t, long long n, double dkdT, double* dkmap, int* bad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = t[i];
  if (!isfinite(v)) atomicOr(bad, 1);
  dkmap[i] = dkdT * v;
}

__global__ void __launch_bounds__(kHeatX / 2 * kHeatLanes) heat_load_kernel(const HeatArgs a) {
  __shared__ double red[kHeatLanes][kHeatX];
  const int xp = blockIdx.x * (kHeatX / 2) + threadIdx.x;  // x pair
  const int x = 2 * xp;
  const int y = blockIdx.y;
  const long long plane = (long long)a.nx * a.ny;
  const long long ps = plane / 2;  // plane stride in float4 (nx even)
  double s0 = 0.0, s1 = 0.0;
  if (x < a.nx) {
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      if (f >= a.nf) break;
      const float4* p = reinterpret_cast<const float4*>(a.data + f * a.fstride + (long long)y * a.nx + x);
      double f0 = 0.0, f1 = 0.0;
      int t = threadIdx.y;
      // kHeatU tau samples in flight per thread; their squares summed pairwise in FP32
      for (; t + (kHeatU - 1) * kHeatLanes < a.nt; t += kHeatU * kHeatLanes) {
        float4 v[kHeatU];
#pragma unroll
        for (int u = 0; u < kHeatU; ++u) v[u] = __ldcs(p + (t + u * kHeatLanes) * ps);
        float q0[kHeatU], q1[kHeatU];
#pragma unroll
        for (int u = 0; u < kHeatU; ++u) {
          q0[u] = fmaf(v[u].x, v[u].x, v[u].y * v[u].y);
          q1[u] = fmaf(v[u].z, v[u].z, v[u].w * v[u].w);
        }
#pragma unroll
        for (int w = kHeatU / 2; w > 0; w >>= 1)
#pragma unroll
          for (int u = 0; u < w; ++u) {
            q0[u] += q0[u + w];
            q1[u] += q1[u + w];
          }
        f0 += (double)q0[0];
        f1 += (double)q1[0];
      }
      for (; t < a.nt; t += kHeatLanes) {
        const float4 v = __ldcs(p + t * ps);
        f0 += (double)fmaf(v.x, v.x, v.y * v.y);
        f1 += (double)fmaf(v.z, v.z, v.w * v.w);
      }
      s0 += a.c[f] * f0;
      s1 += a.c[f] * f1;
    }
  }
  red[threadIdx.y][2 * threadIdx.x] = s0;
  red[threadIdx.y][2 * threadIdx.x + 1] = s1;
  __syncthreads();
  if (threadIdx.y == 0 && x < a.nx) {
    double r0 = 0.0, r1 = 0.0;
#pragma unroll
    for (int l = 0; l < kHeatLanes; ++l) {
      r0 += red[l][2 * threadIdx.x];
      r1 += red[l][2 * threadIdx.x + 1];
    }
    double* h = a.heat + (long long)y * a.nx + x;
    h[0] += r0;
    h[1] += r1;
  }
}

bool sine_plan(int n, SineArgs& a) {
  if (n < 2 || n % 2) return false;
  int m = n / 2, st = 0;
  while (m % 2 == 0) {
    if (st == kSineMaxStages) return false;
    a.rad[st++] = 2;
    m /= 2;
  }
  while (m % 3 == 0) {
    if (st == kSineMaxStages) return false;
    a.rad[st++] = 3;
    m /= 3;
  }
  if (m != 1) return false;
  a.nst = st;
  a.n = n;
  const int mm = n / 2;
  for (int s = 0; s < st; ++s) {
    const int nb = mm / a.rad[s];
    const int cap = (a.rad[s] == 2 ? kSineMaxB2 : kSineMaxB3) * kSineThreads;
    if (nb > cap) return false;
  }
  return true;
}

template <bool SYNTH>
cudaError_t sine_lines(double* d, const double2* tw, int n, long long elem, long long pitch, int lines,
                       cudaStream_t s) {
  SineArgs a{};
  if (!sine_plan(n, a)) return cudaErrorInvalidValue;
  a.d = d;
  a.tw = tw;
  a.elem = elem;
  a.pitch = pitch;
  const size_t smem = sizeof(double2) * (size_t)(n / 2);
  static SmemMax limit;
  cudaError_t e = raise_smem_limit_to(sine_lines_kernel<SYNTH>, std::max<size_t>(smem, 48 * 1024), limit);
  if (e != cudaSuccess) return e;
  sine_lines_kernel<SYNTH><<<lines, kSineThreads, smem, s>>>(a);
  return cudaPeekAtLastError();
}

}  // namespace

bool sine_length_supported(int n) {
  if (n < 2) return false;
  SineArgs a{};
  return sine_plan(n, a) && sizeof(double2) * (size_t)(n / 2) <= 227 * 1024;
}

cudaError_t run_sine_twiddles(double2* tw, int n, cudaStream_t s) {
  sine_twiddles_kernel<<<(2 * n + 255) / 256, 256, 0, s>>>(tw, n);
  return cudaPeekAtLastError();
}

cudaError_t run_heat_load(const HeatArgs& a, cudaStream_t s) {
  if (a.nx % 2) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((a.nx + kHeatX - 1) / kHeatX), (unsigned)a.ny);
  heat_load_kernel<<<grid, dim3(kHeatX / 2, kHeatLanes), 0, s>>>(a);
  return cudaPeekAtLastError();
}

namespace {
__global__ void map_add_kernel(double* __restrict__ dkmap, const double* __restrict__ base, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dkmap[i] += base[i];
}
}  // namespace

// dkmap += base (the static map under the thermal one)
cudaError_t run_map_add(double* dkmap, const double* base, long long n, cudaStream_t s) {
  map_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dkmap, base, n);
  return cudaPeekAtLastError();
}

cudaError_t run_thermal_solve(const ThermalArgs& a, int* nlaunch, cudaStream_t s) {
  const long long n = (long long)a.nx * a.ny;
  int nl = 0;
  cudaError_t e = cudaMemcpyAsync(a.temp, a.heat, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = sine_lines<false>(a.temp, a.twx, a.nx, 1, a.nx, a.ny, s), ++nl;
  if (e == cudaSuccess && a.ny > 1) e = sine_lines<false>(a.temp, a.twy, a.ny, a.nx, 1, a.nx, s), ++nl;
  if (e == cudaSuccess) {
    thermal_divide_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.temp, a.nx, a.ny, a.dx, a.dy, a.kappa);
    e = cudaPeekAtLastError(), ++nl;
  }
  if (e == cudaSuccess && a.ny > 1) e = sine_lines<true>(a.temp, a.twy, a.ny, a.nx, 1, a.nx, s), ++nl;
  if (e == cudaSuccess) e = sine_lines<true>(a.temp, a.twx, a.nx, 1, a.nx, a.ny, s), ++nl;
  if (e == cudaSuccess) {
    thermal_map_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.temp, n, a.dkdT, a.dkmap, a.bad);
    e = cudaPeekAtLastError(), ++nl;
  }
  *nlaunch = nl;
  return e;
}

}  // namespace brahms
