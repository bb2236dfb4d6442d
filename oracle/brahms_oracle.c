/*
 * FP64 CPU oracle for the split-step Fourier solution of the coupled chi(2)
 * three-wave-mixing equations in (3+1)D (x, y, tau propagated along z).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * statement of what the CUDA path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * What it follows (paper sections and equations):
 *   - coupled equations, Sec. 2, Eqs. CEp/CEs/CEi, with kappa = 2 pi d_eff/(n lambda)
 *   - dispersion operator, Eq. dispOp; diffraction/walk-off operator, Eq. diffOp
 *   - symmetric split step N(dz/2) L(dz) N(dz/2), Sec. 3.1, Eq. expon and the
 *     field-evolution equation that follows it
 *   - fourth-order Runge-Kutta for the nonlinear part, Sec. 3.1
 *   - power / energy, Sec. 6, P = 1/2 c eps0 n  integral |A|^2 dx dy
 *
 * Readings where the paper is silent or inconsistent (each is also pinned by a
 * test against a closed form):
 *   R1  diffraction enters as +(i/2k)(d2/dx2 + d2/dy2), the sign that the
 *       paper's own focused Gaussian beam (Eq. gaussianbeam) solves.
 *   R2  third-order dispersion is the unitary -[... - (k'''/6) d3/dtau3].
 *   R3  the scalar Eqs. CEp/CEs/CEi are used, not the garbled matrix form.
 *   R4  two-field degenerate SHG: fields (SH, F), SH plays the pump and F both
 *       signal and idler, with a 1/2 degeneracy factor on the SH equation:
 *         dA_SH/dz = i (kappa_SH/2) A_F^2 e^{-i Phi},
 *         dA_F /dz = i kappa_F A_SH A_F^*  e^{+i Phi}.
 *   R5  the mismatch phase stays in the nonlinear terms, Phi(z) = int_0^z dk.
 *   R6  the first RK4 half step spans [z_j, z_j + dz/2], the second
 *       [z_j + dz/2, z_j + dz]; Phi is evaluated at each RK4 stage's z.
 *   R7  forward DFT is unnormalised with e^{-2 pi i m n / N}; the inverse
 *       carries 1/N; angular frequencies follow numpy's fftfreq (the Nyquist
 *       bin is negative), so d/dx -> +i kx and d/dtau -> +i Omega.
 *
 * Data layout: fields[f][tau][y][x], x fastest, complex128.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_C0 299792458.0
#define ORC_EPS0 8.8541878128e-12
#define ORC_HBAR 1.054571817e-34
#define ORC_TWO_PI 6.283185307179586476925286766559

typedef struct {
  double lambda; /* vacuum wavelength [m] */
  double n;      /* refractive index */
  double delta;  /* 1/v_s - 1/v_lambda [s/m] */
  double k2;     /* GVD [s^2/m] */
  double k3;     /* TOD [s^3/m] */
  double rho;    /* walk-off angle [rad] */
  double alpha;  /* loss [1/m] */
} orc_field;

typedef struct {
  int nx, ny, nt, nf;
  double dx, dy, dt;
  double d_eff;
  orc_field f[3];
} orc_problem;

/* ------------------------------------------------------------------------ */
/* Threads: a plain fork-join over an index range.                           */
/* ------------------------------------------------------------------------ */
static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

typedef void (*range_fn)(void* ctx, int64_t begin, int64_t end);
typedef struct {
  range_fn fn;
  void* ctx;
  int64_t begin, end;
} range_job;

static void* range_trampoline(void* p) {
  range_job* j = (range_job*)p;
  j->fn(j->ctx, j->begin, j->end);
  return NULL;
}

static void parallel_for(int64_t count, range_fn fn, void* ctx) {
  int nt = g_threads;
  if (nt <= 1 || count < 2) {
    fn(ctx, 0, count);
    return;
  }
  if (nt > count) nt = (int)count;
  pthread_t th[256];
  range_job jobs[256];
  if (nt > 256) nt = 256;
  for (int i = 0; i < nt; ++i) {
    jobs[i].fn = fn;
    jobs[i].ctx = ctx;
    jobs[i].begin = count * i / nt;
    jobs[i].end = count * (i + 1) / nt;
  }
  for (int i = 1; i < nt; ++i) pthread_create(&th[i], NULL, range_trampoline, &jobs[i]);
  range_trampoline(&jobs[0]);
  for (int i = 1; i < nt; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------------ */
/* DFT: the plain O(N^2) definition and a recursive mixed-radix FFT.          */
/* ------------------------------------------------------------------------ */

/* out[m] = sum_n in[n] exp(sign * 2 pi i m n / N), no normalisation. */
void orc_dft_naive(const cplx* in, cplx* out, int n, int sign) {
  for (int m = 0; m < n; ++m) {
    cplx s = 0;
    for (int k = 0; k < n; ++k) {
      long long e = ((long long)m * k) % n;
      double ang = sign * ORC_TWO_PI * (double)e / (double)n;
      s += in[k] * (cos(ang) + I * sin(ang));
    }
    out[m] = s;
  }
}

static int smallest_factor(int n) {
  if (n % 2 == 0) return 2;
  for (int p = 3; p * p <= n; p += 2)
    if (n % p == 0) return p;
  return n;
}

/* Decimation in time: y[0..n) = DFT_n of x[0], x[stride], ..., x[(n-1) stride].
 * w[k] = exp(sign 2 pi i k / ntop) for the top-level length ntop; wstep = ntop/n.
 * For radix R = smallest factor of n, with m = n/R, the R sub-transforms of the
 * decimated sequences x[r + R q] land in y[r m .. r m + m), and are combined as
 *   Y[k + m s] = sum_r  W_n^{r (k + m s)}  Y_r[k].                           */
static void fft_rec(const cplx* x, long stride, cplx* y, int n, const cplx* w, int wstep,
                    int ntop) {
  if (n == 1) {
    y[0] = x[0];
    return;
  }
  int R = smallest_factor(n);
  int m = n / R;
  for (int r = 0; r < R; ++r) fft_rec(x + r * stride, stride * R, y + r * m, m, w, wstep * R, ntop);
  cplx t[64];
  cplx* tt = t;
  cplx* heap = NULL;
  if (R > 64) {
    heap = (cplx*)malloc(sizeof(cplx) * R);
    tt = heap;
  }
  for (int k = 0; k < m; ++k) {
    for (int r = 0; r < R; ++r) tt[r] = y[r * m + k];
    for (int s = 0; s < R; ++s) {
      cplx acc = 0;
      for (int r = 0; r < R; ++r) {
        long long e = ((long long)r * (k + (long long)m * s)) % n; /* exponent of W_n */
        acc += tt[r] * w[(e * wstep) % ntop];
      }
      y[k + m * s] = acc;
    }
  }
  free(heap);
}

static cplx* twiddle_table(int n, int sign) {
  cplx* w = (cplx*)malloc(sizeof(cplx) * n);
  for (int k = 0; k < n; ++k) {
    double ang = sign * ORC_TWO_PI * (double)k / (double)n;
    w[k] = cos(ang) + I * sin(ang);
  }
  return w;
}

/* In place, unnormalised: x <- sum_n x[n] exp(sign 2 pi i m n / N). */
void orc_fft1d(cplx* x, int n, int sign) {
  cplx* w = twiddle_table(n, sign);
  cplx* tmp = (cplx*)malloc(sizeof(cplx) * n);
  memcpy(tmp, x, sizeof(cplx) * n);
  fft_rec(tmp, 1, x, n, w, 1, n);
  free(tmp);
  free(w);
}

/* One axis of a 3D transform: pencils of length n at element stride `stride`. */
typedef struct {
  cplx* a;
  int n;
  long stride;
  int inner;  /* number of consecutive pencils sharing an outer index */
  long outer_stride;
  const cplx* w;
} axis_job;

static void axis_range(void* p, int64_t b, int64_t e) {
  axis_job* j = (axis_job*)p;
  cplx* buf = (cplx*)malloc(sizeof(cplx) * j->n * 2);
  cplx* out = buf + j->n;
  for (int64_t pi = b; pi < e; ++pi) {
    long o = (long)(pi / j->inner), i = (long)(pi % j->inner);
    cplx* base = j->a + o * j->outer_stride + i;
    for (int k = 0; k < j->n; ++k) buf[k] = base[k * j->stride];
    fft_rec(buf, 1, out, j->n, j->w, 1, j->n);
    for (int k = 0; k < j->n; ++k) base[k * j->stride] = out[k];
  }
  free(buf);
}

/* In-place unnormalised 3D DFT of one [nt][ny][nx] array. */
void orc_fft3(cplx* a, int nx, int ny, int nt, int sign) {
  axis_job j;
  j.a = a;
  /* x: pencils contiguous */
  cplx* wx = twiddle_table(nx, sign);
  j.n = nx; j.stride = 1; j.inner = 1; j.outer_stride = nx; j.w = wx;
  parallel_for((int64_t)ny * nt, axis_range, &j);
  free(wx);
  /* y: stride nx, nx pencils per tau plane */
  cplx* wy = twiddle_table(ny, sign);
  j.n = ny; j.stride = nx; j.inner = nx; j.outer_stride = (long)nx * ny; j.w = wy;
  parallel_for((int64_t)nx * nt, axis_range, &j);
  free(wy);
  /* tau: stride nx*ny, all nx*ny pencils */
  cplx* wt = twiddle_table(nt, sign);
  j.n = nt; j.stride = (long)nx * ny; j.inner = nx * ny; j.outer_stride = 0; j.w = wt;
  parallel_for((int64_t)nx * ny, axis_range, &j);
  free(wt);
}

/* ------------------------------------------------------------------------ */
/* Linear step: A_hat <- exp(dz * Lhat(kx, ky, Omega)) A_hat                   */
/* ------------------------------------------------------------------------ */

/* 2 pi * numpy.fft.fftfreq(n, d)[m]; bins m >= ceil(n/2) are negative (R7). */
double orc_angular_freq(int m, int n, double d) {
  int mm = (m < (n + 1) / 2) ? m : m - n;
  return ORC_TWO_PI * (double)mm / ((double)n * d);
}

/* Exponent of the linear operator of field f at (kx, ky, Omega):
 *  Eq. dispOp with d/dtau -> i Omega and the unitary TOD reading (R2):
 *     -alpha/2 - i delta Omega + i (k2/2) Omega^2 - i (k3/6) Omega^3
 *  Eq. diffOp with the sign of R1 and d/dx -> i kx:
 *     - i (kx^2 + ky^2) / (2 k) - i tan(rho) kx,  k = 2 pi n / lambda.       */
cplx orc_linear_exponent(const orc_field* fp, double kx, double ky, double om) {
  double k = ORC_TWO_PI * fp->n / fp->lambda;
  double re = -0.5 * fp->alpha;
  double im = -fp->delta * om + 0.5 * fp->k2 * om * om - fp->k3 / 6.0 * om * om * om
              - (kx * kx + ky * ky) / (2.0 * k) - tan(fp->rho) * kx;
  return re + I * im;
}

typedef struct {
  const orc_problem* pb;
  cplx* a;  /* one field */
  const orc_field* fp;
  double dz;
} mul_job;

static void mul_range(void* p, int64_t b, int64_t e) {
  mul_job* j = (mul_job*)p;
  const orc_problem* pb = j->pb;
  for (int64_t idx = b; idx < e; ++idx) {
    int x = (int)(idx % pb->nx);
    int y = (int)((idx / pb->nx) % pb->ny);
    int t = (int)(idx / ((int64_t)pb->nx * pb->ny));
    double kx = orc_angular_freq(x, pb->nx, pb->dx);
    double ky = orc_angular_freq(y, pb->ny, pb->dy);
    double om = orc_angular_freq(t, pb->nt, pb->dt);
    j->a[idx] *= cexp(j->dz * orc_linear_exponent(j->fp, kx, ky, om));
  }
}

typedef struct {
  cplx* a;
  double s;
} scale_job;
static void scale_range(void* p, int64_t b, int64_t e) {
  scale_job* j = (scale_job*)p;
  for (int64_t i = b; i < e; ++i) j->a[i] *= j->s;
}

/* A <- IDFT3( P * DFT3(A) ) for every field (the e^{L dz} factor of Eq. expon). */
void orc_linear_step(const orc_problem* pb, cplx* fields, double dz) {
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt;
  for (int f = 0; f < pb->nf; ++f) {
    cplx* a = fields + f * n;
    orc_fft3(a, pb->nx, pb->ny, pb->nt, -1);
    mul_job mj = {pb, a, &pb->f[f], dz};
    parallel_for(n, mul_range, &mj);
    orc_fft3(a, pb->nx, pb->ny, pb->nt, +1);
    scale_job sj = {a, 1.0 / (double)n};
    parallel_for(n, scale_range, &sj);
  }
}

/* ------------------------------------------------------------------------ */
/* Nonlinear part: right-hand sides of Eqs. CEp/CEs/CEi without L, and RK4.   */
/* ------------------------------------------------------------------------ */

double orc_kappa(const orc_problem* pb, int f) {
  return ORC_TWO_PI * pb->d_eff / (pb->f[f].n * pb->f[f].lambda);
}

/* dA/dz of the coupling terms at one grid point; phi = Phi(z) (R5). */
static void nl_rhs(int nf, const double* kap, double phi, const cplx* A, cplx* dA) {
  cplx em = cexp(-I * phi); /* e^{-i Phi} */
  cplx ep = cexp(I * phi);  /* e^{+i Phi} */
  if (nf == 3) {
    dA[0] = I * kap[0] * A[1] * A[2] * em;
    dA[1] = I * kap[1] * A[0] * conj(A[2]) * ep;
    dA[2] = I * kap[2] * A[0] * conj(A[1]) * ep;
  } else { /* (SH, F), R4 */
    dA[0] = I * (0.5 * kap[0]) * A[1] * A[1] * em;
    dA[1] = I * kap[1] * A[0] * conj(A[1]) * ep;
  }
}

/* Classical RK4 from z_a over h for one point: Phi(z_a + s) = phi_a + dk s. */
void orc_rk4_point(int nf, const double* kap, double phi_a, double dk, double h, cplx* A) {
  cplx k1[3], k2[3], k3[3], k4[3], tmp[3];
  nl_rhs(nf, kap, phi_a, A, k1);
  for (int f = 0; f < nf; ++f) tmp[f] = A[f] + 0.5 * h * k1[f];
  nl_rhs(nf, kap, phi_a + dk * 0.5 * h, tmp, k2);
  for (int f = 0; f < nf; ++f) tmp[f] = A[f] + 0.5 * h * k2[f];
  nl_rhs(nf, kap, phi_a + dk * 0.5 * h, tmp, k3);
  for (int f = 0; f < nf; ++f) tmp[f] = A[f] + h * k3[f];
  nl_rhs(nf, kap, phi_a + dk * h, tmp, k4);
  for (int f = 0; f < nf; ++f) A[f] += h / 6.0 * (k1[f] + 2.0 * k2[f] + 2.0 * k3[f] + k4[f]);
}

typedef struct {
  const orc_problem* pb;
  cplx* fields;
  double kap[3];
  double phi_a, dk, h;
} nl_job;

static void nl_range(void* p, int64_t b, int64_t e) {
  nl_job* j = (nl_job*)p;
  int64_t n = (int64_t)j->pb->nx * j->pb->ny * j->pb->nt;
  int nf = j->pb->nf;
  for (int64_t i = b; i < e; ++i) {
    cplx A[3];
    for (int f = 0; f < nf; ++f) A[f] = j->fields[f * n + i];
    orc_rk4_point(nf, j->kap, j->phi_a, j->dk, j->h, A);
    for (int f = 0; f < nf; ++f) j->fields[f * n + i] = A[f];
  }
}

/* N(h): RK4 over [z_a, z_a + h] at every grid point. */
void orc_nonlinear_step(const orc_problem* pb, cplx* fields, double phi_a, double dk, double h) {
  nl_job j;
  j.pb = pb;
  j.fields = fields;
  for (int f = 0; f < pb->nf; ++f) j.kap[f] = orc_kappa(pb, f);
  j.phi_a = phi_a;
  j.dk = dk;
  j.h = h;
  parallel_for((int64_t)pb->nx * pb->ny * pb->nt, nl_range, &j);
}

/* N(h) with a transverse mismatch map (f2 of the build's scope):
 * Delta k(x, y, z) = dk + dk_map[y nx + x] on this step, so at every point
 *   Phi(x, y, z_a + s) = phi_a + dk_map(x, y) z_a + (dk + dk_map(x, y)) s,
 * z_a measured from the start of the crystal; each point then takes the
 * RK4 of orc_rk4_point with its own phase origin and slope.                 */
typedef struct {
  const orc_problem* pb;
  cplx* fields;
  double kap[3];
  double phi_a, dk, h, z_a;
  const double* dk_map;
} nlm_job;

static void nlm_range(void* p, int64_t b, int64_t e) {
  nlm_job* j = (nlm_job*)p;
  const int64_t plane = (int64_t)j->pb->nx * j->pb->ny;
  const int64_t n = plane * j->pb->nt;
  const int nf = j->pb->nf;
  for (int64_t i = b; i < e; ++i) {
    const double m = j->dk_map[i % plane];
    cplx A[3];
    for (int f = 0; f < nf; ++f) A[f] = j->fields[f * n + i];
    orc_rk4_point(nf, j->kap, j->phi_a + m * j->z_a, j->dk + m, j->h, A);
    for (int f = 0; f < nf; ++f) j->fields[f * n + i] = A[f];
  }
}

void orc_nonlinear_step_map(const orc_problem* pb, cplx* fields, double phi_a, double dk, double h, double z_a,
                            const double* dk_map) {
  nlm_job j;
  j.pb = pb;
  j.fields = fields;
  for (int f = 0; f < pb->nf; ++f) j.kap[f] = orc_kappa(pb, f);
  j.phi_a = phi_a;
  j.dk = dk;
  j.h = h;
  j.z_a = z_a;
  j.dk_map = dk_map;
  parallel_for((int64_t)pb->nx * pb->ny * pb->nt, nlm_range, &j);
}

/* N(h) with a per-point phase origin: at every point
 *   Phi(x, y, z_a + s) = phi_a + q(x, y) + (dk + dk_map(x, y)) s,
 * q[y nx + x] the integral of the map over the distance already travelled
 * (used when the map changes along z; orc_nonlinear_step_map is the case
 * q = dk_map z_a).                                                         */
typedef struct {
  const orc_problem* pb;
  cplx* fields;
  double kap[3];
  double phi_a, dk, h;
  const double* q;
  const double* dk_map;
} nlq_job;

static void nlq_range(void* p, int64_t b, int64_t e) {
  nlq_job* j = (nlq_job*)p;
  const int64_t plane = (int64_t)j->pb->nx * j->pb->ny;
  const int64_t n = plane * j->pb->nt;
  const int nf = j->pb->nf;
  for (int64_t i = b; i < e; ++i) {
    const int64_t xy = i % plane;
    cplx A[3];
    for (int f = 0; f < nf; ++f) A[f] = j->fields[f * n + i];
    orc_rk4_point(nf, j->kap, j->phi_a + j->q[xy], j->dk + j->dk_map[xy], j->h, A);
    for (int f = 0; f < nf; ++f) j->fields[f * n + i] = A[f];
  }
}

static void nonlinear_step_q(const orc_problem* pb, cplx* fields, double phi_a, double dk, double h, const double* q,
                             const double* dk_map) {
  nlq_job j;
  j.pb = pb;
  j.fields = fields;
  for (int f = 0; f < pb->nf; ++f) j.kap[f] = orc_kappa(pb, f);
  j.phi_a = phi_a;
  j.dk = dk;
  j.h = h;
  j.q = q;
  j.dk_map = dk_map;
  parallel_for((int64_t)pb->nx * pb->ny * pb->nt, nlq_range, &j);
}

/* ------------------------------------------------------------------------ */
/* Split-step propagation (Eq. expon):  N(dz/2)  L(dz)  N(dz/2)  per step.     */
/* ------------------------------------------------------------------------ */

/* dk_steps[j] is the mismatch on step j (nz entries).  *phi holds Phi at the
 * start and is advanced to Phi at the end.  Returns 0, or 5 if the fields
 * are not finite afterwards (the dz-too-large failure of Sec. 3.2).        */
int orc_propagate(const orc_problem* pb, cplx* fields, int nz, double dz, const double* dk_steps,
                  double* phi) {
  double ph = *phi;
  for (int j = 0; j < nz; ++j) {
    double dk = dk_steps[j];
    orc_nonlinear_step(pb, fields, ph, dk, 0.5 * dz);
    orc_linear_step(pb, fields, dz);
    orc_nonlinear_step(pb, fields, ph + dk * 0.5 * dz, dk, 0.5 * dz);
    ph += dk * dz;
  }
  *phi = ph;
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt * pb->nf;
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(creal(fields[i])) || !isfinite(cimag(fields[i]))) return 5;
  return 0;
}

/* As orc_propagate with the transverse mismatch map dk_map[ny][nx] added to
 * every step's dk; z0 is the distance from the start of the crystal.        */
int orc_propagate_map(const orc_problem* pb, cplx* fields, int nz, double dz, const double* dk_steps, double* phi,
                      double z0, const double* dk_map) {
  double ph = *phi;
  for (int j = 0; j < nz; ++j) {
    const double dk = dk_steps[j], zj = z0 + j * dz;
    orc_nonlinear_step_map(pb, fields, ph, dk, 0.5 * dz, zj, dk_map);
    orc_linear_step(pb, fields, dz);
    orc_nonlinear_step_map(pb, fields, ph + dk * 0.5 * dz, dk, 0.5 * dz, zj + 0.5 * dz, dk_map);
    ph += dk * dz;
  }
  *phi = ph;
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt * pb->nf;
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(creal(fields[i])) || !isfinite(cimag(fields[i]))) return 5;
  return 0;
}

/* Segment of step j: the one that holds the step's midpoint (j + 1/2) dz. */
static int segment_of_step(int j, double dz, int nseg, const double* z_edges) {
  const double zmid = (j + 0.5) * dz;
  int s = 0;
  while (s < nseg - 1 && z_edges[s] <= zmid) ++s;
  return s;
}

/* One split step under the map m with the per-point phase offset q at its
 * start; q is advanced by m dz (qh: scratch for the second half step). */
static void step_map_z(const orc_problem* pb, cplx* fields, double ph, double dk, double dz, double* q,
                       const double* m, double* qh) {
  const int64_t plane = (int64_t)pb->nx * pb->ny;
  nonlinear_step_q(pb, fields, ph, dk, 0.5 * dz, q, m);
  orc_linear_step(pb, fields, dz);
  for (int64_t i = 0; i < plane; ++i) qh[i] = q[i] + m[i] * (0.5 * dz);
  nonlinear_step_q(pb, fields, ph + dk * 0.5 * dz, dk, 0.5 * dz, qh, m);
  for (int64_t i = 0; i < plane; ++i) q[i] += m[i] * dz;
}

/* A mismatch map that changes along z (a z-resolved thermal load, say):
 * Delta k(x, y, z) = dk_steps[j] + maps[s][y nx + x] on step j, s the segment
 * that holds the step's midpoint z_j + dz/2, segments separated by the
 * nseg - 1 increasing distances z_edges (from the start of the crystal).
 * The coupling phase is the integral of the mismatch from z = 0,
 *   Phi(x, y, z) = phi(z) + Q(x, y, z),  Q = int_0^z maps[s(z')](x, y) dz',
 * so it stays continuous where the map changes.  Starts at z = 0 with the
 * scalar phase *phi (advanced to its value at the end).                     */
int orc_propagate_map_z(const orc_problem* pb, cplx* fields, int nz, double dz, const double* dk_steps, double* phi,
                        int nseg, const double* z_edges, const double* maps) {
  const int64_t plane = (int64_t)pb->nx * pb->ny;
  double* q = (double*)calloc((size_t)plane, sizeof(double));
  double* qh = (double*)malloc(sizeof(double) * (size_t)plane);
  if (!q || !qh) {
    free(q);
    free(qh);
    return 1;
  }
  double ph = *phi;
  for (int j = 0; j < nz; ++j) {
    const double* m = maps + (int64_t)segment_of_step(j, dz, nseg, z_edges) * plane;
    step_map_z(pb, fields, ph, dk_steps[j], dz, q, m, qh);
    ph += dk_steps[j] * dz;
  }
  free(q);
  free(qh);
  *phi = ph;
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt * pb->nf;
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(creal(fields[i])) || !isfinite(cimag(fields[i]))) return 5;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Energy (Sec. 6):  E = 1/2 c eps0 n sum |A|^2 dx dy dtau, photons = E/(hbar w) */
/* ------------------------------------------------------------------------ */
void orc_energy(const orc_problem* pb, const cplx* fields, double* energy, double* photons) {
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt;
  for (int f = 0; f < pb->nf; ++f) {
    /* Kahan-compensated sum of |A|^2 */
    double s = 0.0, c = 0.0;
    const cplx* a = fields + f * n;
    for (int64_t i = 0; i < n; ++i) {
      double v = creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
      double y = v - c;
      double t = s + y;
      c = (t - s) - y;
      s = t;
    }
    double e = 0.5 * ORC_C0 * ORC_EPS0 * pb->f[f].n * s * pb->dx * pb->dy * pb->dt;
    energy[f] = e;
    if (photons) {
      double omega = ORC_TWO_PI * ORC_C0 / pb->f[f].lambda;
      photons[f] = e / (ORC_HBAR * omega);
    }
  }
}

/* Temporal power trace (Sec. 6 power formula, integrated over the beam at
 * each tau): power[f*nt + k] = 1/2 c eps0 n_f dx dy sum_{x,y} |A_f(x,y,tau_k)|^2 [W].
 * sum_k power dt is the field energy of orc_energy.                          */
void orc_power_trace(const orc_problem* pb, const cplx* fields, double* power) {
  const int64_t plane = (int64_t)pb->nx * pb->ny, n = plane * pb->nt;
  for (int f = 0; f < pb->nf; ++f) {
    const double c = 0.5 * ORC_C0 * ORC_EPS0 * pb->f[f].n * pb->dx * pb->dy;
    for (int k = 0; k < pb->nt; ++k) {
      const cplx* a = fields + f * n + k * plane;
      double s = 0.0;
      for (int64_t i = 0; i < plane; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
      power[f * pb->nt + k] = c * s;
    }
  }
}

/* Energy spectrum over Omega, per bin of width 2 pi / (nt dt):
 *   spectrum[f*nt + m] = 1/2 c eps0 n_f dx dy (dt / nt) sum_{x,y} |DFT_tau A_f|^2 (m),
 * m in FFT order (Omega_m = orc_angular_freq(m, nt, dt)).  By Parseval the
 * bins sum to the field energy.                                              */
void orc_spectrum(const orc_problem* pb, const cplx* fields, double* spectrum) {
  const int64_t plane = (int64_t)pb->nx * pb->ny, n = plane * pb->nt;
  cplx* col = (cplx*)malloc(sizeof(cplx) * pb->nt);
  for (int f = 0; f < pb->nf; ++f) {
    const double c = 0.5 * ORC_C0 * ORC_EPS0 * pb->f[f].n * pb->dx * pb->dy * pb->dt / pb->nt;
    for (int m = 0; m < pb->nt; ++m) spectrum[f * pb->nt + m] = 0.0;
    for (int64_t i = 0; i < plane; ++i) {
      for (int k = 0; k < pb->nt; ++k) col[k] = fields[f * n + k * plane + i];
      orc_fft1d(col, pb->nt, -1);
      for (int m = 0; m < pb->nt; ++m)
        spectrum[f * pb->nt + m] += c * (creal(col[m]) * creal(col[m]) + cimag(col[m]) * cimag(col[m]));
    }
  }
  free(col);
}

/* Heat load of the thermal model (Sec. 4.1, the source term Q of the heat
 * equation): the absorbed optical power density
 *   Q(x, y) = sum_f alpha_f I_f,   I_f = 1/2 c eps0 n_f |A_f|^2,
 * alpha_f the intensity absorption coefficient (the linear step damps the
 * amplitude by exp(-alpha_f dz / 2)).  For nt > 1 the pulse train is
 * time-averaged: Q = rep_rate sum_f alpha_f sum_tau I_f dt.                 */
void orc_heat_load(const orc_problem* pb, const cplx* fields, double rep_rate, double* q) {
  const int64_t plane = (int64_t)pb->nx * pb->ny, n = plane * pb->nt;
  const double tavg = pb->nt > 1 ? rep_rate * pb->dt : 1.0;
  for (int64_t i = 0; i < plane; ++i) q[i] = 0.0;
  for (int f = 0; f < pb->nf; ++f) {
    const double c = pb->f[f].alpha * 0.5 * ORC_C0 * ORC_EPS0 * pb->f[f].n * tavg;
    for (int k = 0; k < pb->nt; ++k)
      for (int64_t i = 0; i < plane; ++i) {
        const cplx a = fields[f * n + k * plane + i];
        q[i] += c * (creal(a) * creal(a) + cimag(a) * cimag(a));
      }
  }
}

/* ======================================================================== */
/* Discrete adjoint (reverse mode) of the split-step propagation.            */
/*                                                                            */
/* Objective J = sum_f w_f sum_points |A_f(L)|^2 (real).  For complex        */
/* variables the gradient is G_z = dJ/dRe z + i dJ/dIm z = 2 dJ/d conj(z);    */
/* for y = f(x):  G_x = sum_y [ conj(G_y) dy/d conj(x) + G_y conj(dy/dx) ].   */
/* The linear step is complex-linear, so its adjoint is IDFT3(conj(P) DFT3).  */
/* The RK4 half step is differentiated stage by stage (reverse order).        */
/* The mismatch enters every RK4 stage through Phi(z) = Phi_j + dk_j (z-z_j); */
/* dJ/dPhi at a stage is Re sum conj(G_k) dk/dPhi with dk/dPhi = -/+ i k.     */
/* ======================================================================== */

/* Coupling coefficients c_f = i kap_f e^{-/+ i phi} (minus for field 0). */
static void nl_coef(int nf, const double* kap, double phi, cplx* c) {
  cplx em = cexp(-I * phi), ep = cexp(I * phi);
  if (nf == 3) {
    c[0] = I * kap[0] * em;
    c[1] = I * kap[1] * ep;
    c[2] = I * kap[2] * ep;
  } else {
    c[0] = I * (0.5 * kap[0]) * em;
    c[1] = I * kap[1] * ep;
  }
}

/* f(u) with coefficients c (the right-hand sides of nl_rhs). */
static void rhs_c(int nf, const cplx* c, const cplx* u, cplx* k) {
  if (nf == 3) {
    k[0] = c[0] * u[1] * u[2];
    k[1] = c[1] * u[0] * conj(u[2]);
    k[2] = c[2] * u[0] * conj(u[1]);
  } else {
    k[0] = c[0] * u[1] * u[1];
    k[1] = c[1] * u[0] * conj(u[1]);
  }
}

/* tangent: df = sum df/du du + df/dconj(u) conj(du) */
static void rhs_jvp(int nf, const cplx* c, const cplx* u, const cplx* du, cplx* dk) {
  if (nf == 3) {
    dk[0] = c[0] * (du[1] * u[2] + u[1] * du[2]);
    dk[1] = c[1] * (du[0] * conj(u[2]) + u[0] * conj(du[2]));
    dk[2] = c[2] * (du[0] * conj(u[1]) + u[0] * conj(du[1]));
  } else {
    dk[0] = c[0] * 2.0 * u[1] * du[1];
    dk[1] = c[1] * (du[0] * conj(u[1]) + u[0] * conj(du[1]));
  }
}

/* adjoint: gu += sum_y [ conj(g_y) dy/dconj(u) + g_y conj(dy/du) ] */
static void rhs_vjp(int nf, const cplx* c, const cplx* u, const cplx* g, cplx* gu) {
  if (nf == 3) {
    gu[0] += g[1] * conj(c[1]) * u[2] + g[2] * conj(c[2]) * u[1];
    gu[1] += g[0] * conj(c[0]) * conj(u[2]) + conj(g[2]) * c[2] * u[0];
    gu[2] += g[0] * conj(c[0]) * conj(u[1]) + conj(g[1]) * c[1] * u[0];
  } else {
    gu[0] += g[1] * conj(c[1]) * u[1];
    gu[1] += g[0] * conj(2.0 * c[0] * u[1]) + conj(g[1]) * c[1] * u[0];
  }
}

/* sum_f Re( conj(g_f) dk_f/dPhi ),  dk_0/dPhi = -i k_0, others +i k_f */
static double phase_sens(int nf, const cplx* g, const cplx* k) {
  double s = creal(conj(g[0]) * (-I * k[0]));
  for (int f = 1; f < nf; ++f) s += creal(conj(g[f]) * (I * k[f]));
  return s;
}

/* Tangent of one RK4 step from z_a over h (same stages as orc_rk4_point). */
void orc_rk4_jvp_point(int nf, const double* kap, double phi_a, double dk, double h, const cplx* x,
                       const cplx* dx, cplx* y, cplx* dy) {
  cplx c1[3], c2[3], c3[3], u[3], du[3], k[4][3], dkk[4][3];
  nl_coef(nf, kap, phi_a, c1);
  nl_coef(nf, kap, phi_a + dk * 0.5 * h, c2);
  nl_coef(nf, kap, phi_a + dk * h, c3);
  rhs_c(nf, c1, x, k[0]);
  rhs_jvp(nf, c1, x, dx, dkk[0]);
  for (int f = 0; f < nf; ++f) { u[f] = x[f] + 0.5 * h * k[0][f]; du[f] = dx[f] + 0.5 * h * dkk[0][f]; }
  rhs_c(nf, c2, u, k[1]);
  rhs_jvp(nf, c2, u, du, dkk[1]);
  for (int f = 0; f < nf; ++f) { u[f] = x[f] + 0.5 * h * k[1][f]; du[f] = dx[f] + 0.5 * h * dkk[1][f]; }
  rhs_c(nf, c2, u, k[2]);
  rhs_jvp(nf, c2, u, du, dkk[2]);
  for (int f = 0; f < nf; ++f) { u[f] = x[f] + h * k[2][f]; du[f] = dx[f] + h * dkk[2][f]; }
  rhs_c(nf, c3, u, k[3]);
  rhs_jvp(nf, c3, u, du, dkk[3]);
  for (int f = 0; f < nf; ++f) {
    y[f] = x[f] + h / 6.0 * (k[0][f] + 2.0 * k[1][f] + 2.0 * k[2][f] + k[3][f]);
    dy[f] = dx[f] + h / 6.0 * (dkk[0][f] + 2.0 * dkk[1][f] + 2.0 * dkk[2][f] + dkk[3][f]);
  }
}

/* Adjoint of one RK4 step at input x: gx = (dy/dx)^T gy; sens[0..2] +=
 * dJ/dPhi at the stage points z_a, z_a + h/2 (stages 2 and 3), z_a + h. */
void orc_rk4_vjp_point(int nf, const double* kap, double phi_a, double dk, double h, const cplx* x,
                       const cplx* gy, cplx* gx, double* sens) {
  cplx c1[3], c2[3], c3[3], u[4][3], k[4][3], gk[4][3], gu[3];
  nl_coef(nf, kap, phi_a, c1);
  nl_coef(nf, kap, phi_a + dk * 0.5 * h, c2);
  nl_coef(nf, kap, phi_a + dk * h, c3);
  for (int f = 0; f < nf; ++f) u[0][f] = x[f];
  rhs_c(nf, c1, u[0], k[0]);
  for (int f = 0; f < nf; ++f) u[1][f] = x[f] + 0.5 * h * k[0][f];
  rhs_c(nf, c2, u[1], k[1]);
  for (int f = 0; f < nf; ++f) u[2][f] = x[f] + 0.5 * h * k[1][f];
  rhs_c(nf, c2, u[2], k[2]);
  for (int f = 0; f < nf; ++f) u[3][f] = x[f] + h * k[2][f];
  rhs_c(nf, c3, u[3], k[3]);
  /* y = x + h/6 (k1 + 2 k2 + 2 k3 + k4) */
  for (int f = 0; f < nf; ++f) {
    gx[f] = gy[f];
    gk[0][f] = h / 6.0 * gy[f];
    gk[1][f] = h / 3.0 * gy[f];
    gk[2][f] = h / 3.0 * gy[f];
    gk[3][f] = h / 6.0 * gy[f];
  }
  /* stage 4: u4 = x + h k3 */
  for (int f = 0; f < nf; ++f) gu[f] = 0;
  rhs_vjp(nf, c3, u[3], gk[3], gu);
  sens[2] += phase_sens(nf, gk[3], k[3]);
  for (int f = 0; f < nf; ++f) { gx[f] += gu[f]; gk[2][f] += h * gu[f]; }
  /* stage 3: u3 = x + h/2 k2 */
  for (int f = 0; f < nf; ++f) gu[f] = 0;
  rhs_vjp(nf, c2, u[2], gk[2], gu);
  sens[1] += phase_sens(nf, gk[2], k[2]);
  for (int f = 0; f < nf; ++f) { gx[f] += gu[f]; gk[1][f] += 0.5 * h * gu[f]; }
  /* stage 2: u2 = x + h/2 k1 */
  for (int f = 0; f < nf; ++f) gu[f] = 0;
  rhs_vjp(nf, c2, u[1], gk[1], gu);
  sens[1] += phase_sens(nf, gk[1], k[1]);
  for (int f = 0; f < nf; ++f) { gx[f] += gu[f]; gk[0][f] += 0.5 * h * gu[f]; }
  /* stage 1: u1 = x */
  for (int f = 0; f < nf; ++f) gu[f] = 0;
  rhs_vjp(nf, c1, u[0], gk[0], gu);
  sens[0] += phase_sens(nf, gk[0], k[0]);
  for (int f = 0; f < nf; ++f) gx[f] += gu[f];
}

/* Adjoint of the linear step: A <- IDFT3( conj(P) DFT3(A) ). */
void orc_linear_step_adjoint(const orc_problem* pb, cplx* fields, double dz) {
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt;
  for (int f = 0; f < pb->nf; ++f) {
    cplx* a = fields + f * n;
    orc_fft3(a, pb->nx, pb->ny, pb->nt, -1);
    for (int64_t idx = 0; idx < n; ++idx) {
      int x = (int)(idx % pb->nx);
      int y = (int)((idx / pb->nx) % pb->ny);
      int t = (int)(idx / ((int64_t)pb->nx * pb->ny));
      double kx = orc_angular_freq(x, pb->nx, pb->dx);
      double ky = orc_angular_freq(y, pb->ny, pb->dy);
      double om = orc_angular_freq(t, pb->nt, pb->dt);
      a[idx] *= conj(cexp(dz * orc_linear_exponent(&pb->f[f], kx, ky, om)));
    }
    orc_fft3(a, pb->nx, pb->ny, pb->nt, +1);
    for (int64_t i = 0; i < n; ++i) a[i] /= (double)n;
  }
}

/* Spectral phase on one field: A <- IDFT_tau( e^{i phi(Omega)} DFT_tau A ),
 * phi given in centred order: phi[p] belongs to Omega = 2 pi (p - NT/2)/T. */
void orc_spectral_phase(const orc_problem* pb, cplx* a, const double* phi, int sign) {
  int nt = pb->nt;
  int64_t plane = (int64_t)pb->nx * pb->ny;
  cplx* buf = (cplx*)malloc(sizeof(cplx) * nt);
  for (int64_t q = 0; q < plane; ++q) {
    for (int t = 0; t < nt; ++t) buf[t] = a[t * plane + q];
    orc_fft1d(buf, nt, -1);
    for (int m = 0; m < nt; ++m) {
      int p = (m + nt / 2) % nt; /* centred index of bin m */
      buf[m] *= cexp(I * sign * phi[p]);
    }
    orc_fft1d(buf, nt, +1);
    for (int t = 0; t < nt; ++t) a[t * plane + q] = buf[t] / (double)nt;
  }
  free(buf);
}

typedef struct {
  const orc_problem* pb;
  const cplx* x; /* forward state at the start of the half step */
  cplx* g;       /* adjoint in/out */
  double kap[3];
  double phi_a, dk, h;
  double z_a;            /* distance of the half step's start from z = 0 (for the map) */
  const double* dk_map;  /* transverse mismatch map [ny][nx] or NULL */
  const double* q;       /* per-point phase offset at the start [ny][nx] (replaces dk_map z_a) or NULL */
  double* part;  /* [slot][3] partial stage sensitivities */
  int64_t chunk; /* points per slot (fixed, so the sums do not depend on threads) */
} vjp_job;

static void vjp_slots(void* p, int64_t s0, int64_t s1) {
  vjp_job* j = (vjp_job*)p;
  const int64_t plane = (int64_t)j->pb->nx * j->pb->ny;
  int64_t n = plane * j->pb->nt;
  int nf = j->pb->nf;
  for (int64_t s = s0; s < s1; ++s) {
    double acc[3] = {0, 0, 0};
    int64_t b = s * j->chunk, e = b + j->chunk;
    if (e > n) e = n;
    for (int64_t i = b; i < e; ++i) {
      cplx x[3], gy[3], gx[3];
      for (int f = 0; f < nf; ++f) {
        x[f] = j->x[f * n + i];
        gy[f] = j->g[f * n + i];
      }
      /* with a map the point's phase is Phi_a + m z_a (or Phi_a + q) at the start and grows at dk + m */
      const double m = j->dk_map ? j->dk_map[i % plane] : 0.0;
      const double start = j->q ? j->phi_a + j->q[i % plane] : j->phi_a + m * j->z_a;
      orc_rk4_vjp_point(nf, j->kap, start, j->dk + m, j->h, x, gy, gx, acc);
      for (int f = 0; f < nf; ++f) j->g[f * n + i] = gx[f];
    }
    for (int k = 0; k < 3; ++k) j->part[s * 3 + k] = acc[k];
  }
}

/* g <- adjoint of N(h) (RK4 from phi_a over h) at the forward input x;
 * sens[0..2] = dJ/dPhi at the three stage points (start, middle, end).
 * With a transverse map (dk_map non-NULL) the half step starts at distance
 * z_a and each point follows its own phase, as in orc_nonlinear_step_map. */
void orc_nonlinear_step_adjoint_map(const orc_problem* pb, const cplx* x, cplx* g, double phi_a, double dk, double h,
                                    double z_a, const double* dk_map, double* sens) {
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt;
  const int64_t chunk = 4096;
  int64_t slots = (n + chunk - 1) / chunk;
  double* part = (double*)calloc(3 * (size_t)slots, sizeof(double));
  vjp_job j;
  j.pb = pb;
  j.x = x;
  j.g = g;
  for (int f = 0; f < pb->nf; ++f) j.kap[f] = orc_kappa(pb, f);
  j.phi_a = phi_a;
  j.dk = dk;
  j.h = h;
  j.z_a = z_a;
  j.dk_map = dk_map;
  j.q = NULL;
  j.part = part;
  j.chunk = chunk;
  parallel_for(slots, vjp_slots, &j);
  sens[0] = sens[1] = sens[2] = 0.0;
  for (int64_t s = 0; s < slots; ++s)
    for (int k = 0; k < 3; ++k) sens[k] += part[s * 3 + k];
  free(part);
}

/* The same with a per-point phase offset: Phi(x, y, z_a + s) = phi_a + q(x, y)
 * + (dk + dk_map(x, y)) s (a map that changes along z). */
static void nonlinear_step_adjoint_q(const orc_problem* pb, const cplx* x, cplx* g, double phi_a, double dk,
                                     double h, const double* q, const double* dk_map, double* sens) {
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt;
  const int64_t chunk = 4096;
  int64_t slots = (n + chunk - 1) / chunk;
  double* part = (double*)calloc(3 * (size_t)slots, sizeof(double));
  vjp_job j;
  j.pb = pb;
  j.x = x;
  j.g = g;
  for (int f = 0; f < pb->nf; ++f) j.kap[f] = orc_kappa(pb, f);
  j.phi_a = phi_a;
  j.dk = dk;
  j.h = h;
  j.z_a = 0.0;
  j.dk_map = dk_map;
  j.q = q;
  j.part = part;
  j.chunk = chunk;
  parallel_for(slots, vjp_slots, &j);
  sens[0] = sens[1] = sens[2] = 0.0;
  for (int64_t s = 0; s < slots; ++s)
    for (int k = 0; k < 3; ++k) sens[k] += part[s * 3 + k];
  free(part);
}

void orc_nonlinear_step_adjoint(const orc_problem* pb, const cplx* x, cplx* g, double phi_a, double dk, double h,
                                double* sens) {
  orc_nonlinear_step_adjoint_map(pb, x, g, phi_a, dk, h, 0.0, NULL, sens);
}

/* Gradient of J = sum_f w[f] sum |A_f(L)|^2 with respect to the spectral phase
 * phi (applied to field phi_field at z = 0, centred order, nt entries; NULL
 * for none) and to the per-step mismatch dk_steps[0..nz-1], under the
 * transverse map dk_map (NULL for none; the map itself is not a parameter).
 * Forward states of every step are kept (the oracle is for small grids).
 * Returns J. */
/* Under a map that changes along z (maps non-NULL: nseg segments, as in
 * orc_propagate_map_z) each step j keeps its per-point phase offset q_j, the
 * integral of the maps up to z_j, and both half steps and their adjoints run
 * with the map of the step's segment. */
static double adjoint_impl(const orc_problem* pb, const cplx* fields_in, int nz, double dz, const double* dk_steps,
                           const double* phi, int phi_field, const double* w, double* grad_phi, double* grad_dk,
                           const double* dk_map, int nseg, const double* z_edges, const double* maps) {
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt;
  const int64_t plane = (int64_t)pb->nx * pb->ny;
  int nf = pb->nf;
  int64_t sz = n * nf;
  cplx* st = (cplx*)malloc(sizeof(cplx) * sz * (size_t)(nz + 1)); /* A_0 .. A_nz */
  memcpy(st, fields_in, sizeof(cplx) * sz);
  if (phi) orc_spectral_phase(pb, st + phi_field * n, phi, +1);
  double* phis = (double*)malloc(sizeof(double) * (nz + 1)); /* Phi(z_j) */
  double* qs = maps ? (double*)calloc((size_t)plane * (nz + 1), sizeof(double)) : NULL; /* q_j */
  double* qh = maps ? (double*)malloc(sizeof(double) * (size_t)plane) : NULL;
  phis[0] = 0.0;
  for (int j = 0; j < nz; ++j) {
    memcpy(st + (j + 1) * sz, st + j * sz, sizeof(cplx) * sz);
    double ph = phis[j];
    if (maps) {
      const double* m = maps + (int64_t)segment_of_step(j, dz, nseg, z_edges) * plane;
      memcpy(qs + (j + 1) * plane, qs + j * plane, sizeof(double) * plane);
      step_map_z(pb, st + (j + 1) * sz, ph, dk_steps[j], dz, qs + (j + 1) * plane, m, qh);
      ph += dk_steps[j] * dz;
    } else if (dk_map) {
      orc_propagate_map(pb, st + (j + 1) * sz, 1, dz, dk_steps + j, &ph, j * dz, dk_map);
    } else {
      orc_propagate(pb, st + (j + 1) * sz, 1, dz, dk_steps + j, &ph);
    }
    phis[j + 1] = ph;
  }
  /* objective and its gradient at z = L */
  const cplx* af = st + nz * sz;
  double J = 0.0;
  cplx* g = (cplx*)malloc(sizeof(cplx) * sz);
  for (int f = 0; f < nf; ++f)
    for (int64_t i = 0; i < n; ++i) {
      cplx a = af[f * n + i];
      J += w[f] * (creal(a) * creal(a) + cimag(a) * cimag(a));
      g[f * n + i] = 2.0 * w[f] * a;
    }
  /* reverse sweep */
  double* S = (double*)calloc((size_t)nz * 6, sizeof(double)); /* per step: A stages 0..2, B stages 0..2 */
  cplx* a2 = (cplx*)malloc(sizeof(cplx) * sz);
  for (int j = nz - 1; j >= 0; --j) {
    const cplx* aj = st + j * sz;
    double dk = dk_steps[j];
    const double zj = j * dz;
    /* a2 = L(N_A(A_j)) */
    memcpy(a2, aj, sizeof(cplx) * sz);
    if (maps) {
      const double* m = maps + (int64_t)segment_of_step(j, dz, nseg, z_edges) * plane;
      const double* q = qs + j * plane;
      nonlinear_step_q(pb, a2, phis[j], dk, 0.5 * dz, q, m);
      orc_linear_step(pb, a2, dz);
      for (int64_t i = 0; i < plane; ++i) qh[i] = q[i] + m[i] * (0.5 * dz);
      nonlinear_step_adjoint_q(pb, a2, g, phis[j] + dk * 0.5 * dz, dk, 0.5 * dz, qh, m, S + j * 6 + 3);
      orc_linear_step_adjoint(pb, g, dz);
      nonlinear_step_adjoint_q(pb, aj, g, phis[j], dk, 0.5 * dz, q, m, S + j * 6);
      continue;
    }
    if (dk_map)
      orc_nonlinear_step_map(pb, a2, phis[j], dk, 0.5 * dz, zj, dk_map);
    else
      orc_nonlinear_step(pb, a2, phis[j], dk, 0.5 * dz);
    orc_linear_step(pb, a2, dz);
    orc_nonlinear_step_adjoint_map(pb, a2, g, phis[j] + dk * 0.5 * dz, dk, 0.5 * dz, zj + 0.5 * dz, dk_map,
                                   S + j * 6 + 3);
    orc_linear_step_adjoint(pb, g, dz);
    orc_nonlinear_step_adjoint_map(pb, aj, g, phis[j], dk, 0.5 * dz, zj, dk_map, S + j * 6);
  }
  /* dJ/d dk_j: stage offsets within step j, plus dz for every later stage */
  if (grad_dk) {
    const double offA[3] = {0.0, 0.25 * dz, 0.5 * dz};
    const double offB[3] = {0.5 * dz, 0.75 * dz, dz};
    double later = 0.0;
    for (int j = nz - 1; j >= 0; --j) {
      double v = dz * later;
      double tot = 0.0;
      for (int s = 0; s < 3; ++s) {
        v += S[j * 6 + s] * offA[s] + S[j * 6 + 3 + s] * offB[s];
        tot += S[j * 6 + s] + S[j * 6 + 3 + s];
      }
      grad_dk[j] = v;
      later += tot;
    }
  }
  /* dJ/dphi_p = -(1/NT) Im sum_{x,y} conj(G^_m) A^'_m, m the bin of centred index p */
  if (grad_phi && phi) {
    int nt = pb->nt;
    int64_t plane = (int64_t)pb->nx * pb->ny;
    cplx* gb = (cplx*)malloc(sizeof(cplx) * nt);
    cplx* ab = (cplx*)malloc(sizeof(cplx) * nt);
    double* acc = (double*)calloc(nt, sizeof(double));
    const cplx* a0 = st + phi_field * n;
    const cplx* g0 = g + phi_field * n;
    for (int64_t q = 0; q < plane; ++q) {
      for (int t = 0; t < nt; ++t) {
        gb[t] = g0[t * plane + q];
        ab[t] = a0[t * plane + q];
      }
      orc_fft1d(gb, nt, -1);
      orc_fft1d(ab, nt, -1);
      for (int m = 0; m < nt; ++m) acc[m] += cimag(conj(gb[m]) * ab[m]);
    }
    for (int m = 0; m < nt; ++m) grad_phi[(m + nt / 2) % nt] = -acc[m] / (double)nt;
    free(gb);
    free(ab);
    free(acc);
  }
  free(a2);
  free(S);
  free(g);
  free(phis);
  free(qs);
  free(qh);
  free(st);
  return J;
}

double orc_adjoint_gradient(const orc_problem* pb, const cplx* fields_in, int nz, double dz, const double* dk_steps,
                            const double* phi, int phi_field, const double* w, double* grad_phi,
                            double* grad_dk, const double* dk_map) {
  return adjoint_impl(pb, fields_in, nz, dz, dk_steps, phi, phi_field, w, grad_phi, grad_dk, dk_map, 0, NULL, NULL);
}

/* orc_adjoint_gradient under a map that changes along z (orc_propagate_map_z). */
double orc_adjoint_gradient_z(const orc_problem* pb, const cplx* fields_in, int nz, double dz, const double* dk_steps,
                              const double* phi, int phi_field, const double* w, double* grad_phi, double* grad_dk,
                              int nseg, const double* z_edges, const double* maps) {
  return adjoint_impl(pb, fields_in, nz, dz, dk_steps, phi, phi_field, w, grad_phi, grad_dk, NULL, nseg, z_edges,
                      maps);
}

/* J only (for finite differences): the same forward map as above. */
double orc_objective(const orc_problem* pb, const cplx* fields_in, int nz, double dz, const double* dk_steps,
                     const double* phi, int phi_field, const double* w, const double* dk_map) {
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt;
  int nf = pb->nf;
  cplx* a = (cplx*)malloc(sizeof(cplx) * n * nf);
  memcpy(a, fields_in, sizeof(cplx) * n * nf);
  if (phi) orc_spectral_phase(pb, a + phi_field * n, phi, +1);
  double ph = 0.0;
  if (dk_map)
    orc_propagate_map(pb, a, nz, dz, dk_steps, &ph, 0.0, dk_map);
  else
    orc_propagate(pb, a, nz, dz, dk_steps, &ph);
  double J = 0.0;
  for (int f = 0; f < nf; ++f)
    for (int64_t i = 0; i < n; ++i) J += w[f] * (creal(a[f * n + i]) * creal(a[f * n + i]) + cimag(a[f * n + i]) * cimag(a[f * n + i]));
  free(a);
  return J;
}

/* J only, under a map that changes along z. */
double orc_objective_z(const orc_problem* pb, const cplx* fields_in, int nz, double dz, const double* dk_steps,
                       const double* phi, int phi_field, const double* w, int nseg, const double* z_edges,
                       const double* maps) {
  int64_t n = (int64_t)pb->nx * pb->ny * pb->nt;
  int nf = pb->nf;
  cplx* a = (cplx*)malloc(sizeof(cplx) * n * nf);
  memcpy(a, fields_in, sizeof(cplx) * n * nf);
  if (phi) orc_spectral_phase(pb, a + phi_field * n, phi, +1);
  double ph = 0.0;
  orc_propagate_map_z(pb, a, nz, dz, dk_steps, &ph, nseg, z_edges, maps);
  double J = 0.0;
  for (int f = 0; f < nf; ++f)
    for (int64_t i = 0; i < n; ++i) J += w[f] * (creal(a[f * n + i]) * creal(a[f * n + i]) + cimag(a[f * n + i]) * cimag(a[f * n + i]));
  free(a);
  return J;
}
