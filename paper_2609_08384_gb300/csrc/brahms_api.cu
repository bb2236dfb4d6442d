// Host runtime behind the C ABI of include/brahms.h: context, workspace
// layout, table set-up, step sequencing and diagnostics.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "brahms.h"
#include "kernels.cuh"

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kHbar = 1.054571817e-34;
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kRedBlocks = 152 * 4;  // energy partials per field
constexpr int kKinds = 5;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout {
  size_t state, px, py, pt, twx, twy, twt, partial, energy, total;
};

Layout make_layout(int nx, int ny, int nt, int nf) {
  Layout L{};
  size_t off = 0;
  const size_t n = (size_t)nx * ny * nt;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return o;
  };
  L.state = take(sizeof(float2) * n * nf);
  L.px = take(sizeof(float2) * nx * nf);
  L.py = take(sizeof(float2) * ny * nf);
  L.pt = take(sizeof(float2) * nt * nf);
  L.twx = take(sizeof(float4) * nx);
  L.twy = take(sizeof(float4) * ny);
  L.twt = take(sizeof(float4) * nt);
  L.partial = take(sizeof(double) * kRedBlocks * nf);
  L.energy = take(sizeof(double) * nf);
  L.total = off;
  return L;
}

struct TimedLaunch {
  int kind;
  cudaEvent_t a, b;
};

}  // namespace

struct brahms_ctx {
  int nx = 0, ny = 0, nt = 0, nf = 0;
  double dx = 0, dy = 0, dt = 0, d_eff = 0, dk = 0;
  brahms_field_params fp[3]{};
  cudaStream_t stream = nullptr;
  bool own_ws = false;
  char* ws = nullptr;
  Layout L{};
  float2 *state = nullptr, *px = nullptr, *py = nullptr, *pt = nullptr;
  float4 *twx = nullptr, *twy = nullptr, *twt = nullptr;
  double *partial = nullptr, *energy_dev = nullptr;
  double* energy_host = nullptr;  // pinned, nf entries
  double tab_dz = NAN;
  bool have_fields = false;
  double z = 0.0, phi = 0.0;
  long long step = 0;
  std::vector<double> dk_profile;
  std::string err;
  long long launches = 0;
  // timing
  bool timing = false;
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;
  double kind_ms[kKinds]{};
  long long kind_n[kKinds]{};

  long long npoints() const { return (long long)nx * ny * nt; }
};

namespace {

brahms_status fail(brahms_ctx* c, brahms_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

brahms_status cuda_fail(brahms_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, BRAHMS_E_CUDA, m);
}

#define BR_CK(call)                                      \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

cudaEvent_t take_event(brahms_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch wrapper: counts launches and, when timing is on, brackets the
// launch with events on the context stream.
template <class Fn>
cudaError_t launch(brahms_ctx* c, int kind, int nlaunch, Fn fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->timing) {
    a = take_event(c);
    b = take_event(c);
    if (a && b) cudaEventRecord(a, c->stream);
  }
  cudaError_t e = fn();
  c->launches += nlaunch;
  if (c->timing && a && b) {
    cudaEventRecord(b, c->stream);
    c->timed.push_back({kind, a, b});
  }
  return e;
}

brahms_status collect_timing(brahms_ctx* ctx) {
  if (ctx->timed.empty()) return BRAHMS_OK;
  BR_CK(cudaStreamSynchronize(ctx->stream));
  for (auto& t : ctx->timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      ctx->kind_ms[t.kind] += ms;
      ctx->kind_n[t.kind] += 1;
    }
    ctx->event_pool.push_back(t.a);
    ctx->event_pool.push_back(t.b);
  }
  ctx->timed.clear();
  return BRAHMS_OK;
}

bool finite_params(const brahms_field_params& f) {
  return std::isfinite(f.lambda) && std::isfinite(f.n) && std::isfinite(f.delta) && std::isfinite(f.k2) &&
         std::isfinite(f.k3) && std::isfinite(f.rho) && std::isfinite(f.alpha) && f.lambda > 0 && f.n > 0 &&
         std::fabs(f.rho) < 1.5;
}

double kappa(const brahms_ctx* c, int f) { return kTwoPi * c->d_eff / (c->fp[f].n * c->fp[f].lambda); }

brahms_status build_tables(brahms_ctx* ctx, double dz) {
  if (ctx->tab_dz == dz) return BRAHMS_OK;
  brahms::TableArgs a{};
  a.px = ctx->px;
  a.py = ctx->py;
  a.pt = ctx->pt;
  a.nx = ctx->nx;
  a.ny = ctx->ny;
  a.nt = ctx->nt;
  a.nf = ctx->nf;
  a.dx = ctx->dx;
  a.dy = ctx->dy;
  a.dt = ctx->dt;
  a.dz = dz;
  for (int f = 0; f < ctx->nf; ++f) {
    a.k[f] = kTwoPi * ctx->fp[f].n / ctx->fp[f].lambda;
    a.rho[f] = ctx->fp[f].rho;
    a.delta[f] = ctx->fp[f].delta;
    a.k2[f] = ctx->fp[f].k2;
    a.k3[f] = ctx->fp[f].k3;
    a.alpha[f] = ctx->fp[f].alpha;
  }
  BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_prop_tables(a, ctx->stream); }));
  ctx->tab_dz = dz;
  return BRAHMS_OK;
}

brahms::XPassArgs xargs(brahms_ctx* c, int mode, double dz) {
  brahms::XPassArgs a{};
  a.data = c->state;
  a.fstride = c->npoints();
  a.rows = (long long)c->ny * c->nt;
  a.tw = c->twx;
  a.mode = mode;
  a.dz = dz;
  for (int f = 0; f < c->nf; ++f) {
    double k = kappa(c, f);
    if (c->nf == 2 && f == 0) k *= 0.5;  // degenerate SHG: 1/2 on the SH equation
    a.kh[f] = (float)(k * 0.5 * dz);
  }
  a.scale = 1.f;
  return a;
}

brahms::AxisArgs aargs(brahms_ctx* c, int axis) {
  brahms::AxisArgs a{};
  a.data = c->state;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nt = c->nt;
  a.fstride = c->npoints();
  const int n = axis == 1 ? c->ny : c->nt;
  const int tx = brahms::col_tile_of(n);
  a.xtiles = (c->nx + tx - 1) / tx;
  a.ntiles = (long long)c->nf * (axis == 1 ? c->nt : c->ny) * a.xtiles;
  a.tw = axis == 1 ? c->twy : c->twt;
  a.px = c->px;
  a.py = c->py;
  a.pt = c->pt;
  const double inv_n = 1.0 / (double)c->npoints();
  a.scale = (float)inv_n;
  a.scale_lo = (float)(inv_n - (double)a.scale);
  return a;
}

double dk_of_step(const brahms_ctx* c, long long j) {
  return j < (long long)c->dk_profile.size() ? c->dk_profile[(size_t)j] : c->dk;
}

// Enqueue an FP64 |A|^2 reduction per field into energy_host (pinned).
brahms_status enqueue_energy(brahms_ctx* ctx) {
  BR_CK(launch(ctx, 4, 2, [&] {
    return brahms::run_energy(ctx->state, ctx->npoints(), ctx->nf, ctx->npoints(), ctx->partial, kRedBlocks,
                              ctx->energy_dev, ctx->stream);
  }));
  BR_CK(cudaMemcpyAsync(ctx->energy_host, ctx->energy_dev, sizeof(double) * ctx->nf, cudaMemcpyDeviceToHost,
                        ctx->stream));
  return BRAHMS_OK;
}

brahms_status finish_with_check(brahms_ctx* ctx) {
  brahms_status s = enqueue_energy(ctx);
  if (s != BRAHMS_OK) return s;
  BR_CK(cudaStreamSynchronize(ctx->stream));
  for (int f = 0; f < ctx->nf; ++f)
    if (!std::isfinite(ctx->energy_host[f]))
      return fail(ctx, BRAHMS_E_NONFINITE, "fields are not finite (dz too large for the coupling, Sec. 3.2)");
  return BRAHMS_OK;
}

}  // namespace

extern "C" {

const char* brahms_status_string(brahms_status s) {
  switch (s) {
    case BRAHMS_OK: return "BRAHMS_OK";
    case BRAHMS_E_ARG: return "BRAHMS_E_ARG";
    case BRAHMS_E_SIZE: return "BRAHMS_E_SIZE";
    case BRAHMS_E_CUDA: return "BRAHMS_E_CUDA";
    case BRAHMS_E_OOM: return "BRAHMS_E_OOM";
    case BRAHMS_E_NONFINITE: return "BRAHMS_E_NONFINITE";
    case BRAHMS_E_TIMEOUT: return "BRAHMS_E_TIMEOUT";
    case BRAHMS_E_STATE: return "BRAHMS_E_STATE";
  }
  return "BRAHMS_E_UNKNOWN";
}

const char* brahms_last_error(const brahms_ctx* ctx) {
  if (!ctx) return "no context";
  return ctx->err.c_str();
}

brahms_status brahms_workspace_size(int nx, int ny, int nt, int nfields, size_t* bytes) {
  if (!bytes || (nfields != 2 && nfields != 3)) return BRAHMS_E_ARG;
  if (!brahms::size_supported(nx) || !brahms::size_supported(ny) || !brahms::size_supported(nt))
    return BRAHMS_E_SIZE;
  *bytes = make_layout(nx, ny, nt, nfields).total;
  return BRAHMS_OK;
}

brahms_status brahms_init_grid(brahms_ctx** out, int nx, int ny, int nt, double dx, double dy, double dt,
                               int nfields, const brahms_field_params* fp, double d_eff, double dk,
                               void* workspace, size_t workspace_bytes, void* cuda_stream) {
  if (!out || !fp) return BRAHMS_E_ARG;
  *out = nullptr;
  if (nfields != 2 && nfields != 3) return BRAHMS_E_ARG;
  if (!brahms::size_supported(nx) || !brahms::size_supported(ny) || !brahms::size_supported(nt))
    return BRAHMS_E_SIZE;
  if (!(dx > 0) || !(dy > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dt) ||
      !std::isfinite(d_eff) || !std::isfinite(dk))
    return BRAHMS_E_ARG;
  for (int f = 0; f < nfields; ++f)
    if (!finite_params(fp[f])) return BRAHMS_E_ARG;
  if (workspace && ((uintptr_t)workspace & 255)) return BRAHMS_E_ARG;

  brahms_ctx* ctx = new brahms_ctx();
  ctx->nx = nx;
  ctx->ny = ny;
  ctx->nt = nt;
  ctx->nf = nfields;
  ctx->dx = dx;
  ctx->dy = dy;
  ctx->dt = dt;
  ctx->d_eff = d_eff;
  ctx->dk = dk;
  for (int f = 0; f < nfields; ++f) ctx->fp[f] = fp[f];
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->L = make_layout(nx, ny, nt, nfields);
  if (workspace) {
    if (workspace_bytes < ctx->L.total) {
      delete ctx;
      return BRAHMS_E_OOM;
    }
    ctx->ws = (char*)workspace;
  } else {
    void* p = nullptr;
    if (cudaMalloc(&p, ctx->L.total) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return BRAHMS_E_OOM;
    }
    ctx->ws = (char*)p;
    ctx->own_ws = true;
  }
  if (cudaMallocHost((void**)&ctx->energy_host, sizeof(double) * 3) != cudaSuccess) {
    cudaGetLastError();
    brahms_free(ctx);
    return BRAHMS_E_OOM;
  }
  ctx->state = (float2*)(ctx->ws + ctx->L.state);
  ctx->px = (float2*)(ctx->ws + ctx->L.px);
  ctx->py = (float2*)(ctx->ws + ctx->L.py);
  ctx->pt = (float2*)(ctx->ws + ctx->L.pt);
  ctx->twx = (float4*)(ctx->ws + ctx->L.twx);
  ctx->twy = (float4*)(ctx->ws + ctx->L.twy);
  ctx->twt = (float4*)(ctx->ws + ctx->L.twt);
  ctx->partial = (double*)(ctx->ws + ctx->L.partial);
  ctx->energy_dev = (double*)(ctx->ws + ctx->L.energy);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = brahms::run_twiddles(ctx->twx, nx, ctx->stream);
  if (e == cudaSuccess) e = brahms::run_twiddles(ctx->twy, ny, ctx->stream);
  if (e == cudaSuccess) e = brahms::run_twiddles(ctx->twt, nt, ctx->stream);
  ctx->launches += 3;
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    brahms_free(ctx);
    return BRAHMS_E_CUDA;
  }
  *out = ctx;
  return BRAHMS_OK;
}

void brahms_free(brahms_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream || ctx->ws) cudaStreamSynchronize(ctx->stream);
  for (auto& t : ctx->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
  if (ctx->energy_host) cudaFreeHost(ctx->energy_host);
  delete ctx;
}

brahms_status brahms_set_fields(brahms_ctx* ctx, const void* const* fields, int dtype, int on_device) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!fields) return fail(ctx, BRAHMS_E_ARG, "fields is NULL");
  if (dtype != BRAHMS_C64 && dtype != BRAHMS_C128) return fail(ctx, BRAHMS_E_ARG, "dtype must be C64 or C128");
  const long long n = ctx->npoints();
  for (int f = 0; f < ctx->nf; ++f)
    if (!fields[f]) return fail(ctx, BRAHMS_E_ARG, "a field pointer is NULL");
  std::vector<float2> stage;
  for (int f = 0; f < ctx->nf; ++f) {
    float2* dst = ctx->state + f * n;
    if (dtype == BRAHMS_C64) {
      BR_CK(cudaMemcpyAsync(dst, fields[f], sizeof(float2) * n,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    } else if (on_device) {
      BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_c128_to_c64((const double2*)fields[f], dst, n, ctx->stream); }));
    } else {
      const double* src = (const double*)fields[f];
      stage.resize((size_t)n);
      for (long long i = 0; i < n; ++i) stage[i] = make_float2((float)src[2 * i], (float)src[2 * i + 1]);
      BR_CK(cudaMemcpyAsync(dst, stage.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, ctx->stream));
      BR_CK(cudaStreamSynchronize(ctx->stream));
    }
  }
  ctx->z = 0.0;
  ctx->phi = 0.0;
  ctx->step = 0;
  ctx->have_fields = true;
  brahms_status s = finish_with_check(ctx);
  if (s == BRAHMS_E_NONFINITE) {
    ctx->have_fields = false;
    return fail(ctx, BRAHMS_E_ARG, "input fields contain non-finite values");
  }
  return s;
}

brahms_status brahms_set_dk_profile(brahms_ctx* ctx, const double* dk, int n) {
  if (!ctx) return BRAHMS_E_ARG;
  if (n < 0 || (n > 0 && !dk)) return fail(ctx, BRAHMS_E_ARG, "bad profile");
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(dk[i])) return fail(ctx, BRAHMS_E_ARG, "profile has non-finite entries");
  ctx->dk_profile.assign(dk, dk + n);
  return BRAHMS_OK;
}

brahms_status brahms_propagate(brahms_ctx* ctx, int nz, double dz) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!ctx->have_fields) return fail(ctx, BRAHMS_E_STATE, "propagate before set_fields");
  if (nz < 0 || !(dz > 0) || !std::isfinite(dz)) return fail(ctx, BRAHMS_E_ARG, "need nz >= 0 and dz > 0");
  if (nz == 0) return BRAHMS_OK;
  brahms_status s = build_tables(ctx, dz);
  if (s != BRAHMS_OK) return s;
  const int nx = ctx->nx, ny = ctx->ny, nt = ctx->nt, nf = ctx->nf;
  const brahms::AxisArgs ay = aargs(ctx, 1);
  const brahms::AxisArgs at = aargs(ctx, 2);
  double phi = ctx->phi;  // Phi(z_j) of the current step j
  long long j = ctx->step;
  {
    brahms::XPassArgs a = xargs(ctx, brahms::XM_NL_FIRST, dz);
    a.phiA = phi;
    a.dkA = dk_of_step(ctx, j);
    BR_CK(launch(ctx, 0, 1, [&] { return brahms::run_xpass(nx, nf, a, ctx->stream); }));
  }
  for (int i = 0; i < nz; ++i, ++j) {
    const double dkj = dk_of_step(ctx, j);
    BR_CK(launch(ctx, 1, 1, [&] { return brahms::run_axis_fft(ny, 1, false, ay, ctx->stream); }));
    BR_CK(launch(ctx, 2, 1, [&] { return brahms::run_tpass_prop(nt, at, ctx->stream); }));
    BR_CK(launch(ctx, 3, 1, [&] { return brahms::run_axis_fft(ny, 1, true, ay, ctx->stream); }));
    const bool last = (i == nz - 1);
    brahms::XPassArgs a = xargs(ctx, last ? brahms::XM_NL_LAST : brahms::XM_NL_MID, dz);
    a.phiB = phi;
    a.dkB = dkj;
    phi += dkj * dz;
    a.phiA = phi;
    a.dkA = dk_of_step(ctx, j + 1);
    BR_CK(launch(ctx, 0, 1, [&] { return brahms::run_xpass(nx, nf, a, ctx->stream); }));
  }
  ctx->phi = phi;
  ctx->step = j;
  ctx->z += nz * dz;
  return BRAHMS_OK;
}

brahms_status brahms_get_fields(brahms_ctx* ctx, void* const* out, int dtype, int on_device) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!out) return fail(ctx, BRAHMS_E_ARG, "out is NULL");
  if (!ctx->have_fields) return fail(ctx, BRAHMS_E_STATE, "no fields set");
  if (dtype != BRAHMS_C64 && dtype != BRAHMS_C128) return fail(ctx, BRAHMS_E_ARG, "dtype must be C64 or C128");
  for (int f = 0; f < ctx->nf; ++f)
    if (!out[f]) return fail(ctx, BRAHMS_E_ARG, "an output pointer is NULL");
  const long long n = ctx->npoints();
  std::vector<float2> stage;
  for (int f = 0; f < ctx->nf; ++f) {
    const float2* src = ctx->state + f * n;
    if (dtype == BRAHMS_C64) {
      BR_CK(cudaMemcpyAsync(out[f], src, sizeof(float2) * n,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    } else if (on_device) {
      BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_c64_to_c128(src, (double2*)out[f], n, ctx->stream); }));
    } else {
      stage.resize((size_t)n);
      BR_CK(cudaMemcpyAsync(stage.data(), src, sizeof(float2) * n, cudaMemcpyDeviceToHost, ctx->stream));
      BR_CK(cudaStreamSynchronize(ctx->stream));
      double* d = (double*)out[f];
      for (long long i = 0; i < n; ++i) {
        d[2 * i] = stage[i].x;
        d[2 * i + 1] = stage[i].y;
      }
    }
  }
  return finish_with_check(ctx);
}

brahms_status brahms_energy(brahms_ctx* ctx, double* energy_j, double* photons) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!energy_j) return fail(ctx, BRAHMS_E_ARG, "energy_j is NULL");
  if (!ctx->have_fields) return fail(ctx, BRAHMS_E_STATE, "no fields set");
  brahms_status s = finish_with_check(ctx);
  const double cell = ctx->dx * ctx->dy * ctx->dt;
  for (int f = 0; f < ctx->nf; ++f) {
    const double e = 0.5 * kC0 * kEps0 * ctx->fp[f].n * ctx->energy_host[f] * cell;
    energy_j[f] = e;
    if (photons) photons[f] = e / (kHbar * kTwoPi * kC0 / ctx->fp[f].lambda);
  }
  return s;
}

brahms_status brahms_sync(brahms_ctx* ctx) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!ctx->have_fields) {
    BR_CK(cudaStreamSynchronize(ctx->stream));
    return BRAHMS_OK;
  }
  return finish_with_check(ctx);
}

brahms_status brahms_transform(brahms_ctx* ctx, int direction) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!ctx->have_fields) return fail(ctx, BRAHMS_E_STATE, "no fields set");
  if (direction != -1 && direction != 1) return fail(ctx, BRAHMS_E_ARG, "direction must be -1 or +1");
  const brahms::AxisArgs ay = aargs(ctx, 1), at = aargs(ctx, 2);
  const bool inv = direction == 1;
  brahms::XPassArgs a = xargs(ctx, inv ? brahms::XM_INV : brahms::XM_FWD, 1.0);
  a.scale = (float)(1.0 / (double)ctx->npoints());
  BR_CK(launch(ctx, 0, 1, [&] { return brahms::run_xpass(ctx->nx, ctx->nf, a, ctx->stream); }));
  BR_CK(launch(ctx, 1, 1, [&] { return brahms::run_axis_fft(ctx->ny, 1, inv, ay, ctx->stream); }));
  BR_CK(launch(ctx, 2, 1, [&] { return brahms::run_axis_fft(ctx->nt, 2, inv, at, ctx->stream); }));
  BR_CK(cudaStreamSynchronize(ctx->stream));
  return BRAHMS_OK;
}

brahms_status brahms_get_z(const brahms_ctx* ctx, double* z, double* phi) {
  if (!ctx) return BRAHMS_E_ARG;
  if (z) *z = ctx->z;
  if (phi) *phi = ctx->phi;
  return BRAHMS_OK;
}

brahms_status brahms_timing(brahms_ctx* ctx, int enable, double* ms, long long* launches, int nkinds) {
  if (!ctx) return BRAHMS_E_ARG;
  brahms_status s = collect_timing(ctx);
  if (s != BRAHMS_OK) return s;
  for (int k = 0; k < nkinds && k < kKinds; ++k) {
    if (ms) ms[k] = ctx->kind_ms[k];
    if (launches) launches[k] = ctx->kind_n[k];
  }
  if (enable) {
    for (int k = 0; k < kKinds; ++k) {
      ctx->kind_ms[k] = 0.0;
      ctx->kind_n[k] = 0;
    }
  }
  ctx->timing = enable != 0;
  return BRAHMS_OK;
}

long long brahms_launch_count(const brahms_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
