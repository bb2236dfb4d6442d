// Host runtime behind the C ABI of include/brahms.h: context, workspace
// layout, table set-up, step sequencing and diagnostics.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx_internal.h"

using namespace brahms_host;


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

namespace {
// x needs a transform of its own (it carries the nonlinear step); y and tau
// may also have a single sample (a 1D transverse or a cw problem)
bool grid_supported(int nx, int ny, int nt) {
  return brahms::size_supported(nx) && (ny == 1 || brahms::size_supported(ny)) &&
         (nt == 1 || brahms::size_supported(nt));
}
}  // namespace

brahms_status brahms_workspace_size(int nx, int ny, int nt, int nfields, size_t* bytes) {
  if (!bytes || (nfields != 2 && nfields != 3)) return BRAHMS_E_ARG;
  if (!grid_supported(nx, ny, nt)) return BRAHMS_E_SIZE;
  *bytes = make_layout(nx, ny, nt, nfields).total;
  return BRAHMS_OK;
}

brahms_status brahms_init_grid(brahms_ctx** out, int nx, int ny, int nt, double dx, double dy, double dt,
                               int nfields, const brahms_field_params* fp, double d_eff, double dk,
                               void* workspace, size_t workspace_bytes, void* cuda_stream) {
  if (!out || !fp) return BRAHMS_E_ARG;
  *out = nullptr;
  if (nfields != 2 && nfields != 3) return BRAHMS_E_ARG;
  if (!grid_supported(nx, ny, nt)) return BRAHMS_E_SIZE;
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
    if (brahms::dev_alloc(&p, ctx->L.total) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return BRAHMS_E_OOM;
    }
    ctx->ws = (char*)p;
    ctx->own_ws = true;
  }
  if (brahms::pinned_alloc((void**)&ctx->energy_host, sizeof(double) * 4) != cudaSuccess) {
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
  ctx->dev_err = (int*)(ctx->ws + ctx->L.err);
  ctx->diag_dev = (double*)(ctx->ws + ctx->L.diag);
  ctx->ws_map = (double*)(ctx->ws + ctx->L.dkmap);
  ctx->ws_umap = (double*)(ctx->ws + ctx->L.usermap);
  ctx->maps_dev = ctx->ws_map;
  ctx->umaps_dev = ctx->ws_umap;
  ctx->mphase_dev = (double*)(ctx->ws + ctx->L.mphase);
  ctx->emap_dev = (float2*)(ctx->ws + ctx->L.emap);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = brahms::upload_twiddles(ctx->twx, nx, ctx->stream);
  if (e == cudaSuccess && ny > 1) e = brahms::upload_twiddles(ctx->twy, ny, ctx->stream);
  if (e == cudaSuccess && nt > 1) e = brahms::upload_twiddles(ctx->twt, nt, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->mphase_dev, 0, sizeof(double) * nx * ny, ctx->stream);
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
  for (int f = 0; f < 3; ++f) {
    if (ctx->fstream[f]) cudaStreamDestroy(ctx->fstream[f]);
    if (ctx->ev_y[f]) cudaEventDestroy(ctx->ev_y[f]);
    if (ctx->ev_done[f]) cudaEventDestroy(ctx->ev_done[f]);
  }
  if (ctx->ev_x) cudaEventDestroy(ctx->ev_x);
  if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
  if (ctx->adj_mem) cudaFree(ctx->adj_mem);
  if (ctx->th_mem) cudaFree(ctx->th_mem);
  if (ctx->seg_mem) cudaFree(ctx->seg_mem);
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
  {
    const brahms_status sr = map_phase_reset(ctx);
    if (sr != BRAHMS_OK) return sr;
  }
  ctx->have_fields = true;
  touch(ctx);
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
  touch(ctx);
  return BRAHMS_OK;
}

brahms_status brahms_propagate(brahms_ctx* ctx, int nz, double dz) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!ctx->have_fields) return fail(ctx, BRAHMS_E_STATE, "propagate before set_fields");
  if (nz < 0 || !(dz > 0) || !std::isfinite(dz)) return fail(ctx, BRAHMS_E_ARG, "need nz >= 0 and dz > 0");
  if (nz == 0) return BRAHMS_OK;
  touch(ctx);
  brahms_status s = build_tables(ctx, dz);
  if (s != BRAHMS_OK) return s;
  const int nx = ctx->nx, ny = ctx->ny, nt = ctx->nt, nf = ctx->nf;
  const brahms::AxisArgs ay = aargs(ctx, 1);
  const brahms::AxisArgs at = aargs(ctx, 2);
  double phi = ctx->phi;  // Phi(z_j) of the current step j
  long long j = ctx->step;
  const double z0 = ctx->z;
  {
    brahms::XPassArgs a = xargs(ctx, brahms::XM_NL_FIRST, dz);
    a.phiA = phi;
    a.dkA = dk_of_step(ctx, j);
    s = enqueue_map_tables(ctx, 0.0, 0.0, z0, a.phiA, a.dkA, z0, dz);
    if (s != BRAHMS_OK) return s;
    BR_CK(launch(ctx, 0, 1, [&] { return brahms::run_xpass(nx, nf, a, ctx->stream); }));
  }
  // per-field streams for the y/tau/y passes only when the option asks for
  // them (off by default: a gain on 128x128x256 with three fields only)
  const bool split = use_field_streams(ctx);
  for (int i = 0; i < nz; ++i, ++j) {
    const double dkj = dk_of_step(ctx, j);
    if (split) {
      s = enqueue_linear_split(ctx, ay, at);
      if (s != BRAHMS_OK) return s;
    } else {
      if (ny > 1) BR_CK(launch(ctx, 1, 1, [&] { return brahms::run_axis_fft(ny, 1, false, ay, ctx->stream); }));
      if (nt == 1)
        BR_CK(launch(ctx, 2, 1, [&] { return brahms::run_prop_pointwise(at, nf, ctx->stream); }));
      else if (ctx->use_tma)
        BR_CK(launch(ctx, 2, 1, [&] {
          return brahms::run_tpass_prop_tma(nt, ctx->use_tma, ctx->tmap_state, at, ctx->dev_err, ctx->tma_wait_ns,
                                            ctx->stream);
        }));
      else
        BR_CK(launch(ctx, 2, 1, [&] { return brahms::run_tpass_prop(nt, at, ctx->stream); }));
      if (ny > 1) BR_CK(launch(ctx, 3, 1, [&] { return brahms::run_axis_fft(ny, 1, true, ay, ctx->stream); }));
    }
    const bool last = (i == nz - 1);
    brahms::XPassArgs a = xargs(ctx, last ? brahms::XM_NL_LAST : brahms::XM_NL_MID, dz);
    a.phiB = phi;
    a.dkB = dkj;
    phi += dkj * dz;
    a.phiA = phi;
    a.dkA = dk_of_step(ctx, j + 1);
    s = enqueue_map_tables(ctx, a.phiB, a.dkB, z0 + i * dz, a.phiA, a.dkA, z0 + (i + 1) * dz, dz);
    if (s != BRAHMS_OK) return s;
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

brahms_status brahms_shg_efficiency_weights(brahms_ctx* ctx, double* weights) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!weights) return fail(ctx, BRAHMS_E_ARG, "weights is NULL");
  if (ctx->nf != 2) return fail(ctx, BRAHMS_E_ARG, "SHG efficiency weights need the two fields (SH, F)");
  if (!ctx->have_fields) return fail(ctx, BRAHMS_E_STATE, "no fields set");
  const brahms_status s = finish_with_check(ctx);  // energy_host[f] = sum |A_f|^2
  if (s != BRAHMS_OK) return s;
  const double sum_f = ctx->energy_host[1];
  if (!(sum_f > 0.0)) return fail(ctx, BRAHMS_E_ARG, "the fundamental is zero");
  // eta = E_SH(L) / E_F(0): E = 1/2 c eps0 n sum |A|^2 dx dy dtau, the common factors cancel
  weights[0] = ctx->fp[0].n / (ctx->fp[1].n * sum_f);
  weights[1] = 0.0;
  return BRAHMS_OK;
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
  touch(ctx);
  const brahms::AxisArgs ay = aargs(ctx, 1), at = aargs(ctx, 2, false);
  const bool inv = direction == 1;
  brahms::XPassArgs a = xargs(ctx, inv ? brahms::XM_INV : brahms::XM_FWD, 1.0);
  a.scale = (float)(1.0 / (double)ctx->npoints());
  BR_CK(launch(ctx, 0, 1, [&] { return brahms::run_xpass(ctx->nx, ctx->nf, a, ctx->stream); }));
  if (ctx->ny > 1) BR_CK(launch(ctx, 1, 1, [&] { return brahms::run_axis_fft(ctx->ny, 1, inv, ay, ctx->stream); }));
  if (ctx->nt > 1) BR_CK(launch(ctx, 2, 1, [&] { return brahms::run_axis_fft(ctx->nt, 2, inv, at, ctx->stream); }));
  BR_CK(cudaStreamSynchronize(ctx->stream));
  return BRAHMS_OK;
}

brahms_status brahms_set_dk_map_z(brahms_ctx* ctx, int nseg, const double* z_edges, const double* maps) {
  if (!ctx) return BRAHMS_E_ARG;
  if (nseg < 1 || nseg > kMaxMapSegments) return fail(ctx, BRAHMS_E_ARG, "nseg out of range");
  if (nseg > 1 && !z_edges) return fail(ctx, BRAHMS_E_ARG, "z_edges is NULL");
  for (int i = 0; i + 1 < nseg; ++i)
    if (!std::isfinite(z_edges[i]) || !(z_edges[i] > (i ? z_edges[i - 1] : 0.0)))
      return fail(ctx, BRAHMS_E_ARG, "z_edges must be finite, positive and increasing");
  const size_t nxy = (size_t)ctx->nx * ctx->ny;
  if (maps)
    for (size_t i = 0; i < nxy * nseg; ++i)
      if (!std::isfinite(maps[i])) return fail(ctx, BRAHMS_E_ARG, "dk_map has non-finite entries");
  // the maps in effect so far keep their share of the phase
  brahms_status s = map_phase_sync(ctx);
  if (s != BRAHMS_OK) return s;
  if (nseg != ctx->nseg) {
    BR_CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->seg_mem) cudaFree(ctx->seg_mem);
    ctx->seg_mem = nullptr;
    ctx->maps_dev = ctx->ws_map;
    ctx->umaps_dev = ctx->ws_umap;
    ctx->nseg = 1;
    ctx->zedge.clear();
    ctx->have_user_map = ctx->have_therm = false;
    // zero maps until the new ones are in (what stays in effect if the allocation fails)
    BR_CK(cudaMemsetAsync(ctx->ws_map, 0, sizeof(double) * nxy, ctx->stream));
    BR_CK(cudaMemsetAsync(ctx->ws_umap, 0, sizeof(double) * nxy, ctx->stream));
    if (nseg > 1) {
      const size_t plane = align256(sizeof(double) * nxy * nseg);
      if (brahms::dev_alloc((void**)&ctx->seg_mem, 2 * plane) != cudaSuccess) {
        cudaGetLastError();
        ctx->seg_mem = nullptr;
        update_have_map(ctx);
        return fail(ctx, BRAHMS_E_OOM, "z-segment maps");
      }
      ctx->maps_dev = (double*)ctx->seg_mem;
      ctx->umaps_dev = (double*)(ctx->seg_mem + plane);
    }
    // heat loads belong to the old segments
    ctx->have_heat.clear();
  } else if (nseg > 1 && !std::equal(ctx->zedge.begin(), ctx->zedge.end(), z_edges)) {
    ctx->have_heat.clear();
  }
  ctx->nseg = nseg;
  if (nseg > 1)
    ctx->zedge.assign(z_edges, z_edges + (nseg - 1));
  else
    ctx->zedge.clear();
  const size_t bytes = sizeof(double) * nxy * nseg;
  if (maps) {
    BR_CK(cudaMemcpyAsync(ctx->umaps_dev, maps, bytes, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    BR_CK(cudaMemsetAsync(ctx->umaps_dev, 0, bytes, ctx->stream));
  }
  BR_CK(cudaMemcpyAsync(ctx->maps_dev, ctx->umaps_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  BR_CK(cudaStreamSynchronize(ctx->stream));
  ctx->have_user_map = maps != nullptr;
  ctx->have_therm = false;
  update_have_map(ctx);
  touch(ctx);
  return BRAHMS_OK;
}

brahms_status brahms_set_dk_map(brahms_ctx* ctx, const double* dk_map) {
  return brahms_set_dk_map_z(ctx, 1, nullptr, dk_map);
}

brahms_status brahms_diagnostics(brahms_ctx* ctx, double* power, double* spectrum) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!ctx->have_fields) return fail(ctx, BRAHMS_E_STATE, "no fields set");
  if (!power && !spectrum) return BRAHMS_OK;
  const int nt = ctx->nt, nf = ctx->nf;
  double* pw = ctx->diag_dev;
  double* sp = ctx->diag_dev + (size_t)nf * nt;
  const bool want_power = power || nt == 1;
  if (want_power)
    BR_CK(launch(ctx, 4, 1, [&] {
      return brahms::run_power_trace(ctx->state, ctx->nx, ctx->ny, nt, nf, ctx->npoints(), pw, ctx->stream);
    }));
  if (spectrum && nt > 1) {
    const brahms::AxisArgs at = aargs(ctx, 2, false);
    BR_CK(cudaMemsetAsync(sp, 0, sizeof(double) * nf * nt, ctx->stream));
    BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_tau_spectrum(nt, at, sp, ctx->stream); }));
  }
  std::vector<double> h((size_t)2 * nf * nt);
  BR_CK(cudaMemcpyAsync(h.data(), ctx->diag_dev, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
  BR_CK(cudaStreamSynchronize(ctx->stream));
  for (int f = 0; f < nf; ++f) {
    const double c = 0.5 * kC0 * kEps0 * ctx->fp[f].n * ctx->dx * ctx->dy;
    for (int k = 0; k < nt; ++k) {
      const double p = c * h[(size_t)f * nt + k];
      if (power) power[(size_t)f * nt + k] = p;
      // nt = 1: the tau transform is the identity and the one bin holds P dt
      if (spectrum) spectrum[(size_t)f * nt + k] = nt == 1 ? p * ctx->dt : c * ctx->dt / nt * h[(size_t)(nf + f) * nt + k];
    }
  }
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
      ctx->kind_seen[k] = 0;
    }
    ctx->timing_every = enable > 1 ? enable : 1;
  }
  ctx->timing = enable != 0;
  return BRAHMS_OK;
}

long long brahms_launch_count(const brahms_ctx* ctx) { return ctx ? ctx->launches : 0; }

brahms_status brahms_set_option(brahms_ctx* ctx, int option, int value) {
  if (!ctx) return BRAHMS_E_ARG;
  if (option == BRAHMS_OPT_TMA_TAU) {
    if (!value) {
      ctx->use_tma = 0;
      return BRAHMS_OK;
    }
    if (value != 1 && value != 8 && value != 16)
      return fail(ctx, BRAHMS_E_ARG, "TMA tau-pass: 1 (prefetching) or a tile width of 8 or 16 columns");
    if (!brahms::tma_tau_supported(ctx->nx, ctx->nt))
      return fail(ctx, BRAHMS_E_SIZE, "TMA tau-pass needs nt in {256, 512} and nx >= 16");
    BR_CK(brahms::make_tau_tensor_map(ctx->tmap_state, ctx->state, ctx->nx, ctx->ny, ctx->nt, ctx->nf,
                                      value == 1 ? 16 : value));
    ctx->use_tma = value;
    return BRAHMS_OK;
  }
  if (option == BRAHMS_OPT_FIELD_STREAMS) {
    if (value != 0 && value != 1) return fail(ctx, BRAHMS_E_ARG, "field streams: 0 or 1");
    ctx->field_streams = value;
    return BRAHMS_OK;
  }
  if (option == BRAHMS_OPT_TMA_WAIT_US) {
    if (value < 0 || value > 2000000) return fail(ctx, BRAHMS_E_ARG, "TMA wait limit: 0 to 2000000 us");
    ctx->tma_wait_ns = 1000ULL * (unsigned long long)value;
    return BRAHMS_OK;
  }
  return fail(ctx, BRAHMS_E_ARG, "unknown option");
}

int brahms_get_option(const brahms_ctx* ctx, int option) {
  if (!ctx) return -1;
  if (option == BRAHMS_OPT_TMA_TAU) return ctx->use_tma;
  if (option == BRAHMS_OPT_FIELD_STREAMS) return ctx->field_streams;
  if (option == BRAHMS_OPT_TMA_WAIT_US) return (int)(ctx->tma_wait_ns / 1000ULL);
  return -1;
}

}  // extern "C"
