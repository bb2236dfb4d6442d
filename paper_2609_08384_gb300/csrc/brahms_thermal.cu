// Thermal model entry points (Sec. 4.1: the steady-state heat equation
// lap T = -Q / kappa on the fields' grid, and the temperature-dependent phase
// mismatch): heat load of the fields, the transverse Poisson solve and the
// mismatch map it induces.  Kernels in k_thermal.cu.
#include "ctx_internal.h"

using namespace brahms_host;

namespace brahms {
// k_thermal.cu: dkmap += base
cudaError_t run_map_add(double* dkmap, const double* base, long long n, cudaStream_t s);
}  // namespace brahms

namespace {

brahms_status thermal_alloc(brahms_ctx* ctx) {
  if (ctx->th_mem) return BRAHMS_OK;
  const size_t nxy = (size_t)ctx->nx * ctx->ny;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += align256(b);
    return o;
  };
  const size_t o_h = take(sizeof(double) * nxy), o_t = take(sizeof(double) * nxy);
  const size_t o_x = take(sizeof(double2) * ctx->nx), o_y = take(sizeof(double2) * ctx->ny);
  const size_t o_b = take(sizeof(int));
  if (brahms::dev_alloc((void**)&ctx->th_mem, off) != cudaSuccess) {
    cudaGetLastError();
    ctx->th_mem = nullptr;
    return fail(ctx, BRAHMS_E_OOM, "thermal model memory");
  }
  ctx->th_heat = (double*)(ctx->th_mem + o_h);
  ctx->th_temp = (double*)(ctx->th_mem + o_t);
  ctx->th_twx = (double2*)(ctx->th_mem + o_x);
  ctx->th_twy = (double2*)(ctx->th_mem + o_y);
  ctx->th_bad = (int*)(ctx->th_mem + o_b);
  BR_CK(cudaMemsetAsync(ctx->th_heat, 0, sizeof(double) * nxy, ctx->stream));
  BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_sine_twiddles(ctx->th_twx, ctx->nx, ctx->stream); }));
  if (ctx->ny > 1)
    BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_sine_twiddles(ctx->th_twy, ctx->ny, ctx->stream); }));
  return BRAHMS_OK;
}

}  // namespace

extern "C" {

brahms_status brahms_heat_accumulate(brahms_ctx* ctx, double rep_rate, double weight) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!ctx->have_fields) return fail(ctx, BRAHMS_E_STATE, "no fields set");
  if (!std::isfinite(weight) || !std::isfinite(rep_rate) || rep_rate < 0)
    return fail(ctx, BRAHMS_E_ARG, "rep_rate must be finite and >= 0, weight finite");
  brahms_status s = thermal_alloc(ctx);
  if (s != BRAHMS_OK) return s;
  brahms::HeatArgs a{};
  a.data = ctx->state;
  a.fstride = ctx->npoints();
  a.nx = ctx->nx;
  a.ny = ctx->ny;
  a.nt = ctx->nt;
  a.nf = ctx->nf;
  // nt > 1: pulse energy absorbed per volume times the repetition rate
  const double tavg = ctx->nt > 1 ? rep_rate * ctx->dt : 1.0;
  for (int f = 0; f < ctx->nf; ++f) a.c[f] = weight * ctx->fp[f].alpha * 0.5 * kC0 * kEps0 * ctx->fp[f].n * tavg;
  a.heat = ctx->th_heat;
  BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_heat_load(a, ctx->stream); }));
  ctx->have_heat = true;
  return BRAHMS_OK;
}

brahms_status brahms_heat_set(brahms_ctx* ctx, const double* q) {
  if (!ctx) return BRAHMS_E_ARG;
  const size_t n = (size_t)ctx->nx * ctx->ny;
  if (q)
    for (size_t i = 0; i < n; ++i)
      if (!std::isfinite(q[i])) return fail(ctx, BRAHMS_E_ARG, "heat load has non-finite entries");
  brahms_status s = thermal_alloc(ctx);
  if (s != BRAHMS_OK) return s;
  if (q)
    BR_CK(cudaMemcpyAsync(ctx->th_heat, q, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  else
    BR_CK(cudaMemsetAsync(ctx->th_heat, 0, sizeof(double) * n, ctx->stream));
  BR_CK(cudaStreamSynchronize(ctx->stream));
  ctx->have_heat = true;
  return BRAHMS_OK;
}

brahms_status brahms_thermal_map(brahms_ctx* ctx, double kappa_th, double dkdT, double* temperature) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!(kappa_th > 0) || !std::isfinite(kappa_th) || !std::isfinite(dkdT))
    return fail(ctx, BRAHMS_E_ARG, "kappa_th must be finite and > 0, dkdT finite");
  if (!ctx->have_heat) return fail(ctx, BRAHMS_E_STATE, "no heat load accumulated or set");
  brahms::ThermalArgs a{};
  a.heat = ctx->th_heat;
  a.temp = ctx->th_temp;
  a.twx = ctx->th_twx;
  a.twy = ctx->th_twy;
  a.nx = ctx->nx;
  a.ny = ctx->ny;
  a.dx = ctx->dx;
  a.dy = ctx->dy;
  a.kappa = kappa_th;
  a.dkdT = dkdT;
  a.dkmap = ctx->dkmap_dev;
  a.bad = ctx->th_bad;
  BR_CK(cudaMemsetAsync(ctx->th_bad, 0, sizeof(int), ctx->stream));
  int nl = 0;
  BR_CK(launch(ctx, 4, 0, [&] { return brahms::run_thermal_solve(a, &nl, ctx->stream); }));
  ctx->launches += nl;
  if (ctx->have_user_map)
    BR_CK(launch(ctx, 4, 1, [&] {
      return brahms::run_map_add(ctx->dkmap_dev, ctx->usermap_dev, (long long)ctx->nx * ctx->ny, ctx->stream);
    }));
  int bad = 0;
  BR_CK(cudaMemcpyAsync(&bad, ctx->th_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (temperature)
    BR_CK(cudaMemcpyAsync(temperature, ctx->th_temp, sizeof(double) * ctx->nx * ctx->ny, cudaMemcpyDeviceToHost,
                          ctx->stream));
  BR_CK(cudaStreamSynchronize(ctx->stream));
  touch(ctx);
  if (bad) {
    // the solve wrote the map in place: put back the map of brahms_set_dk_map
    // (or none), so that propagation goes on under the map the caller set
    if (ctx->have_user_map)
      BR_CK(cudaMemcpyAsync(ctx->dkmap_dev, ctx->usermap_dev, sizeof(double) * ctx->nx * ctx->ny,
                            cudaMemcpyDeviceToDevice, ctx->stream));
    BR_CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_map = ctx->have_user_map;
    return fail(ctx, BRAHMS_E_NONFINITE, "heat load or temperature not finite; the map of brahms_set_dk_map stays");
  }
  ctx->have_map = true;
  return BRAHMS_OK;
}

}  // extern "C"
