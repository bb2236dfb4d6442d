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

// Loads and temperatures of every z-segment (allocated on first use and again
// when the number of segments changes); loads of segments that have none are
// zero.
brahms_status thermal_alloc(brahms_ctx* ctx) {
  const size_t nxy = (size_t)ctx->nx * ctx->ny;
  if (ctx->th_mem && ctx->th_nseg != ctx->nseg) {
    BR_CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->th_mem);
    ctx->th_mem = nullptr;
    ctx->th_nseg = 0;
  }
  if (!ctx->th_mem) {
    size_t off = 0;
    auto take = [&](size_t b) {
      size_t o = off;
      off += align256(b);
      return o;
    };
    const size_t o_h = take(sizeof(double) * nxy * ctx->nseg), o_t = take(sizeof(double) * nxy * ctx->nseg);
    const size_t o_x = take(sizeof(double2) * 2 * ctx->nx), o_y = take(sizeof(double2) * 2 * ctx->ny);
    const size_t o_b = take(sizeof(int));
    if (brahms::dev_alloc((void**)&ctx->th_mem, off) != cudaSuccess) {
      cudaGetLastError();
      ctx->th_mem = nullptr;
      return fail(ctx, BRAHMS_E_OOM, "thermal model memory");
    }
    ctx->th_nseg = ctx->nseg;
    ctx->th_heat = (double*)(ctx->th_mem + o_h);
    ctx->th_temp = (double*)(ctx->th_mem + o_t);
    ctx->th_twx = (double2*)(ctx->th_mem + o_x);
    ctx->th_twy = (double2*)(ctx->th_mem + o_y);
    ctx->th_bad = (int*)(ctx->th_mem + o_b);
    ctx->have_heat.clear();
    BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_sine_twiddles(ctx->th_twx, ctx->nx, ctx->stream); }));
    if (ctx->ny > 1)
      BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_sine_twiddles(ctx->th_twy, ctx->ny, ctx->stream); }));
  }
  if ((int)ctx->have_heat.size() != ctx->nseg) {
    BR_CK(cudaMemsetAsync(ctx->th_heat, 0, sizeof(double) * nxy * ctx->nseg, ctx->stream));
    ctx->have_heat.assign(ctx->nseg, 0);
  }
  return BRAHMS_OK;
}

}  // namespace

extern "C" {

brahms_status brahms_heat_accumulate_segment(brahms_ctx* ctx, int segment, double rep_rate, double weight) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!ctx->have_fields) return fail(ctx, BRAHMS_E_STATE, "no fields set");
  if (segment < 0 || segment >= ctx->nseg) return fail(ctx, BRAHMS_E_ARG, "segment out of range");
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
  a.heat = ctx->th_heat + (size_t)segment * ctx->nx * ctx->ny;
  BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_heat_load(a, ctx->stream); }));
  ctx->have_heat[segment] = 1;
  return BRAHMS_OK;
}

brahms_status brahms_heat_accumulate(brahms_ctx* ctx, double rep_rate, double weight) {
  if (!ctx) return BRAHMS_E_ARG;
  return brahms_heat_accumulate_segment(ctx, seg_of(ctx, ctx->z), rep_rate, weight);
}

brahms_status brahms_heat_set(brahms_ctx* ctx, const double* q) {
  if (!ctx) return BRAHMS_E_ARG;
  const size_t n = (size_t)ctx->nx * ctx->ny * ctx->nseg;
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
  ctx->have_heat.assign(ctx->nseg, 1);
  return BRAHMS_OK;
}

brahms_status brahms_thermal_map(brahms_ctx* ctx, double kappa_th, double dkdT, double* temperature) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!(kappa_th > 0) || !std::isfinite(kappa_th) || !std::isfinite(dkdT))
    return fail(ctx, BRAHMS_E_ARG, "kappa_th must be finite and > 0, dkdT finite");
  if ((int)ctx->have_heat.size() != ctx->nseg || !ctx->th_mem || ctx->th_nseg != ctx->nseg)
    return fail(ctx, BRAHMS_E_STATE, "no heat load accumulated or set");
  for (int sg = 0; sg < ctx->nseg; ++sg)
    if (!ctx->have_heat[sg]) return fail(ctx, BRAHMS_E_STATE, "a z-segment has no heat load accumulated or set");
  // the maps in effect so far keep their share of the phase
  brahms_status s = map_phase_sync(ctx);
  if (s != BRAHMS_OK) return s;
  const size_t nxy = (size_t)ctx->nx * ctx->ny;
  BR_CK(cudaMemsetAsync(ctx->th_bad, 0, sizeof(int), ctx->stream));
  for (int sg = 0; sg < ctx->nseg; ++sg) {
    brahms::ThermalArgs a{};
    a.heat = ctx->th_heat + sg * nxy;
    a.temp = ctx->th_temp + sg * nxy;
    a.twx = ctx->th_twx;
    a.twy = ctx->th_twy;
    a.nx = ctx->nx;
    a.ny = ctx->ny;
    a.dx = ctx->dx;
    a.dy = ctx->dy;
    a.kappa = kappa_th;
    a.dkdT = dkdT;
    a.dkmap = ctx->maps_dev + sg * nxy;
    a.bad = ctx->th_bad;
    int nl = 0;
    BR_CK(launch(ctx, 4, 0, [&] { return brahms::run_thermal_solve(a, &nl, ctx->stream); }));
    ctx->launches += nl;
  }
  if (ctx->have_user_map)
    BR_CK(launch(ctx, 4, 1, [&] {
      return brahms::run_map_add(ctx->maps_dev, ctx->umaps_dev, (long long)(nxy * ctx->nseg), ctx->stream);
    }));
  int bad = 0;
  BR_CK(cudaMemcpyAsync(&bad, ctx->th_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (temperature)
    BR_CK(cudaMemcpyAsync(temperature, ctx->th_temp, sizeof(double) * nxy * ctx->nseg, cudaMemcpyDeviceToHost,
                          ctx->stream));
  BR_CK(cudaStreamSynchronize(ctx->stream));
  touch(ctx);
  if (bad) {
    // the solve wrote the maps in place: put back the caller's maps (zero if
    // none), so that propagation goes on under the maps the caller set
    BR_CK(cudaMemcpyAsync(ctx->maps_dev, ctx->umaps_dev, sizeof(double) * nxy * ctx->nseg, cudaMemcpyDeviceToDevice,
                          ctx->stream));
    BR_CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_therm = false;
    update_have_map(ctx);
    return fail(ctx, BRAHMS_E_NONFINITE, "heat load or temperature not finite; the map of brahms_set_dk_map stays");
  }
  ctx->have_therm = true;
  update_have_map(ctx);
  return BRAHMS_OK;
}

}  // extern "C"
