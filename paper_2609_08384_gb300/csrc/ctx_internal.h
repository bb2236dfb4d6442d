// Host-side context of the C ABI and the helpers shared by the forward
// (brahms_api.cu) and adjoint (brahms_adjoint.cu) entry points.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "alloc_hook.h"
#include "brahms.h"
#include "kernels.cuh"

namespace brahms_host {

constexpr double kC0 = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kHbar = 1.054571817e-34;
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kRedBlocks = 152 * 2;  // energy partials per field (all fields' blocks in one wave)
constexpr int kKinds = 5;
constexpr int kMaxMapSegments = 4096;  // z-segments of a mismatch map

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout {
  size_t state, px, py, pt, twx, twy, twt, partial, energy, err, diag, dkmap, usermap, mphase, emap, total;
};

inline Layout make_layout(int nx, int ny, int nt, int nf) {
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
  L.twx = take(sizeof(float4) * brahms::tw_table_size_of(nx));
  L.twy = take(sizeof(float4) * brahms::tw_table_size_of(ny));
  L.twt = take(sizeof(float4) * brahms::tw_table_size_of(nt));
  L.partial = take(sizeof(double) * kRedBlocks * nf);
  L.energy = take(sizeof(double) * nf);
  L.err = take(sizeof(int));
  L.diag = take(sizeof(double) * 2 * nt * nf);
  L.dkmap = take(sizeof(double) * nx * ny);
  L.usermap = take(sizeof(double) * nx * ny);
  L.mphase = take(sizeof(double) * nx * ny);
  L.emap = take(sizeof(float2) * 4 * nx * ny);
  L.total = off;
  return L;
}

struct TimedLaunch {
  int kind;
  cudaEvent_t a, b;
};

}  // namespace

struct brahms_ctx {
  using Layout = brahms_host::Layout;
  using TimedLaunch = brahms_host::TimedLaunch;
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
  double* energy_host = nullptr;  // pinned, nf entries + the device error word
  double* diag_dev = nullptr;     // diagnostics: power [nf][nt], spectrum [nf][nt]
  // Transverse mismatch maps, one per z-segment (nseg segments separated by
  // the nseg - 1 distances zedge; one segment: the workspace's two planes)
  int nseg = 1;
  std::vector<double> zedge;
  double* maps_dev = nullptr;     // maps in effect [nseg][ny][nx] (1/m)
  double* umaps_dev = nullptr;    // the caller's maps [nseg][ny][nx] (the thermal map adds to them)
  double* ws_map = nullptr;       // the workspace's planes for one segment
  double* ws_umap = nullptr;
  char* seg_mem = nullptr;        // both arrays when nseg > 1
  float2* emap_dev = nullptr;     // stage phase factors for one x-pass [4][ny][nx]
  // the map's share of the coupling phase: P (mphase_dev [ny][nx]) is its
  // integral up to map_zp, map_cur the segment in effect since (-1: none yet)
  double* mphase_dev = nullptr;
  double map_zp = 0.0;
  int map_cur = -1;
  bool mphase_live = false;       // P may be non-zero (a map changed during this run)
  bool have_map = false;          // the x-pass takes the map path
  bool have_user_map = false;
  bool have_therm = false;        // a thermal map is installed
  int* dev_err = nullptr;          // set by kernels whose bounded waits expired
  unsigned long long tma_wait_ns = 2000000000ULL;  // limit of each TMA tile wait (BRAHMS_OPT_TMA_WAIT_US)
  alignas(64) unsigned char tmap_state[128];  // TMA map of the state for the tau-pass
  int use_tma = 0;  // 0 plain tau-pass; 16 or 8: TMA tau-pass with tiles of that many columns
  // per-field streams for the y/tau/y chain of a step (created on first use)
  int field_streams = 0;  // 0 off (default), 1 on
  cudaStream_t fstream[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_x = nullptr, ev_y[3] = {nullptr, nullptr, nullptr}, ev_done[3] = {nullptr, nullptr, nullptr};
  double tab_dz = NAN;
  bool have_fields = false;
  // generation of the state: every call that changes the fields, the map or
  // the profile advances it; the adjoint's reverse sweep runs only for the
  // generation its forward left
  unsigned long long gen = 0;
  double z = 0.0, phi = 0.0;
  long long step = 0;
  std::vector<double> dk_profile;
  std::string err;
  long long launches = 0;
  // timing: events around every timing_every-th launch of each kind
  bool timing = false;
  int timing_every = 1;
  long long kind_seen[brahms_host::kKinds]{};
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;
  double kind_ms[brahms_host::kKinds]{};
  long long kind_n[brahms_host::kKinds]{};
  // adjoint (allocated on first use by brahms_adjoint_forward)
  char* adj_mem = nullptr;
  size_t adj_bytes = 0;
  float2* adj_ckpt = nullptr;  // checkpoints, one state each
  float2* adj_seg = nullptr;   // recorded states of one segment: B half-step inputs [K], A half-step inputs [K]
  float2* adj_work = nullptr;  // recomputed state within a step
  float2* adj_g = nullptr;     // adjoint state
  float2* adj_tab = nullptr;   // spectral-phase tables: x (nx), y (ny), tau (nt)
  double* adj_part = nullptr;  // stage-sensitivity partials of one reverse x-pass [CTAs][6]
  double* adj_sens = nullptr;  // [nz][6] stage sensitivities
  double* adj_phi_dev = nullptr;  // spectral phase (nt)
  double* adj_acc = nullptr;      // phase-gradient accumulators (nt)
  bool adj_has_phi = false;
  int adj_nz = 0, adj_K = 0, adj_nseg = 0, adj_phi_field = -1;
  double adj_dz = 0.0;
  bool adj_ready = false;
  unsigned long long adj_gen = 0;  // gen at the end of the last brahms_adjoint_forward
  bool adj_store_all = false;  // the forward recorded every step (no recomputation)
  std::vector<double> adj_weights, adj_dk, adj_phis;
  std::vector<int> adj_zseg, adj_zcnt;  // z-segment of every step; steps per z-segment before every step
  // thermal model (allocated on first use)
  char* th_mem = nullptr;
  int th_nseg = 0;             // segments th_mem holds
  double* th_heat = nullptr;   // heat load per segment [nseg][ny][nx] W/m^3
  double* th_temp = nullptr;   // temperature rise per segment [nseg][ny][nx] K
  double2* th_twx = nullptr;   // sine-transform tables (2 nx, 2 ny entries)
  double2* th_twy = nullptr;
  int* th_bad = nullptr;       // non-finite temperature flag
  std::vector<char> have_heat; // per segment: a load was accumulated or set

  long long npoints() const { return (long long)nx * ny * nt; }
};

namespace brahms_host {

inline brahms_status fail(brahms_ctx* c, brahms_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

// the state, the map or the profile changed
inline void touch(brahms_ctx* c) { ++c->gen; }

inline brahms_status cuda_fail(brahms_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, BRAHMS_E_CUDA, m);
}

#define BR_CK(call)                                      \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

inline cudaEvent_t take_event(brahms_ctx* c) {
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
// launch with events on the stream it is enqueued on.
template <class Fn>
inline cudaError_t launch_on(brahms_ctx* c, cudaStream_t st, int kind, int nlaunch, Fn fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  const bool timed = c->timing && (c->kind_seen[kind]++ % c->timing_every) == 0;
  if (timed) {
    a = take_event(c);
    b = take_event(c);
    if (a && b) cudaEventRecord(a, st);
  }
  cudaError_t e = fn();
  c->launches += nlaunch;
  if (timed && a && b) {
    cudaEventRecord(b, st);
    c->timed.push_back({kind, a, b});
  }
  return e;
}
template <class Fn>
inline cudaError_t launch(brahms_ctx* c, int kind, int nlaunch, Fn fn) {
  return launch_on(c, c->stream, kind, nlaunch, fn);
}

inline brahms_status collect_timing(brahms_ctx* ctx) {
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

inline bool finite_params(const brahms_field_params& f) {
  return std::isfinite(f.lambda) && std::isfinite(f.n) && std::isfinite(f.delta) && std::isfinite(f.k2) &&
         std::isfinite(f.k3) && std::isfinite(f.rho) && std::isfinite(f.alpha) && f.lambda > 0 && f.n > 0 &&
         std::fabs(f.rho) < 1.5;
}

inline double kappa(const brahms_ctx* c, int f) { return kTwoPi * c->d_eff / (c->fp[f].n * c->fp[f].lambda); }

inline brahms_status build_tables(brahms_ctx* ctx, double dz) {
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

inline brahms::XPassArgs xargs(brahms_ctx* c, int mode, double dz) {
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
    a.kh2[f] = 0.5f * a.kh[f];
  }
  a.scale = 1.f;
  a.ny = c->ny;
  a.emap = c->have_map ? c->emap_dev : nullptr;
  return a;
}

// segment that holds distance z (the one that starts at z on an edge)
inline int seg_of(const brahms_ctx* c, double z) {
  int s = 0;
  while (s < c->nseg - 1 && c->zedge[s] <= z) ++s;
  return s;
}

inline void update_have_map(brahms_ctx* c) { c->have_map = c->have_user_map || c->have_therm || c->mphase_live; }

// Before the maps are replaced: bring P up to the current distance with the
// map in effect, so that the phase stays continuous where the new maps take
// over.
inline brahms_status map_phase_sync(brahms_ctx* ctx) {
  if (ctx->have_fields && ctx->have_map && ctx->map_cur >= 0 && ctx->z > ctx->map_zp) {
    const double len = ctx->z - ctx->map_zp;
    const double* m = ctx->maps_dev + (size_t)ctx->map_cur * ctx->nx * ctx->ny;
    BR_CK(launch(ctx, 4, 1, [&] {
      return brahms::run_map_phase_advance(ctx->mphase_dev, m, len, (long long)ctx->nx * ctx->ny, ctx->stream);
    }));
    ctx->mphase_live = true;
  }
  ctx->map_zp = ctx->z;
  ctx->map_cur = -1;
  return BRAHMS_OK;
}

// A new run (brahms_set_fields): P = 0 from z = 0.
inline brahms_status map_phase_reset(brahms_ctx* ctx) {
  if (ctx->mphase_live)
    BR_CK(cudaMemsetAsync(ctx->mphase_dev, 0, sizeof(double) * ctx->nx * ctx->ny, ctx->stream));
  ctx->mphase_live = false;
  ctx->map_zp = 0.0;
  ctx->map_cur = -1;
  update_have_map(ctx);
  return BRAHMS_OK;
}

// Stage phase factors of the next x-pass under the mismatch map: B applies
// the second half of the step that starts at distance zB (mismatch phase
// phiB, mismatch dkB), A the first half of the step that starts at zA.  Each
// step takes the map of the segment that holds its midpoint.
inline brahms_status enqueue_map_tables(brahms_ctx* ctx, double phiB, double dkB, double zB, double phiA,
                                        double dkA, double zA, double dz) {
  if (!ctx->have_map) return BRAHMS_OK;
  const size_t nxy = (size_t)ctx->nx * ctx->ny;
  const int sA = seg_of(ctx, zA + 0.5 * dz);
  // no map in effect yet: the map of step A starts here (P holds at zA)
  const int sB = ctx->map_cur >= 0 ? ctx->map_cur : sA;
  brahms::MapArgs m{};
  m.mapB = ctx->maps_dev + sB * nxy;
  m.mapA = ctx->maps_dev + sA * nxy;
  m.mphase = ctx->mphase_dev;
  m.emap = ctx->emap_dev;
  m.nxy = (long long)nxy;
  m.phiB = phiB;
  m.dkB = dkB;
  m.zB = zB;
  m.phiA = phiA;
  m.dkA = dkA;
  m.zA = zA;
  m.dz = dz;
  m.zp = ctx->map_zp;
  m.advance = sA != sB;
  BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_map_tables(m, ctx->stream); }));
  if (m.advance) {
    ctx->map_zp = zA;
    ctx->mphase_live = true;
  }
  ctx->map_cur = sA;
  return BRAHMS_OK;
}

// axis 1: y-pass; axis 2 with tau_prop: tau propagator; axis 2 without: tau FFT only
inline brahms::AxisArgs aargs(brahms_ctx* c, int axis, bool tau_prop = true) {
  brahms::AxisArgs a{};
  a.data = c->state;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nt = c->nt;
  a.fstride = c->npoints();
  const int n = axis == 1 ? c->ny : c->nt;
  const int tx0 = (axis == 2 && tau_prop) ? brahms::tau_col_tile_of(n) : brahms::col_tile_of(n);
  const int tx = tx0 > 0 ? tx0 : 1;  // an axis of length 1 has no tiles of its own
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

// Per-field streams for the y-forward, tau-propagator and y-inverse of a
// step, when the option asks for them (measured on GB300: 5 % faster on
// 128x128x256 with three fields, 2-28 % slower on two-field and small grids,
// within 3 % either way on larger ones).
inline bool use_field_streams(const brahms_ctx* c) {
  return c->field_streams == 1 && c->ny > 1 && c->nt > 1 && !c->use_tma;
}

// streams and events of the per-field chains, created on first use
inline brahms_status field_streams_ready(brahms_ctx* ctx) {
  if (ctx->ev_x) return BRAHMS_OK;
  for (int f = 0; f < 3; ++f) {
    BR_CK(cudaStreamCreateWithFlags(&ctx->fstream[f], cudaStreamNonBlocking));
    BR_CK(cudaEventCreateWithFlags(&ctx->ev_y[f], cudaEventDisableTiming));
    BR_CK(cudaEventCreateWithFlags(&ctx->ev_done[f], cudaEventDisableTiming));
  }
  BR_CK(cudaEventCreateWithFlags(&ctx->ev_x, cudaEventDisableTiming));
  return BRAHMS_OK;
}

// strided-pencil arguments restricted to field f
inline brahms::AxisArgs field_args(const brahms_ctx* ctx, const brahms::AxisArgs& a, int f) {
  brahms::AxisArgs b = a;
  b.data = a.data + (long long)f * a.fstride;
  b.px = a.px + (long long)f * ctx->nx;
  b.py = a.py + (long long)f * ctx->ny;
  b.pt = a.pt + (long long)f * ctx->nt;
  b.ntiles = a.ntiles / ctx->nf;
  return b;
}

// The y-forward, tau-propagator and y-inverse of one step with field f's on
// stream f, field f+1 starting its y-forward once field f's is done, so that
// one field's DRAM-bound y-passes overlap another's tau-pass; the context
// stream waits for all of them.
inline brahms_status enqueue_linear_split(brahms_ctx* ctx, const brahms::AxisArgs& ay, const brahms::AxisArgs& at) {
  brahms_status s = field_streams_ready(ctx);
  if (s != BRAHMS_OK) return s;
  BR_CK(cudaEventRecord(ctx->ev_x, ctx->stream));
  for (int f = 0; f < ctx->nf; ++f) {
    cudaStream_t st = ctx->fstream[f];
    const brahms::AxisArgs ayf = field_args(ctx, ay, f), atf = field_args(ctx, at, f);
    BR_CK(cudaStreamWaitEvent(st, ctx->ev_x, 0));
    if (f > 0) BR_CK(cudaStreamWaitEvent(st, ctx->ev_y[f - 1], 0));
    BR_CK(launch_on(ctx, st, 1, 1, [&] { return brahms::run_axis_fft(ctx->ny, 1, false, ayf, st); }));
    BR_CK(cudaEventRecord(ctx->ev_y[f], st));
    BR_CK(launch_on(ctx, st, 2, 1, [&] { return brahms::run_tpass_prop(ctx->nt, atf, st); }));
    BR_CK(launch_on(ctx, st, 3, 1, [&] { return brahms::run_axis_fft(ctx->ny, 1, true, ayf, st); }));
    BR_CK(cudaEventRecord(ctx->ev_done[f], st));
  }
  for (int f = 0; f < ctx->nf; ++f) BR_CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_done[f], 0));
  return BRAHMS_OK;
}

inline double dk_of_step(const brahms_ctx* c, long long j) {
  return j < (long long)c->dk_profile.size() ? c->dk_profile[(size_t)j] : c->dk;
}

// Enqueue an FP64 |A|^2 reduction per field into energy_host (pinned).
inline brahms_status enqueue_energy(brahms_ctx* ctx) {
  BR_CK(launch(ctx, 4, 2, [&] {
    return brahms::run_energy(ctx->state, ctx->npoints(), ctx->nf, ctx->npoints(), ctx->partial, kRedBlocks,
                              ctx->energy_dev, ctx->stream);
  }));
  BR_CK(cudaMemcpyAsync(ctx->energy_host, ctx->energy_dev, sizeof(double) * ctx->nf, cudaMemcpyDeviceToHost,
                        ctx->stream));
  return BRAHMS_OK;
}

inline brahms_status finish_with_check(brahms_ctx* ctx) {
  brahms_status s = enqueue_energy(ctx);
  if (s != BRAHMS_OK) return s;
  int* herr = reinterpret_cast<int*>(ctx->energy_host + 3);
  BR_CK(cudaMemcpyAsync(herr, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  BR_CK(cudaStreamSynchronize(ctx->stream));
  if (*herr != 0) {
    BR_CK(cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), ctx->stream));
    return fail(ctx, BRAHMS_E_TIMEOUT, "a bounded device wait expired (TMA copy not completed)");
  }
  for (int f = 0; f < ctx->nf; ++f)
    if (!std::isfinite(ctx->energy_host[f]))
      return fail(ctx, BRAHMS_E_NONFINITE, "fields are not finite (dz too large for the coupling, Sec. 3.2)");
  return BRAHMS_OK;
}

}  // namespace
