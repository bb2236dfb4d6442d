// Adjoint of the split-step propagation with sqrt(nz) checkpointing:
// gradients of J = sum_f w_f sum |A_f(L)|^2 with respect to an input spectral
// phase and to the per-step mismatch profile.
//
// Forward: the state is checkpointed every K steps (K = ceil(sqrt(nz)) by
// default) while the fused propagation runs.  Backward: segments are visited
// last to first.  Each is recomputed from its checkpoint with the recording
// x-pass, which keeps the states entering every B half step (a2_j) and every
// A half step (A_j).  With a negative checkpoint interval the forward itself
// runs the recording x-pass over all nz steps (2 nz states of memory) and the
// backward recomputes nothing.  The adjoint then runs the forward's pass structure in
// reverse: at each boundary b between steps b-1 and b one reverse x-pass
// (inverse x-FFT, reverse of N_A at A_b, reverse of N_B at a2_{b-1}, forward
// x-FFT), then the adjoint of the linear step, IDFT3(conj(P) DFT3), as the
// y-forward, conjugated tau-propagator and y-inverse passes.
// The mismatch gradient follows from the stage sensitivities dJ/dPhi with
// Phi(z) = Phi_j + dk_j (z - z_j); the phase gradient from the tau-spectra of
// the adjoint and of the phased input.
#include <algorithm>

#include "ctx_internal.h"
#include "map_seg.h"

using namespace brahms_host;

namespace {

// y-forward, tau-propagator (conjugated for the adjoint) and y-inverse on data
brahms_status linear_yty(brahms_ctx* ctx, float2* data, bool adjoint) {
  brahms::AxisArgs ay = aargs(ctx, 1), at = aargs(ctx, 2);
  ay.data = data;
  at.data = data;
  at.conj_p = adjoint ? 1 : 0;
  if (use_field_streams(ctx)) return enqueue_linear_split(ctx, ay, at);
  BR_CK(launch(ctx, 1, 1, [&] { return brahms::run_axis_fft(ctx->ny, 1, false, ay, ctx->stream); }));
  BR_CK(launch(ctx, 2, 1, [&] { return brahms::run_tpass_prop(ctx->nt, at, ctx->stream); }));
  BR_CK(launch(ctx, 3, 1, [&] { return brahms::run_axis_fft(ctx->ny, 1, true, ay, ctx->stream); }));
  return BRAHMS_OK;
}

// Stage factors of the x-pass that applies the B half of step jB and the A
// half of step jA (distances from z = 0).  One map: the running-sum tables of
// the forward.  A map that changes along z: the closed form from the steps'
// z-segments recorded by brahms_adjoint_forward (adj_zseg, and adj_zcnt, the
// steps of every z-segment before each step).
brahms_status adj_map_tables(brahms_ctx* ctx, int jB, int jA, double phiB, double dkB, double phiA, double dkA,
                             double dz) {
  if (!ctx->have_map) return BRAHMS_OK;
  if (ctx->nseg == 1) return enqueue_map_tables(ctx, phiB, dkB, jB * dz, phiA, dkA, jA * dz, dz);
  const int nz = ctx->adj_nz, nseg = ctx->nseg;
  const int b = std::min(std::max(jB, 0), nz), a = std::min(std::max(jA, 0), nz);
  brahms::MapSegArgs m{};
  m.maps = ctx->maps_dev;
  m.emap = ctx->emap_dev;
  m.nxy = (long long)ctx->nx * ctx->ny;
  m.nseg = nseg;
  m.sB = ctx->adj_zseg[std::min(b, nz - 1)];
  m.sA = ctx->adj_zseg[std::min(a, nz - 1)];
  for (int s = 0; s < nseg; ++s) {
    m.cB[s] = dz * ctx->adj_zcnt[(size_t)b * nseg + s];
    m.cA[s] = dz * ctx->adj_zcnt[(size_t)a * nseg + s];
  }
  m.phiB = phiB;
  m.dkB = dkB;
  m.phiA = phiA;
  m.dkA = dkA;
  m.dz = dz;
  BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_map_tables_seg(m, ctx->stream); }));
  return BRAHMS_OK;
}

// Steps j0 .. j1-1 from the real-space state in data (the state entering
// step j0's A half step) in the forward's pass structure, with the recording
// x-pass: a2_j (entering step j's B half step) goes to recB[j - j0] and A_j
// (entering step j's A half step, j > j0) to recA[j - j0].  Needs adj_nz,
// adj_dk and adj_phis.
brahms_status record_steps(brahms_ctx* ctx, float2* data, int j0, int j1, double dz, float2* recB, float2* recA) {
  const int nx = ctx->nx, nf = ctx->nf;
  const long long n = ctx->npoints();
  auto dk_at = [&](int j) { return j < ctx->adj_nz ? ctx->adj_dk[j] : ctx->dk; };
  {
    brahms::XPassArgs x = xargs(ctx, brahms::XM_NL_FIRST, dz);
    x.data = data;
    x.phiA = ctx->adj_phis[j0];
    x.dkA = dk_at(j0);
    brahms_status sm = adj_map_tables(ctx, j0, j0, 0.0, 0.0, x.phiA, x.dkA, dz);
    if (sm != BRAHMS_OK) return sm;
    BR_CK(launch(ctx, 0, 1, [&] { return brahms::run_xpass(nx, nf, x, ctx->stream); }));
  }
  for (int j = j0; j < j1; ++j) {
    brahms_status s2 = linear_yty(ctx, data, false);
    if (s2 != BRAHMS_OK) return s2;
    const bool last = j == j1 - 1;
    brahms::XPassArgs x = xargs(ctx, last ? brahms::XM_NL_LAST : brahms::XM_NL_MID, dz);
    x.data = data;
    x.phiB = ctx->adj_phis[j];
    x.dkB = dk_at(j);
    x.phiA = ctx->adj_phis[j + 1];
    x.dkA = dk_at(j + 1);
    x.rec_b = recB + (size_t)(j - j0) * nf * n;
    x.rec_a = last ? nullptr : recA + (size_t)(j + 1 - j0) * nf * n;
    s2 = adj_map_tables(ctx, j, j + 1, x.phiB, x.dkB, x.phiA, x.dkA, dz);
    if (s2 != BRAHMS_OK) return s2;
    BR_CK(launch(ctx, 0, 1, [&] { return brahms::run_xpass_record(nx, nf, x, ctx->stream); }));
  }
  return BRAHMS_OK;
}

brahms_status adj_alloc(brahms_ctx* ctx, int nz, int K, int nseg) {
  const size_t state = sizeof(float2) * (size_t)ctx->nf * (size_t)ctx->npoints();
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += align256(b);
    return o;
  };
  // checkpoints; per segment the recorded states entering each step's B half
  // (K) and A half (K); the recomputation's state; the adjoint
  const size_t o_ck = take(state * nseg), o_seg = take(state * 2 * K), o_w = take(state), o_g = take(state);
  const size_t o_tab = take(sizeof(float2) * (ctx->nx + ctx->ny + ctx->nt));
  const size_t o_phi = take(sizeof(double) * ctx->nt), o_acc = take(sizeof(double) * ctx->nt);
  const long long ncta = brahms::xpass_adjoint_ctas(ctx->nx, (long long)ctx->ny * ctx->nt);
  const size_t o_part = take(sizeof(double) * (size_t)(ncta > 0 ? ncta : 1) * 6);
  const size_t o_sens = take(sizeof(double) * (size_t)nz * 6);
  if (off > ctx->adj_bytes) {
    if (ctx->adj_mem) cudaFree(ctx->adj_mem);
    ctx->adj_mem = nullptr;
    ctx->adj_bytes = 0;
    if (brahms::dev_alloc((void**)&ctx->adj_mem, off) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BRAHMS_E_OOM, "adjoint checkpoint memory");
    }
    ctx->adj_bytes = off;
  }
  char* m = ctx->adj_mem;
  ctx->adj_ckpt = (float2*)(m + o_ck);
  ctx->adj_seg = (float2*)(m + o_seg);
  ctx->adj_work = (float2*)(m + o_w);
  ctx->adj_g = (float2*)(m + o_g);
  ctx->adj_tab = (float2*)(m + o_tab);
  ctx->adj_phi_dev = (double*)(m + o_phi);
  ctx->adj_acc = (double*)(m + o_acc);
  ctx->adj_part = (double*)(m + o_part);
  ctx->adj_sens = (double*)(m + o_sens);
  return BRAHMS_OK;
}

}  // namespace

extern "C" {

brahms_status brahms_adjoint_forward(brahms_ctx* ctx, const void* const* fields, int dtype, int on_device,
                                     const double* phi, int phi_field, const double* dk, int nz, double dz,
                                     const double* weights, int checkpoint_interval, double* J) {
  if (!ctx) return BRAHMS_E_ARG;
  // any failure below leaves no forward for brahms_adjoint_backward to reverse
  ctx->adj_ready = false;
  if (ctx->ny < 2 || ctx->nt < 2) return fail(ctx, BRAHMS_E_SIZE, "the adjoint needs ny >= 2 and nt >= 2");
  if (ctx->nseg > brahms::kMapSegMax)
    return fail(ctx, BRAHMS_E_STATE, "the adjoint takes a mismatch map of at most 16 z-segments");
  if (!dk || !weights || nz < 1 || !(dz > 0) || !std::isfinite(dz))
    return fail(ctx, BRAHMS_E_ARG, "need dk[nz], weights[nfields], nz >= 1, dz > 0");
  if (phi && (phi_field < 0 || phi_field >= ctx->nf)) return fail(ctx, BRAHMS_E_ARG, "phi_field out of range");
  if (phi)
    for (int i = 0; i < ctx->nt; ++i)
      if (!std::isfinite(phi[i])) return fail(ctx, BRAHMS_E_ARG, "phi has non-finite entries");
  const bool store_all = checkpoint_interval < 0;
  const int K = store_all ? nz
                          : (checkpoint_interval > 0 ? std::min(checkpoint_interval, nz)
                                                     : std::max(1, (int)std::ceil(std::sqrt((double)nz))));
  const int nseg = (nz + K - 1) / K;
  brahms_status s = adj_alloc(ctx, nz, K, nseg);
  if (s != BRAHMS_OK) return s;
  s = brahms_set_fields(ctx, fields, dtype, on_device);
  if (s != BRAHMS_OK) return s;
  s = brahms_set_dk_profile(ctx, dk, nz);
  if (s != BRAHMS_OK) return s;
  const long long n = ctx->npoints();
  ctx->adj_has_phi = phi != nullptr;
  if (phi) {
    // A_f <- IDFT_tau( e^{i phi} DFT_tau A_f ) on the chosen field
    BR_CK(cudaMemcpyAsync(ctx->adj_phi_dev, phi, sizeof(double) * ctx->nt, cudaMemcpyHostToDevice, ctx->stream));
    float2* px = ctx->adj_tab;
    float2* py = px + ctx->nx;
    float2* pt = py + ctx->ny;
    BR_CK(launch(ctx, 4, 1, [&] {
      return brahms::run_phase_tables(px, ctx->nx, py, ctx->ny, pt, ctx->nt, ctx->adj_phi_dev, +1, ctx->stream);
    }));
    brahms::AxisArgs at = aargs(ctx, 2);
    at.data = ctx->state + phi_field * n;
    at.ntiles = (long long)ctx->ny * at.xtiles;
    at.px = px;
    at.py = py;
    at.pt = pt;
    const double inv = 1.0 / (double)ctx->nt;
    at.scale = (float)inv;
    at.scale_lo = (float)(inv - (double)at.scale);
    BR_CK(launch(ctx, 2, 1, [&] { return brahms::run_tpass_prop(ctx->nt, at, ctx->stream); }));
  }
  // bookkeeping for the reverse sweep (Phi_j exactly as brahms_propagate accumulates it)
  ctx->adj_ready = false;
  ctx->adj_nz = nz;
  ctx->adj_K = K;
  ctx->adj_nseg = nseg;
  ctx->adj_dz = dz;
  ctx->adj_phi_field = phi ? phi_field : -1;
  ctx->adj_weights.assign(weights, weights + ctx->nf);
  ctx->adj_dk.assign(dk, dk + nz);
  ctx->adj_phis.assign(nz + 1, 0.0);
  double ph = 0.0;
  for (int i = 0; i < nz; ++i) {
    ctx->adj_phis[i] = ph;
    ph += dk[i] * dz;
  }
  ctx->adj_phis[nz] = ph;
  ctx->adj_store_all = store_all;
  if (ctx->nseg > 1) {
    // the z-segment of every step, as brahms_propagate picks it from the
    // distances it accumulates (one call of nz steps, or one per checkpoint)
    const int zs = ctx->nseg;
    ctx->adj_zseg.assign(nz, 0);
    ctx->adj_zcnt.assign((size_t)(nz + 1) * zs, 0);
    double zc = 0.0;
    for (int j0 = 0; j0 < nz; j0 += store_all ? nz : K) {
      const int cnt = std::min(store_all ? nz : K, nz - j0);
      for (int i = 0; i < cnt; ++i) ctx->adj_zseg[j0 + i] = seg_of(ctx, (i == 0 ? zc : zc + i * dz) + 0.5 * dz);
      zc += cnt * dz;
    }
    for (int j = 0; j < nz; ++j)
      for (int q = 0; q < zs; ++q)
        ctx->adj_zcnt[(size_t)(j + 1) * zs + q] = ctx->adj_zcnt[(size_t)j * zs + q] + (ctx->adj_zseg[j] == q);
  }
  if (store_all) {
    // the forward records every step's B and A inputs; A_0 is the checkpoint
    BR_CK(cudaMemcpyAsync(ctx->adj_ckpt, ctx->state, sizeof(float2) * ctx->nf * n, cudaMemcpyDeviceToDevice,
                          ctx->stream));
    s = build_tables(ctx, dz);
    if (s != BRAHMS_OK) return s;
    s = record_steps(ctx, ctx->state, 0, nz, dz, ctx->adj_seg, ctx->adj_seg + (size_t)K * ctx->nf * n);
    if (s != BRAHMS_OK) return s;
    ctx->phi = ph;
    ctx->step += nz;
    ctx->z += nz * dz;
    if (ctx->nseg > 1 && ctx->have_map) {
      // the map's share of the phase at z = L, for a propagation that goes on from here
      for (int q = 0; q < ctx->nseg; ++q) {
        const double len = dz * ctx->adj_zcnt[(size_t)nz * ctx->nseg + q];
        const double* mq = ctx->maps_dev + (size_t)q * ctx->nx * ctx->ny;
        if (len != 0.0)
          BR_CK(launch(ctx, 4, 1, [&] {
            return brahms::run_map_phase_advance(ctx->mphase_dev, mq, len, (long long)ctx->nx * ctx->ny, ctx->stream);
          }));
      }
      ctx->mphase_live = true;
      ctx->map_zp = ctx->z;
      ctx->map_cur = -1;
    }
  } else {
    for (int seg = 0; seg < nseg; ++seg) {
      BR_CK(cudaMemcpyAsync(ctx->adj_ckpt + (size_t)seg * ctx->nf * n, ctx->state, sizeof(float2) * ctx->nf * n,
                            cudaMemcpyDeviceToDevice, ctx->stream));
      s = brahms_propagate(ctx, std::min(K, nz - seg * K), dz);
      if (s != BRAHMS_OK) return s;
    }
  }
  s = finish_with_check(ctx);
  if (s != BRAHMS_OK) return s;
  double j = 0.0;
  for (int f = 0; f < ctx->nf; ++f) j += weights[f] * ctx->energy_host[f];
  if (J) *J = j;
  ctx->adj_gen = ctx->gen;
  ctx->adj_ready = true;
  return BRAHMS_OK;
}

brahms_status brahms_adjoint_backward(brahms_ctx* ctx, double gscale, double* grad_phi, double* grad_dk) {
  if (!ctx) return BRAHMS_E_ARG;
  if (!ctx->adj_ready) return fail(ctx, BRAHMS_E_STATE, "adjoint_backward without a completed adjoint_forward");
  if (ctx->adj_gen != ctx->gen)
    return fail(ctx, BRAHMS_E_STATE, "the fields, map or profile changed after adjoint_forward");
  if (!std::isfinite(gscale)) return fail(ctx, BRAHMS_E_ARG, "gscale is not finite");
  const int nz = ctx->adj_nz, K = ctx->adj_K, nseg = ctx->adj_nseg, nf = ctx->nf, nx = ctx->nx;
  const double dz = ctx->adj_dz;
  const long long n = ctx->npoints();
  const size_t sbytes = sizeof(float2) * nf * (size_t)n;
  // G = 2 w_f gscale A_f(L); the final forward state is still in ctx->state
  float sc[3] = {0.f, 0.f, 0.f};
  for (int f = 0; f < nf; ++f) sc[f] = (float)(2.0 * ctx->adj_weights[f] * gscale);
  BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_scale_fields(ctx->state, ctx->adj_g, n, nf, n, sc, ctx->stream); }));
  const brahms::XPassArgs base = xargs(ctx, brahms::XM_NL_FIRST, dz);
  brahms_status st = build_tables(ctx, dz);
  if (st != BRAHMS_OK) return st;
  auto dk_at = [&](int j) { return j < nz ? ctx->adj_dk[j] : ctx->dk; };
  // the segment's recorded states: B[j - j0] enters step j's B half step
  // (a2_j), A[j - j0] enters step j's A half step (A_j, j > j0)
  float2* recB = ctx->adj_seg;
  float2* recA = ctx->adj_seg + (size_t)K * nf * n;
  // reverse x-pass at boundary b (xa: A_b or NULL, xb: a2_{b-1} or NULL)
  auto reverse_x = [&](int b, const float2* xa, const float2* xb) -> brahms_status {
    brahms::XAdjArgs r{};
    r.g = ctx->adj_g;
    r.xa = xa;
    r.xb = xb;
    r.fstride = n;
    r.rows = (long long)ctx->ny * ctx->nt;
    r.tw = ctx->twx;
    r.from_k = b < nz ? 1 : 0;
    r.to_k = b > 0 ? 1 : 0;
    r.h = 0.5 * dz;
    for (int f = 0; f < nf; ++f) r.kh[f] = base.kh[f];
    if (xa) {
      r.phiA = ctx->adj_phis[b];
      r.dkA = dk_at(b);
    }
    if (xb) {
      r.dkB = dk_at(b - 1);
      r.phiB = ctx->adj_phis[b - 1] + r.dkB * 0.5 * dz;
    }
    r.partial = ctx->adj_part;
    r.ny = ctx->ny;
    if (ctx->have_map) {
      // stage factors of step b-1's B half and step b's A half (distances from z = 0)
      r.emap = ctx->emap_dev;
      const brahms_status sm = adj_map_tables(ctx, b - 1, b, b > 0 ? ctx->adj_phis[b - 1] : 0.0,
                                              b > 0 ? dk_at(b - 1) : 0.0, ctx->adj_phis[b], dk_at(b), dz);
      if (sm != BRAHMS_OK) return sm;
    }
    long long ncta = 0;
    BR_CK(launch(ctx, 0, 1, [&] { return brahms::run_xpass_adjoint(nx, nf, r, &ncta, ctx->stream); }));
    double* sA = xa ? ctx->adj_sens + (size_t)b * 6 : nullptr;
    double* sB = xb ? ctx->adj_sens + (size_t)(b - 1) * 6 + 3 : nullptr;
    BR_CK(launch(ctx, 4, 1, [&] { return brahms::run_sens_boundary(ctx->adj_part, ncta, sA, sB, ctx->stream); }));
    return BRAHMS_OK;
  };
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int j0 = seg * K, j1 = std::min(nz, j0 + K);
    // recompute the segment from its checkpoint, recording a2_j and A_j
    // (already recorded by a forward that stored every step)
    if (!ctx->adj_store_all) {
      BR_CK(cudaMemcpyAsync(ctx->adj_work, ctx->adj_ckpt + (size_t)seg * nf * n, sbytes, cudaMemcpyDeviceToDevice,
                            ctx->stream));
      brahms_status s2 = record_steps(ctx, ctx->adj_work, j0, j1, dz, recB, recA);
      if (s2 != BRAHMS_OK) return s2;
    }
    // reverse through boundaries j1 .. j0 + 1, each followed by the linear
    // adjoint of the step before it
    for (int b = j1; b > j0; --b) {
      const float2* xa = b == nz ? nullptr
                                 : (b == j1 ? ctx->adj_ckpt + (size_t)(seg + 1) * nf * n
                                            : recA + (size_t)(b - j0) * nf * n);
      const float2* xb = recB + (size_t)(b - 1 - j0) * nf * n;
      brahms_status s2 = reverse_x(b, xa, xb);
      if (s2 != BRAHMS_OK) return s2;
      s2 = linear_yty(ctx, ctx->adj_g, true);
      if (s2 != BRAHMS_OK) return s2;
    }
  }
  // boundary 0: the reverse of step 0's A half step, back to real space
  {
    brahms_status s2 = reverse_x(0, ctx->adj_ckpt, nullptr);
    if (s2 != BRAHMS_OK) return s2;
  }
  // mismatch gradient from the stage sensitivities
  std::vector<double> S((size_t)nz * 6);
  BR_CK(cudaMemcpyAsync(S.data(), ctx->adj_sens, sizeof(double) * S.size(), cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<double> acc;
  if (grad_phi && ctx->adj_has_phi) {
    // dJ/dphi_p = -(1/nt) sum_{x,y} Im(conj(G^_m) A^_m), m = (p - nt/2) mod nt
    const int pf = ctx->adj_phi_field;
    float2* gw = ctx->adj_work;
    float2* aw = ctx->adj_work + n;
    BR_CK(cudaMemcpyAsync(gw, ctx->adj_g + (size_t)pf * n, sizeof(float2) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    BR_CK(cudaMemcpyAsync(aw, ctx->adj_ckpt + (size_t)pf * n, sizeof(float2) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    brahms::AxisArgs at = aargs(ctx, 2, false);
    at.data = ctx->adj_work;
    at.ntiles = 2LL * ctx->ny * at.xtiles;  // the two copies
    BR_CK(launch(ctx, 2, 1, [&] { return brahms::run_axis_fft(ctx->nt, 2, false, at, ctx->stream); }));
    BR_CK(launch(ctx, 4, 1, [&] {
      return brahms::run_phase_grad(gw, aw, (long long)ctx->nx * ctx->ny, ctx->nt, ctx->adj_acc, ctx->stream);
    }));
    acc.resize(ctx->nt);
    BR_CK(cudaMemcpyAsync(acc.data(), ctx->adj_acc, sizeof(double) * ctx->nt, cudaMemcpyDeviceToHost, ctx->stream));
  }
  BR_CK(cudaStreamSynchronize(ctx->stream));
  if (grad_dk) {
    const double offA[3] = {0.0, 0.25 * dz, 0.5 * dz};
    const double offB[3] = {0.5 * dz, 0.75 * dz, dz};
    double later = 0.0;
    for (int j = nz - 1; j >= 0; --j) {
      double v = dz * later, tot = 0.0;
      for (int k = 0; k < 3; ++k) {
        v += S[j * 6 + k] * offA[k] + S[j * 6 + 3 + k] * offB[k];
        tot += S[j * 6 + k] + S[j * 6 + 3 + k];
      }
      grad_dk[j] = v;
      later += tot;
    }
  }
  if (grad_phi) {
    const int nt = ctx->nt;
    for (int m = 0; m < nt; ++m) grad_phi[(m + nt / 2) % nt] = acc.empty() ? 0.0 : -acc[m] / (double)nt;
  }
  return BRAHMS_OK;
}

}  // extern "C"
