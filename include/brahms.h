/*
 * brahms.h -- C ABI of the GB300 split-step solver for the coupled chi(2)
 * three-wave-mixing equations in (3+1)D.
 *
 * The solver advances the slowly varying envelopes A_f(x, y, tau) of two
 * (degenerate SHG: SH, F) or three (p, s, i) fields along z with the
 * symmetric split step of Sec. 3.1 (Eq. expon):
 *     A(z+dz) = N(dz/2) IDFT3{ P(dz) DFT3{ N(dz/2) A(z) } },
 * where N is one classical RK4 step over dz/2 of the coupling terms of
 * Eqs. CEp/CEs/CEi (Sec. 2) and P is the linear propagator of Eqs. dispOp and
 * diffOp.  Conventions fixed by this library where the paper is silent:
 *   - diffraction enters as +(i/2k) transverse Laplacian (the sign that the
 *     paper's focused Gaussian beam, Eq. gaussianbeam, solves);
 *   - third-order dispersion is the unitary -[... - (k3/6) d^3/dtau^3];
 *   - two-field SHG: dA_SH/dz = i (kappa_SH/2) A_F^2 e^{-i Phi},
 *                    dA_F/dz  = i kappa_F A_SH A_F^* e^{+i Phi};
 *   - Phi(z) is the integral of Delta k; the first RK4 half step spans
 *     [z_j, z_j+dz/2], the second [z_j+dz/2, z_j+dz];
 *   - grid x_j = (j - N/2) dx, angular frequencies 2 pi fftfreq(N, d) with
 *     the Nyquist bin negative, forward DFT e^{-2 pi i m n/N}.
 *
 * Layout of every field buffer: complex [nt][ny][nx], x fastest (Sec. 4.1,
 * the IDX(x, y, tau) ordering), interleaved (re, im).  Units are SI.
 *
 * Errors: no call aborts; each returns a brahms_status and stores a message
 * retrievable with brahms_last_error(ctx).  Calls on one context are not
 * thread-safe.  Device work is enqueued on the context's CUDA stream.
 */
#ifndef BRAHMS_H
#define BRAHMS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BRAHMS_OK = 0,
  BRAHMS_E_ARG = 1,       /* invalid argument (null pointer, bad count, non-finite value) */
  BRAHMS_E_SIZE = 2,      /* grid length not supported (must be one of the FFT lengths) */
  BRAHMS_E_CUDA = 3,      /* a CUDA runtime call failed */
  BRAHMS_E_OOM = 4,       /* device allocation failed or workspace too small */
  BRAHMS_E_NONFINITE = 5, /* fields became non-finite: dz too large (Sec. 3.2) */
  BRAHMS_E_TIMEOUT = 6,   /* a bounded device-side wait expired */
  BRAHMS_E_STATE = 7      /* call out of order (e.g. propagate before set_fields) */
} brahms_status;

enum { BRAHMS_C64 = 0, BRAHMS_C128 = 1 };

/* Per-field linear coefficients, SI (Eqs. dispOp, diffOp; kappa = 2 pi d_eff/(n lambda)). */
typedef struct {
  double lambda; /* vacuum wavelength [m] */
  double n;      /* refractive index */
  double delta;  /* group-velocity mismatch 1/v_s - 1/v_f [s/m] */
  double k2;     /* group-velocity dispersion [s^2/m] */
  double k3;     /* third-order dispersion [s^3/m] */
  double rho;    /* walk-off angle [rad] */
  double alpha;  /* linear loss [1/m] */
} brahms_field_params;

typedef struct brahms_ctx brahms_ctx;

/* Bytes of device workspace a context of this shape needs (fields, tables,
 * reduction partials).  Pass this much to brahms_init_grid, or NULL there to
 * let the library allocate it.  Returns E_SIZE / E_ARG for bad shapes. */
brahms_status brahms_workspace_size(int nx, int ny, int nt, int nfields, size_t* bytes);

/* Create a context.  nx, ny, nt: grid lengths, each one of 2,4,...,4096 or
 * 3*2^k for 6 <= 3*2^k <= 768; ny and nt may also be 1 (a 1D transverse
 * grid, or a cw field with no tau extent: its linear step is the (kx, ky)
 * multiply alone); else E_SIZE.  dx, dy [m], dt [s]: spacings > 0.
 * nfields: 2 (SH, F) or 3 (p, s, i); fp: nfields coefficient records.
 * d_eff [m/V]; dk [1/m]: constant mismatch Delta k = k_p - k_s - k_i (Eq. mismatch).
 * workspace: device memory of at least brahms_workspace_size() bytes, 256-byte
 * aligned, owned by the caller and kept alive until brahms_free; or NULL.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * On success *out owns the context; free it with brahms_free. */
brahms_status brahms_init_grid(brahms_ctx** out, int nx, int ny, int nt, double dx, double dy, double dt,
                               int nfields, const brahms_field_params* fp, double d_eff, double dk,
                               void* workspace, size_t workspace_bytes, void* cuda_stream);

/* Copy the initial envelopes in.  fields: nfields pointers, each to nt*ny*nx
 * complex values of dtype BRAHMS_C64 (float pairs) or BRAHMS_C128 (double
 * pairs), on the device if on_device != 0 else in host memory.  Resets z and
 * Phi to zero.  Host copies are complete when the call returns; device copies
 * are ordered on the context stream.  Non-finite host input gives E_ARG. */
brahms_status brahms_set_fields(brahms_ctx* ctx, const void* const* fields, int dtype, int on_device);

/* Piecewise mismatch profile: step j (counted from the last set_fields) uses
 * dk[j] for j < n and the constant dk afterwards; n = 0 clears it.  The
 * library copies the array. */
brahms_status brahms_set_dk_profile(brahms_ctx* ctx, const double* dk, int n);

/* Advance nz >= 0 split steps of length dz > 0 [m] (Sec. 3.1).  Asynchronous:
 * work is enqueued on the context stream; z and Phi accumulate in the
 * context.  A non-finite result is reported by the next synchronising call
 * (brahms_sync, brahms_get_fields, brahms_energy) as E_NONFINITE. */
brahms_status brahms_propagate(brahms_ctx* ctx, int nz, double dz);

/* Copy the current envelopes out (same conventions as set_fields); waits
 * for the stream. */
brahms_status brahms_get_fields(brahms_ctx* ctx, void* const* out, int dtype, int on_device);

/* Per-field pulse energy E_f = 1/2 c eps0 n_f sum |A_f|^2 dx dy dtau [J]
 * (Sec. 6, the power integral over tau) and photon number E_f/(hbar w_f)
 * (photons may be NULL).  FP64 accumulation; waits for the stream; returns
 * E_NONFINITE if any field is not finite. */
brahms_status brahms_energy(brahms_ctx* ctx, double* energy_j, double* photons);

/* Wait for the context stream; reports CUDA errors and E_NONFINITE. */
brahms_status brahms_sync(brahms_ctx* ctx);

/* Diagnostic: apply the unnormalised forward 3D DFT (direction -1) or the
 * normalised inverse (direction +1) to the state in place. */
brahms_status brahms_transform(brahms_ctx* ctx, int direction);

/* Transverse mismatch map (the mismatch field of a fan-out grating or of a
 * static dephasing profile): dk_map[ny][nx] in 1/m, x fastest, is added to
 * every step's Delta k.  The coupling phase is the integral of the mismatch
 * from the last brahms_set_fields (z = 0):
 *   Phi(x, y, z) = Phi_j + Delta k_j (z - z_j) + int_0^z dk_map(x, y, z') dz',
 * which for a map set before the run is Phi_j + Delta k_j (z - z_j) +
 * dk_map(x, y) z.  A map set between brahms_propagate calls applies from the
 * current z on, and the phase stays continuous there.  The library copies
 * the map; NULL removes it (and any z-segments, below).  E_ARG for non-finite
 * entries.  The adjoint propagates and differentiates under the map (the map
 * itself is not a parameter). */
brahms_status brahms_set_dk_map(brahms_ctx* ctx, const double* dk_map);

/* A mismatch map that changes along z (e.g. the temperature of a crystal
 * whose heat load varies along the beam, Sec. 4.1): nseg >= 1 segments
 * separated by the nseg - 1 distances z_edges [m] from z = 0 (finite,
 * positive, increasing; NULL when nseg == 1), maps[nseg][ny][nx] in 1/m.
 * Step j (from z_j to z_j + dz) takes the map of the segment that holds its
 * midpoint z_j + dz/2, so a segment edge acts at the step boundary nearest
 * to it; the phase is the integral above, continuous at every edge.  maps ==
 * NULL sets the segments with zero maps (the segments of the thermal model
 * alone).  The segmentation also divides the thermal model's heat load
 * (below); a change of segments drops the loads accumulated so far.  nseg == 1
 * is brahms_set_dk_map.  E_ARG for nseg outside 1..4096, bad edges or
 * non-finite maps; E_OOM if the segment maps (2 nseg ny nx doubles) cannot be
 * allocated.  The adjoint takes up to 16 segments (E_STATE beyond). */
brahms_status brahms_set_dk_map_z(brahms_ctx* ctx, int nseg, const double* z_edges, const double* maps);

/* Diagnostics of the current fields (the Sec. 6 power formula resolved in
 * tau or Omega); the state is not modified.  Each output holds nfields * nt
 * doubles, [f][k], and may be NULL:
 *   power[f][k]    = 1/2 c eps0 n_f dx dy sum_{x,y} |A_f(x, y, tau_k)|^2   [W]
 *   spectrum[f][m] = 1/2 c eps0 n_f dx dy (dt / nt) sum_{x,y} |DFT_tau A_f|^2 (m)
 *                    [J per bin of width 2 pi / (nt dt)], m in FFT order
 *                    (Omega_m = 2 pi fftfreq(nt, dt)[m], the Nyquist bin negative).
 * sum_k power dt and sum_m spectrum both equal the field energy.  Sums are
 * FP64 (the spectrum's transform is FP32).  Waits for the stream. */
brahms_status brahms_diagnostics(brahms_ctx* ctx, double* power, double* spectrum);

/* Thermal model (Sec. 4.1: the steady-state heat equation lap T = -Q / kappa
 * solved on the fields' grid, and the temperature dependence of the phase
 * mismatch).  The heat load is kept per z-segment of the context (one
 * segment unless brahms_set_dk_map_z set several).  Four calls:
 *
 * brahms_heat_accumulate_segment adds weight * Q(x, y) of the current fields
 * to segment's heat load [W/m^3], Q the absorbed optical power density
 *   Q = sum_f alpha_f I_f,  I_f = 1/2 c eps0 n_f |A_f|^2,
 * alpha_f the intensity absorption of field f (its brahms_field_params
 * alpha, the same loss the linear step applies).  For nt > 1 the pulses are
 * time-averaged: Q = rep_rate * sum_f alpha_f sum_tau I_f dt (rep_rate in Hz,
 * >= 0); for nt == 1 (cw) rep_rate is ignored.  Sampling the fields at
 * several z within a segment and choosing the weights of a quadrature rule
 * (summing to one) gives the segment's z-averaged load.  Asynchronous; FP64
 * accumulation.  E_STATE without fields, E_ARG for a segment outside
 * 0..nseg-1, a negative rep_rate or non-finite arguments.
 * brahms_heat_accumulate adds to the segment that holds the current
 * distance z (the segment that starts at z when z is on an edge).
 *
 * brahms_heat_set replaces the loads with q[nseg][ny][nx] (host, W/m^3,
 * x fastest; any finite values, negative ones being heat sinks); NULL zeroes
 * them.
 *
 * brahms_thermal_map solves, in FP64, for every segment the transverse heat
 * equation
 *   -kappa_th (d_xx + d_yy) T_s = Q_s
 * with the 5-point stencil on the fields' (x, y) grid and T = 0 (the mount
 * temperature) half a cell outside the window on every side, i.e. on the
 * crystal's side faces at x_{-1/2} and x_{nx-1/2}.  With insulated end faces
 * and one segment this is the equation of the z-averaged temperature rise
 * under the z-averaged load; with several, each segment's temperature under
 * its own load, heat flow along z between segments neglected (a load that
 * changes along z over lengths well above the beam width).  An axis of length
 * 1 is invariant (no derivative along it).  The solve is direct
 * (sine-transform diagonalisation).  It installs dk_map_s = M_s + dkdT * T_s
 * as the mismatch map of segment s, M_s the map last given to
 * brahms_set_dk_map or brahms_set_dk_map_z (a fan-out grating, say; zero if
 * none), from the current z on (the phase stays continuous); a later
 * brahms_set_dk_map replaces both terms, brahms_set_dk_map(ctx, NULL)
 * removes them.  If temperature is not NULL, it copies T [K above the mount,
 * nseg*ny*nx doubles, x fastest] to it.  kappa_th [W/(m K)] must be > 0,
 * dkdT [1/(m K)] finite.  E_STATE if a segment has no load accumulated or
 * set.  E_NONFINITE if a load or a temperature is not finite: the thermal
 * maps are then not installed and the maps in effect become those of
 * brahms_set_dk_map / brahms_set_dk_map_z (none if none).  Waits for the
 * stream. */
brahms_status brahms_heat_accumulate(brahms_ctx* ctx, double rep_rate, double weight);
brahms_status brahms_heat_accumulate_segment(brahms_ctx* ctx, int segment, double rep_rate, double weight);
brahms_status brahms_heat_set(brahms_ctx* ctx, const double* q);
brahms_status brahms_thermal_map(brahms_ctx* ctx, double kappa_th, double dkdT, double* temperature);

/* Current propagation distance [m] and accumulated mismatch phase [rad]. */
brahms_status brahms_get_z(const brahms_ctx* ctx, double* z, double* phi);

/* Per-kernel timing with CUDA events on the context stream.  enable != 0
 * starts recording (and clears previous records): enable == 1 brackets every
 * launch, enable = k > 1 every k-th launch of each kernel kind (the events
 * cost about 2 us of device time each); enable == 0 stops.  With
 * ms/launches non-NULL the accumulated device time [ms] and count of the
 * timed launches of each kernel kind (0 x-pass, 1 y-pass forward, 2 tau-pass,
 * 3 y-pass inverse, 4 other) are written to the first nkinds entries; this
 * waits for the stream. */
brahms_status brahms_timing(brahms_ctx* ctx, int enable, double* ms, long long* launches, int nkinds);

/* Implementation options; every setting computes identical numbers.
 * BRAHMS_OPT_FIELD_STREAMS: 1 runs each field's y-forward, tau-propagator
 * and y-inverse of a step on a stream of its own (created by the library),
 * each field's y-forward starting after the previous field's, so that
 * DRAM-bound and compute-bound passes of different fields overlap; the
 * x-pass, which couples the fields, waits for all of them on the context
 * stream.  0 (the default) runs every pass on the context stream.  Measured
 * on GB300: 5 % faster per step on 128x128x256 with three fields, slower on
 * two-field and small grids.  Per-kernel timing with field streams measures
 * kernels that may share the GPU.
 * BRAHMS_OPT_TMA_TAU: value 16 or 8 makes the
 * tau-pass of brahms_propagate a persistent kernel that stages tiles of that
 * many x columns through shared memory with double-buffered TMA copies; 1
 * makes it a persistent kernel with two CTAs per SM, each prefetching its
 * next 16-column tile with a TMA copy while it transforms the current one
 * (its FFT exchanges go through half the shared memory, one real component
 * at a time).  Both need nt in {256, 512} and nx >= 16, else E_SIZE; both
 * compute the plain tau-pass's numbers and measured slower on GB300.  0 (the
 * default) keeps the plain tau-pass (and turns the field streams off while
 * set).
 * BRAHMS_OPT_TMA_WAIT_US: the limit, in microseconds (0 .. 2000000, default
 * 2000000 = 2 s), of each wait of the TMA tau-pass for a tile's copy; 0
 * gives up at the first check that finds the copy unfinished.  When a
 * wait runs out the kernel lets its copies in flight land (waiting at most
 * 2 s more), leaves its remaining tiles untransformed and returns; the next
 * synchronising call reports E_TIMEOUT and the fields must be set again.
 * (A short limit makes the waits run out on purpose: the way to test that
 * error path without hanging the GPU.)
 * E_ARG for an unknown option or value.  brahms_get_option returns the
 * current value or -1. */
enum { BRAHMS_OPT_TMA_TAU = 1, BRAHMS_OPT_FIELD_STREAMS = 2, BRAHMS_OPT_TMA_WAIT_US = 3 };
brahms_status brahms_set_option(brahms_ctx* ctx, int option, int value);
int brahms_get_option(const brahms_ctx* ctx, int option);

/* Number of kernel launches this context has enqueued since creation. */
long long brahms_launch_count(const brahms_ctx* ctx);

/* ------------------------------------------------------------------------
 * Adjoint: gradients of J = sum_f w_f sum_points |A_f(L)|^2 (e.g. the SHG
 * efficiency with w_SH = n_SH / (n_F sum |A_F(0)|^2), w_F = 0) with respect to
 * a spectral phase phi applied at z = 0 to one field,
 *   A <- IDFT_tau( e^{i phi(Omega)} DFT_tau A ),  phi in centred order
 *   (phi[p] belongs to Omega = 2 pi (p - nt/2) / (nt dt)),
 * and to the per-step mismatch profile dk[0..nz-1].  The gradient is the
 * exact adjoint of the discrete propagation (the paper has no adjoint):
 * the linear step reversed as IDFT3(conj(P) DFT3), each RK4 half step in
 * reverse mode with its stages recomputed, and the mismatch through the RK4
 * stage phases Phi(z) = Phi_j + dk_j (z - z_j).  Memory: the forward keeps a
 * checkpoint every K steps (K = ceil(sqrt(nz)) when checkpoint_interval == 0,
 * K = checkpoint_interval when > 0) and the backward recomputes each segment,
 * recording the 2K states entering its steps' two half steps; the library
 * allocates (ceil(nz/K) + 2K + 2) field states plus small tables for it.
 * checkpoint_interval < 0: the forward records all 2 nz such states itself
 * (2 nz + 3 field states; on a large-memory GPU usually affordable) and the
 * backward recomputes nothing.  The gradient is bit-identical either way
 * under a map constant in z.  Under a map that changes along z
 * (brahms_set_dk_map_z, up to 16 segments) the recomputation and the reverse
 * sweep form each step's map phase from the segments' step counts, which
 * agrees with the forward's running sum to rounding, so the checkpointed and
 * the recorded forms then agree to rounding.
 * ---------------------------------------------------------------------- */

/* Set the fields (as brahms_set_fields), apply the phase (phi may be NULL),
 * propagate nz steps of dz with the profile dk, keep checkpoints, and return
 * J (weights: nfields entries).  Leaves the fields at z = nz dz.  Waits.
 * E_SIZE on grids with ny = 1 or nt = 1; E_STATE under a map of more than 16
 * z-segments. */
brahms_status brahms_adjoint_forward(brahms_ctx* ctx, const void* const* fields, int dtype, int on_device,
                                     const double* phi, int phi_field, const double* dk, int nz, double dz,
                                     const double* weights, int checkpoint_interval, double* J);

/* Reverse sweep for the last brahms_adjoint_forward: writes gscale * dJ/dphi
 * (nt entries, centred order; zeros if no phase was applied) and
 * gscale * dJ/d dk_j (nz entries); either pointer may be NULL.  May be called
 * again for the same forward (another gscale).  E_STATE if the last
 * brahms_adjoint_forward failed or never ran, or if any call changed the
 * fields, the mismatch map or the profile since it returned
 * (brahms_set_fields, brahms_propagate, brahms_transform, brahms_set_dk_map,
 * brahms_set_dk_profile, brahms_thermal_map): the reverse sweep reads the
 * forward's final fields and map, so it runs only on those. */
brahms_status brahms_adjoint_backward(brahms_ctx* ctx, double gscale, double* grad_phi, double* grad_dk);

/* Weights that make J of brahms_adjoint_forward the SHG efficiency
 * eta = E_SH(L) / E_F(0) of the current two fields (SH, F), as set by
 * brahms_set_fields with the input: w_SH = n_SH / (n_F sum |A_F|^2),
 * w_F = 0 (the common factor 1/2 c eps0 dx dy dtau of both energies cancels;
 * a spectral phase on F keeps E_F(0)).  The sum takes the FP32 squares of
 * the complex64 field into FP64 (relative error ~1e-9); waits.
 * weights: 2 doubles.  E_ARG for three fields or a zero fundamental,
 * E_STATE without fields. */
brahms_status brahms_shg_efficiency_weights(brahms_ctx* ctx, double* weights);

/* ------------------------------------------------------------------------
 * Batched form (two-field SHG sweeps): many independent simulations of
 * uneven grids, mismatch and crystal length, run by one CUDA graph launch.
 * Each instance follows the same split step as brahms_propagate (constant dk
 * per instance, starting at z = 0 with Phi = 0) and gives its numbers bit for
 * bit.  Two forms (brahms_batch_set_mode):
 *   grouped (1): the instances of one grid shape are stored one after
 *     another and every pass of all of them is one launch of the
 *     single-instance kernels; each shape's launches run on a stream of
 *     their own, so passes of different shapes overlap.  Any grid the
 *     single-instance path supports with ny, nt >= 2 can join.
 *   persistent (2): one persistent cooperative kernel with a work queue of
 *     (instance, pass, tile range) items and per-instance bounded pass
 *     barriers; shapes (nx = ny, nt) in (32,64), (64,128), (96,192),
 *     (128,256) only.
 *   automatic (0, the default): the grouped form until brahms_batch_tune
 *     has timed both and kept the faster.
 * The batch allocates its own device memory (state and tables per instance,
 * regrouped by shape at the first run after instances were added).  Work is
 * enqueued on cuda_stream (NULL = legacy default stream).
 * ---------------------------------------------------------------------- */
typedef struct brahms_batch brahms_batch;

/* Create an empty batch. */
brahms_status brahms_batch_create(brahms_batch** out, void* cuda_stream);

/* Add one SHG instance (fields SH, F; fp holds 2 records) that will run nz
 * steps of dz [m]; *index receives its position.  Tables are built here.
 * E_SIZE for grid lengths the single-instance path does not support, for
 * ny or nt = 1, and, once the persistent form is set, for a shape outside
 * its four. */
brahms_status brahms_batch_add(brahms_batch* b, int nx, int ny, int nt, double dx, double dy, double dt,
                               const brahms_field_params* fp, double d_eff, double dk, int nz, double dz,
                               int* index);

/* Copy instance `index`'s initial envelopes in: 2 pointers to nt*ny*nx
 * complex64 values, device (on_device != 0) or host memory (copied before
 * return).  Every instance needs fields before brahms_batch_run. */
brahms_status brahms_batch_set_fields(brahms_batch* b, int index, const void* const* fields, int dtype,
                                      int on_device);

/* Tile schedule of the persistent form for one of its shapes (0..3 in the
 * order above): CTA tiles per work item for the x-, y- and tau-passes
 * (1..64). */
brahms_status brahms_batch_set_granularity(brahms_batch* b, int shape, int gx, int gy, int gt);

/* Autotune: each trial times the whole batch with every instance capped at
 * tune_steps steps (fields restored afterwards).  The grouped form is timed
 * once; the persistent form, where its shapes allow it, is searched: per
 * shape the tiles per item (one of 1, 2, 4, 8, 16 for all three passes,
 * then each pass's doubled or halved while that helps, within 1..64), then
 * CTAs per SM (1, 2).  In the automatic mode the faster form is kept.
 * Waits for the stream.  *best_ms (nullable) receives the best capped run
 * time. */
brahms_status brahms_batch_tune(brahms_batch* b, int tune_steps, double* best_ms);

/* The current schedule of one shape. */
brahms_status brahms_batch_get_schedule(const brahms_batch* b, int shape, int* gx, int* gy, int* gt,
                                        int* ctas_per_sm);

/* Form of the batch: 0 automatic, 1 grouped, 2 persistent (E_SIZE if an
 * instance's shape is not one of the persistent form's); E_ARG otherwise.
 * brahms_batch_get_mode returns the form the next run uses (1 or 2). */
brahms_status brahms_batch_set_mode(brahms_batch* b, int mode);
int brahms_batch_get_mode(const brahms_batch* b);

/* Advance every instance through all of its nz steps (z = 0 to nz dz) in one
 * graph launch.  Asynchronous. */
brahms_status brahms_batch_run(brahms_batch* b);

/* Wait for the stream; E_TIMEOUT if the persistent kernel gave up waiting
 * for a pass of some instance (its bounded waits expired).  The instances'
 * fields are then partly advanced: set them again before the next run. */
brahms_status brahms_batch_sync(brahms_batch* b);

/* Limit [s] of each bounded wait of the persistent kernel (a CTA waiting for
 * runnable work or for the previous pass of an instance), 0 .. 3600;
 * default 5.  On expiry the kernel records E_TIMEOUT (reported by
 * brahms_batch_sync) and every CTA returns.  (A zero limit makes the waits
 * run out on purpose: the way to test that error path without hanging the
 * GPU.)  Takes effect at the next brahms_batch_run.  E_ARG out of range. */
brahms_status brahms_batch_set_timeout(brahms_batch* b, double seconds);

/* Copy instance `index`'s envelopes out (2 pointers, complex64); waits. */
brahms_status brahms_batch_get_fields(brahms_batch* b, int index, void* const* out, int dtype, int on_device);

/* Instances, persistent grid size (0 in the grouped form), threads per CTA
 * of the persistent kernel, kernel launches made by the runs so far. */
brahms_status brahms_batch_info(const brahms_batch* b, int* ninstances, int* grid, int* threads,
                                long long* launches);

/* Release the batch and its device memory. */
void brahms_batch_free(brahms_batch* b);

/* Last error message of the batch. */
const char* brahms_batch_last_error(const brahms_batch* b);

/* Allocation-free energy of caller-owned device fields.  (The paper has no
 * counterpart; this serves callers that cannot let the library allocate
 * device memory: hosts whose GPU memory is all owned by another allocator,
 * plugin environments that forbid a library's own cudaMalloc, and tight
 * loops that cannot afford the device-wide synchronisation cudaMalloc and
 * cudaFree may cause.)  Computes the same per-field energy as brahms_energy,
 * E_f = 1/2 c eps0 n_f sum |A_f|^2 dx dy dtau [J], without a context and
 * without allocating anything.
 *   fields: nfields device pointers, each to nt*ny*nx complex64 [nt][ny][nx];
 *   fp: nfields records (only n is used); energy_j_dev: device array of
 *   nfields doubles, written on cuda_stream (NULL = legacy default stream).
 * The partial sums live in one fixed 24 KiB device array inside the library
 * (3 fields x 1024 partials), which every GPU that loads the library keeps
 * until the process exits.  Limits: 1 <= nfields <= 3 and nx*ny*nt <= 2^40,
 * else BRAHMS_E_SIZE.  Each call writes every partial it reads, so no state
 * carries over, but all calls share that array: calls whose work overlaps on
 * the GPU (other streams, other threads) race and must be serialised by the
 * caller.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and so does the first
 * call after a cudaDeviceReset has replaced the device's context (the array
 * then lives at a new address); make those calls before any stream capture.  Returns E_ARG for NULL pointers or
 * non-positive spacings, E_CUDA if a launch fails; asynchronous otherwise. */
brahms_status brahms_energy_static(const void* const* fields, int nfields, int nx, int ny, int nt, double dx,
                                   double dy, double dt, const brahms_field_params* fp, double* energy_j_dev,
                                   void* cuda_stream);

/* Measured FP32 fused multiply-add rate of the current GPU [TFLOP/s, 2 flops
 * per FMA]: the peak that the ALU view of a kernel's roofline divides by.
 * (The paper has no counterpart; the target's roofline is HBM bandwidth, and
 * the FFT and RK4 passes are also bounded by FP32 issue, whose peak no
 * published figure gives for this GPU.)  Runs about 0.1 s of independent FMA
 * chains on every SM on cuda_stream, timed with CUDA events after a warm-up
 * launch; waits.  E_ARG for a NULL output, E_CUDA if a launch fails. */
brahms_status brahms_fp32_fma_rate(void* cuda_stream, double* tflops);

/* Measured all-to-all exchange rate [TB/s] of distributed shared memory
 * within thread-block clusters of cluster_ctas CTAs (2, 4, 8 or 16), each CTA
 * holding smem_bytes (1 KB .. 227 KB) of shared memory in cluster_ctas
 * chunks and storing chunk j into CTA j's shared memory, 200 rounds with a
 * cluster barrier after each, one resident wave of clusters; the rate counts
 * the bytes that cross between CTAs.  (The paper has no counterpart: the
 * measurement that decides whether a step keeping whole (x, y) planes of all
 * fields on chip, exchanged twice per plane through this memory, can beat
 * two more HBM passes.)  Waits.  E_SIZE if no cluster of that shape fits,
 * E_ARG for other sizes, E_CUDA if a launch fails. */
brahms_status brahms_dsmem_exchange_rate(int cluster_ctas, int smem_bytes, void* cuda_stream, double* tbps);

/* Fault injection for tests of the error paths: the next `count` device or
 * pinned-host allocations the library makes (context workspace and its
 * pinned readback word, adjoint checkpoints, thermal buffers, batch memory)
 * report failure (the calls return BRAHMS_E_OOM) without calling the CUDA
 * allocator; count 0 clears it.  Process-wide and thread-safe.  E_ARG for a
 * negative count.  brahms_pending_allocation_failures returns how many of
 * them have not been consumed yet. */
brahms_status brahms_fail_next_allocations(int count);
int brahms_pending_allocation_failures(void);

/* Release the context and any memory the library allocated for it. */
void brahms_free(brahms_ctx* ctx);

/* Last error message of ctx ("" if none); a static string if ctx is NULL. */
const char* brahms_last_error(const brahms_ctx* ctx);

/* Name of a status code. */
const char* brahms_status_string(brahms_status s);

#ifdef __cplusplus
}
#endif

#endif /* BRAHMS_H */
