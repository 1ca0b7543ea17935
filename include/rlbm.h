/*
 * rlbm.h -- C ABI of the GB300 (sm_103a) relativistic lattice Boltzmann library.
 *
 * The library advances the relativistic lattice Boltzmann method for a massless
 * two-dimensional fluid of M. Watson, "Turbulence in two-dimensional relativistic
 * hydrodynamic systems with a lattice Boltzmann model" (arXiv 2205.04658):
 *
 *   f*_0 = f_eq(eps_init, u_init)                (Sec. "The Standard/Classical LBM",
 *   repeat:                                        enumerated procedure, item 1)
 *     f_n = stream(f*_n)     bilinear pull of the off-lattice momenta, bounce-back at
 *                            solid cells (Sec. "Boltzmann to Lattice Boltzmann";
 *                            Part II "Model and Methods")
 *     T^{mu nu}(f_n) -> Landau matching u_mu T^{mu nu} = eps u^nu -> eps, u^mu,
 *                       T = (pi^2 eps / 3)^{1/4}, tau_R = 5 (eta/s) / T
 *                       (Sec. "Relativistic Lattice Boltzmann"; Sec. "Boltzmann to
 *                       Lattice Boltzmann")
 *     f*_{n+1} = f_n + dt/tau_R (u^0 - v.u)(f_eq - f_n) + dt S_n
 *                       (Eq. boltzmanneq_rel; Eq. forceTerm and App. B for S_n)
 *
 * "The state after n steps" is f_n = stream(f*_n); rlbm_moments reports its moments.
 *
 * Conventions for every entry point:
 *   - Nothing aborts, throws or prints.  A bad argument returns RLBM_E_INVAL and sets
 *     the message returned by rlbm_last_error.
 *   - Device memory is owned by the caller: rlbm_init receives one workspace of at
 *     least rlbm_query_workspace bytes (256-byte aligned) and never frees it.  The
 *     library owns only its host-side context.  All host arrays passed in are copied
 *     before the call returns.
 *   - Work is queued on the CUDA stream given to rlbm_init (0 = legacy default
 *     stream).  rlbm_step is asynchronous; rlbm_moments, rlbm_spectrum, rlbm_sync and
 *     rlbm_get_state synchronise that stream and report conditions the kernels
 *     latched in a device error word (RLBM_E_UNSTABLE, RLBM_E_UNPHYSICAL,
 *     RLBM_E_TIMEOUT).  After such an error the context accepts only rlbm_free.
 *   - Lattice arrays are row-major with x fastest: index = y * nx + x.
 *   - The workspace is reused by every call on the context; calls on one context
 *     must not overlap from several host threads.
 */
#ifndef RLBM_H
#define RLBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RLBM_API __attribute__((visibility("default")))
#else
#define RLBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlbm_ctx rlbm_ctx;  /* opaque; created by rlbm_init, destroyed by rlbm_free */

typedef enum {
  RLBM_OK = 0,
  RLBM_E_INVAL = 1,       /* invalid argument or configuration */
  RLBM_E_NOMEM = 2,       /* workspace too small, or host allocation failed */
  RLBM_E_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
  RLBM_E_UNSTABLE = 4,    /* a cell went non-finite, eps <= 0 or |v| >= 1 */
  RLBM_E_UNPHYSICAL = 5,  /* Landau matching found no timelike eigenvector */
  RLBM_E_TIMEOUT = 6,     /* a bounded device-side wait expired */
  RLBM_E_STATE = 7        /* the context is in an error state, or the call is out of order */
} rlbm_status;

/* Storage precision of the populations.  F64 and F32 store the normalised deviation
 * h_i = f_i / (w_i eps0) - 1 in that type and compute in it (F32 falls back to FP64
 * for the Landau solve of a cell whose |v| exceeds fp64_landau_vmax or whose FP32
 * Newton solve does not converge).  F16 and BF16 store h_i in 16 bits and compute
 * in FP32: BF16 holds h_i, F16 holds 256 h_i (the scale keeps the deviations down to
 * 2^-22 in FP16's normal range; |h_i| is held up to 255.9, and a larger value is stored
 * as that limit by the stochastic rounding, or as infinity by round to nearest, which the
 * next step reports as E_UNSTABLE).  rlbm_get_state / rlbm_set_state
 * exchange h_i itself; the scale is internal. */
typedef enum { RLBM_F64 = 0, RLBM_F32 = 1, RLBM_F16 = 2, RLBM_BF16 = 3 } rlbm_precision;

typedef struct {
  int32_t nx, ny;          /* lattice size, 8 <= nx, ny <= 32768; x is always periodic */
  int32_t walls_y;         /* 0: y periodic; 1: solid ghost rows at y = -1 and y = ny */
  int32_t vset;            /* 3: the paper's 26-direction spherical set (P = eps/3);
                              2: 8 directions on the unit circle (P = eps/2, no force) */
  int32_t precision;       /* rlbm_precision */
  int32_t rounding;        /* F16/BF16 storage: 0 = stochastic rounding (default; unbiased,
                              counter-based per seed, step and cell, so runs repeat
                              exactly), 1 = round to nearest.  Ignored for F64/F32. */
  double a, dt;            /* lattice spacing and time step; requires 0 < dt/a <= 1 */
  double eta_over_s;       /* > 0; tau_R = 5 (eta/s) / T (4 (eta/s) / T for vset 2) */
  double eps0;             /* > 0; reference energy density, T0 = T(eps0) */
  double body_force[2];    /* uniform force (F^x, F^y) added everywhere */
  int32_t kmin, kmax;      /* stirring shell kmin <= |k| <= kmax in integer wave-number
                              units; 0 <= kmin <= kmax < min(nx, ny) / 2 */
  double force_amp;        /* Gaussian amplitude scale of the stirring modes; 0 = off */
  uint64_t seed;           /* Philox4x32-10 key of the stirring draws */
  const uint8_t *solid;    /* host, nx*ny, nonzero = impurity cell; NULL = none */
  const double *init_eps;  /* host, nx*ny initial energy density; NULL = eps0 */
  const double *init_ux;   /* host, nx*ny initial u^x (spatial part of u^mu); NULL = 0 */
  const double *init_uy;   /* host, nx*ny initial u^y; NULL = 0 */
  double fp64_landau_vmax; /* F32/F16/BF16: |v| above which Landau runs in FP64; 0 = 0.5 */
  int32_t open_x;          /* 0 = x periodic (default); 1 = open channel (Part II, "Model and
                              Methods"): at x = 0 the populations streaming in are those of
                              the equilibrium at eps0 moving with u^x = inflow_ux, and at
                              x = nx - 1 the outflow is zero-gradient (the column beyond the
                              last one repeats it).  y stays periodic unless walls_y. */
  double inflow_ux;        /* open_x: spatial u^x of the inflow (in units of the particle
                              speed); |inflow_ux| < 1 */
  /* Strip of a larger lattice (a domain decomposition in y; see rlbm_halo_pack).
   * strip_ny_total = 0: the context is the whole lattice (the default).  Otherwise it
   * holds rows strip_y0 .. strip_y0 + ny - 1 of a lattice of strip_ny_total rows whose y
   * boundary walls_y describes (periodic, or walls below row 0 and above the last row):
   * the stirring phases and the rounding of 16-bit stores use the lattice's own rows, and
   * a face of the strip that is not a wall takes its ghost row from the neighbouring
   * strip (rlbm_halo_unpack).  kmax < min(nx, strip_ny_total) / 2.  Not with open_x. */
  int32_t strip_y0;        /* first lattice row of the strip, 0 <= strip_y0 < strip_ny_total */
  int32_t strip_ny_total;  /* rows of the whole lattice, strip_y0 + ny <= strip_ny_total; 0 = off */
  const uint8_t *strip_solid_halo; /* host, 2 * nx or NULL (= fluid): solid mask of lattice row
                              strip_y0 - 1, then of row strip_y0 + ny (rows wrap when y is
                              periodic); ignored at a face that is a wall */
} rlbm_config;

/* Device bytes the workspace must hold for this configuration (the populations,
 * two buffers of 17 planes for vset 3 or 8 for vset 2, plus tables and scratch).
 * Validates the configuration.  The paper has no counterpart (memory management). */
RLBM_API rlbm_status rlbm_query_workspace(const rlbm_config *cfg, size_t *bytes);

/* Create a context on the current CUDA device.  dev_workspace: device pointer, at
 * least rlbm_query_workspace bytes, 256-byte aligned, owned by the caller and kept
 * alive until rlbm_free.  cuda_stream: a cudaStream_t (NULL = default stream).
 * Initialises the state to f*_0 = f_eq(eps_init, u_init) (procedure item 1 of Sec.
 * "The Standard/Classical LBM") and resets the step counter to 0.  *out is NULL on
 * failure. */
RLBM_API rlbm_status rlbm_init(const rlbm_config *cfg, void *dev_workspace, size_t bytes,
                      void *cuda_stream, rlbm_ctx **out);

/* Queue nsteps >= 0 time steps (stream + moments + Landau + equilibrium + collision
 * + force, one fused kernel per step).  Step n uses the stirring draws
 * Philox4x32-10(counter = (n mod 2^32, mode, n div 2^32, 0), key = seed).  Async.
 * The 2nd .. nsteps-th launches of one call are chained to the previous step
 * (programmatic dependent launch: each waits for the previous step's writes before it
 * reads anything); the results are those of nsteps separate calls, bit for bit. */
RLBM_API rlbm_status rlbm_step(rlbm_ctx *ctx, int64_t nsteps);

/* Moments of the current state f_n: eps, u^x, u^y (host arrays of nx*ny, each may be
 * NULL; zero at solid cells) and totals (host double[4], may be NULL):
 * sum T^00, sum T^0x, sum T^0y, sum 1/2 |v|^2 over fluid cells, v = u^i / u^0.
 * Runs the streaming and Landau matching of the next step without storing it, in the
 * context's compute type: FP64 for F64; FP32 for the others, with the FP64 re-solve of
 * the step kernel and the totals' FP32 deviation sums added per block in FP64. Syncs. */
RLBM_API rlbm_status rlbm_moments(rlbm_ctx *ctx, double *eps, double *ux, double *uy, double *totals);

/* Energy spectrum of the current state's velocity v = u^i / u^0 (Sec. "Turbulence"):
 * E[n] = 1/2 sum_{k: round(|k|) = n} |v^(k)|^2 / (nx ny)^2, n = 0 .. nbins-1, integer
 * wave numbers, v^(k) = sum_x v(x) exp(-i k.x), v = 0 at solid cells.  E: host array of
 * nbins doubles.  Syncs. */
RLBM_API rlbm_status rlbm_spectrum(rlbm_ctx *ctx, int32_t nbins, double *E);

/* Energy of a band of wave vectors of the current state's velocity field (v = u^i / u^0):
 * (1/2) sum over k2lo <= k_x^2 + k_y^2 < k2hi of |v^(k)|^2 / (nx ny)^2, integer wave-number
 * indices; k2hi <= 0 means no upper bound.  With k2lo = 0 and k2hi = kmin^2 it is the mean
 * kinetic energy of the velocities filtered to the range below the stirring shell (Part I,
 * "Model and Methods": the recorded velocities are filtered to remove the driven range);
 * sqrt(2 E) is the filtered rms velocity.  Same normalisation as rlbm_spectrum (the band
 * [0, infinity) is half the mean |v|^2).  Syncs. */
RLBM_API rlbm_status rlbm_band_energy(rlbm_ctx *ctx, int64_t k2lo, int64_t k2hi, double *E);

/* Column means of the current state's velocity v = u^i / u^0 (solid cells count as 0):
 * jx[x] = (1/ny) sum_y v^x(x, y), jy likewise; host arrays of nx values (either may be NULL).
 * The current density of Part II ("Model and Methods") in units of the particle speed:
 * jx[nx - 1] at the outflow border over time gives j(t), jx over a span of columns j(x).
 * Syncs. */
RLBM_API rlbm_status rlbm_column_means(rlbm_ctx *ctx, double *jx, double *jy);

/* Copy the stored populations out or in (checkpoint / resume).  host: (planes x ny x nx)
 * values of h_i = f*_i / (w_i eps0) - 1 in double, plane order of the library's folded
 * velocity classes (rlbm_num_planes gives the count).  set_state also sets the step
 * counter.  Both sync.  The paper has no counterpart (it records moments only). */
RLBM_API rlbm_status rlbm_get_state(rlbm_ctx *ctx, double *host, int64_t *step);
RLBM_API rlbm_status rlbm_set_state(rlbm_ctx *ctx, const double *host, int64_t step);
RLBM_API int32_t rlbm_num_planes(const rlbm_ctx *ctx);

/* Launch shape of the fused step kernel: `ctas` persistent CTAs walk the lattice's
 * 32 x 8 tiles (0 = as many as are resident at once, the default; larger values are
 * clamped), `stages` (1 or 2; 0 keeps the current value) tiles of shared memory rotate
 * in its TMA pipeline (default 2), and `stir_rows` says where the stirring rows of a tile
 * come from: 1 = staged with the tile by TMA (default), 2 = read from global memory (less
 * shared memory per CTA, so more CTAs per SM); 0 keeps the current value.  A tuning
 * control: results do not depend on it.  The paper has no counterpart. */
RLBM_API rlbm_status rlbm_set_launch(rlbm_ctx *ctx, int32_t ctas, int32_t stages, int32_t stir_rows);

/* Autotuner: times every launch shape it knows (pipeline depth x CTA count x stirring
 * rows staged or read from global memory), `reps` launches each, chained as rlbm_step
 * chains consecutive steps, on the current state, and keeps the fastest.  The state and the step
 * counter are left as they were (the launches rewrite the next buffer only).  *ms_out
 * (may be NULL) receives the chosen shape's time per step in milliseconds.  Syncs.
 * The paper has no counterpart. */
RLBM_API rlbm_status rlbm_autotune(rlbm_ctx *ctx, int32_t reps, double *ms_out);

/* Energy spectrum of device velocity fields, allocating nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc, such as
 * code that owns all device memory through its own allocator or a fixed budget, or code
 * in a loop where cudaMalloc's implicit device-wide synchronisation would stall other
 * streams.  (rlbm_spectrum needs a context, whose workspace the caller allocates.)
 *
 * d_ux, d_uy: device arrays of nx * ny doubles (u^x, u^y, row-major, x fastest; the
 * result uses v = u^i / u^0); d_E: device array receiving nbins doubles,
 * E[n] = 1/2 sum_{round|k| = n} |v^(k)|^2 / (nx ny)^2 exactly as rlbm_spectrum.  Queued
 * on cuda_stream (NULL = default stream); no synchronisation.
 *
 * Limits: 8 <= nx, ny <= 16384, nx * ny <= 131072 (2^17) cells, 1 <= nbins <= 8200;
 * larger requests return RLBM_E_INVAL with a message in rlbm_last_error(NULL).  The
 * work buffers are one fixed array of 4 784 192 bytes (about 4.8 MB) in the library's own
 * device memory (every GPU that loads the library holds it until the process exits).  The
 * first call on each device looks up that array's device address (cudaGetSymbolAddress),
 * so make the first call on a device before any stream capture; a lookup that fails
 * returns RLBM_E_CUDA and is tried again by the next call.  A length with a prime factor
 * p above 8 is transformed by direct sums of length p (O(n p) work per row or column,
 * spread over the threads of a block): lengths with small prime factors are fastest.  All calls share the array and
 * it keeps the last call's contents (the bins are cleared at the start of each call):
 * calls that overlap on the GPU, from several streams or threads, race and must be
 * serialised by the caller. */
RLBM_API rlbm_status rlbm_spectrum_noalloc(const double *d_ux, const double *d_uy, int32_t nx, int32_t ny,
                                           int32_t nbins, double *d_E, void *cuda_stream);

/* The folded velocity classes behind the planes of rlbm_get_state / rlbm_set_state:
 * for vset 3 (17 classes) or 2 (8 classes), out[4*q + 0..3] = (v_x, v_y, v_z^2, w) of
 * class q, where w is the summed weight of the 3-D directions the class stands for.
 * Returns the class count (and writes nothing when out is NULL), or -1 for a bad vset.
 * The paper has no counterpart (a layout query). */
RLBM_API int32_t rlbm_velocity_classes(int32_t vset, double *out);

/* ---- Strips: one lattice decomposed into horizontal strips --------------------------
 * The update reads, at each cell, only the cell's own populations and those of its eight
 * neighbours (the streaming pull moves populations by at most one cell, dt/a <= 1; Sec.
 * "Boltzmann to Lattice Boltzmann", and Sec. "The Standard/Classical LBM", whose collision
 * is local).  A lattice split into strips of whole rows therefore steps exactly as one
 * lattice if, before every step, each strip's ghost rows hold its neighbours' boundary
 * rows: the populations that cross each face, one padded row per crossing plane (6 of
 * the 17 planes for vset 3, 3 of 8 for vset 2).
 *
 * Per step, for strips created with strip_ny_total > 0 (on one device or on several):
 *   rlbm_halo_pack(strip, 0, buf_lo); rlbm_halo_pack(strip, 1, buf_hi);   every strip
 *   move buf_lo of each strip to the strip below, buf_hi to the strip above (device
 *     copies on one GPU, point-to-point sends between GPUs or hosts)
 *   rlbm_halo_unpack(strip, 0, from_below); rlbm_halo_unpack(strip, 1, from_above);
 *   rlbm_step(strip, 1)
 * A face that is a wall (walls_y, at the first or last row of the lattice) is neither
 * packed for nor unpacked.  Do the exchange once after rlbm_init (before the first step)
 * and after the last step before rlbm_moments: the moments read the ghost rows too.
 * rlbm_moments reports the strip's own fields and totals (sum the totals over strips);
 * rlbm_spectrum, rlbm_band_energy, rlbm_column_means and rlbm_gradient refuse a strip
 * (RLBM_E_INVAL): they need the whole lattice.  The paper has no counterpart (its runs
 * were one lattice per process). */

/* Bytes of one face's halo message of a strip context (*bytes = 0 for a whole lattice). */
RLBM_API rlbm_status rlbm_halo_bytes(const rlbm_ctx *ctx, size_t *bytes);

/* Queue on the context's stream a copy of the strip's boundary row that a neighbour needs
 * into dev_out (device, rlbm_halo_bytes): face 0 = row 0 (planes moving down, v_y < 0), for
 * the strip below; face 1 = row ny - 1 (planes moving up), for the strip above.  Padded rows
 * of the storage type, x ghost columns included.  RLBM_E_INVAL for a whole lattice, a face
 * other than 0 or 1, or a face that is a wall. */
RLBM_API rlbm_status rlbm_halo_pack(rlbm_ctx *ctx, int32_t face, void *dev_out);

/* Queue on the context's stream the copy of a neighbour's message dev_in (device, the
 * neighbour's rlbm_halo_pack output) into this strip's ghost row: face 0 = the row below
 * row 0 (from the lower strip's face 1), face 1 = the row above row ny - 1 (from the upper
 * strip's face 0).  Same refusals as rlbm_halo_pack. */
RLBM_API rlbm_status rlbm_halo_unpack(rlbm_ctx *ctx, int32_t face, const void *dev_in);

/* ---- Batches: many lattices advanced by one persistent launch per step -------------
 * An ensemble (stirred realisations, impurity samples) of uneven sizes steps as one job:
 * each step is a single launch of the fused kernel over the tiles of all members, and
 * whole chunks of steps replay a captured CUDA graph.
 * Members are ordinary contexts (rlbm_init) that share the velocity set, storage type,
 * a, dt, eta/s, eps0, body force, stirring shell and amplitude, rounding and
 * fp64_landau_vmax; they may differ in size, walls, solids, seeds and initial fields,
 * and in their current step.  After rlbm_batch_step every member has advanced by nsteps
 * (rlbm_current_step, rlbm_moments ... work on it as usual); work of the batch is queued
 * on the batch's stream, so give the members the same stream or synchronise.  Graphs are
 * used on a non-default stream only.  The paper has no counterpart (its runs were one
 * lattice per process). */
typedef struct rlbm_batch rlbm_batch;

/* Device bytes of a batch workspace for nmembers members (member descriptors, tile and
 * work prefixes, the step counter). */
RLBM_API rlbm_status rlbm_batch_query_workspace(int32_t nmembers, size_t *bytes);

/* Create a batch over members[0 .. nmembers-1] (the contexts stay owned by the caller and
 * must outlive the batch).  dev_workspace: 256-byte aligned, caller-owned. */
RLBM_API rlbm_status rlbm_batch_init(rlbm_ctx *const *members, int32_t nmembers, void *dev_workspace,
                                     size_t bytes, void *cuda_stream, rlbm_batch **out);

/* Launch shape of the batched step kernel (as rlbm_set_launch). */
RLBM_API rlbm_status rlbm_batch_set_launch(rlbm_batch *b, int32_t ctas, int32_t stages);

/* Autotuner of the batched launch: times every launch shape it knows (pipeline depth x
 * persistent CTA count), `reps` launches each, on the members' current states without
 * advancing them, and keeps the fastest.  *ms_out (may be NULL) receives its time per
 * batched step in milliseconds.  Syncs the batch's stream.  The paper has no counterpart. */
RLBM_API rlbm_status rlbm_batch_autotune(rlbm_batch *b, int32_t reps, double *ms_out);

/* Advance every member by nsteps >= 0 steps.  Async. */
RLBM_API rlbm_status rlbm_batch_step(rlbm_batch *b, int64_t nsteps);

/* Message of the last failing call on b (or of the last failing batch call on this thread
 * when b is NULL). */
RLBM_API const char *rlbm_batch_last_error(const rlbm_batch *b);

/* Release the batch (not its workspace, not the members). */
RLBM_API void rlbm_batch_free(rlbm_batch *b);

/* ---- Stirring multipliers and the adjoint ------------------------------------------
 * The stirring of Sec. "The Driving Term" draws, at every step n, a Gaussian amplitude a_m
 * for each mode m of the shell.  Multipliers sigma_m (default 1) scale those amplitudes:
 * the force becomes sum_m sigma_m a_m (cos psi_m, sin psi_m) cos(k_m.x + phi_m).
 * The paper has no counterpart; they are the parameters of the gradient below. */

/* Number of stirring modes of the context's shell (0 without stirring); -1 if ctx is NULL. */
RLBM_API int32_t rlbm_num_modes(const rlbm_ctx *ctx);

/* Set sigma_m (host array of rlbm_num_modes(ctx) finite values, copied) for the current
 * and all later steps.  Syncs.  E_INVAL on a wrong count or a non-finite value. */
RLBM_API rlbm_status rlbm_set_mode_scale(rlbm_ctx *ctx, const double *sigma, int32_t nmodes);

/* Objective (no counterpart in the paper): the time average over the states after steps
 * s0+1 .. s0+nsteps (s0 = rlbm_current_step on entry) of the fluid-cell mean of
 * |v|^2 / 2, v = u^i / u^0 from Landau matching,
 *     J = (1 / nsteps) sum_n (1 / N_fluid) sum_x |v_n(x)|^2 / 2.
 * rlbm_gradient runs the nsteps forward steps (the context ends at s0 + nsteps, exactly as
 * after rlbm_step(ctx, nsteps)), keeping the post-collision state every `segment` steps
 * (0: ceil(sqrt(nsteps))), then the hand-written adjoint backwards, recomputing each
 * segment from its checkpoint: about sqrt(nsteps) states of memory and one extra forward
 * pass.  The recomputation keeps, for every step of the segment in hand, the step's Landau
 * solution, force and streamed deviations h (5 + 17 values per cell for the paper's set,
 * in the storage type), which the reverse steps read.  segment >= nsteps keeps those
 * values for every step instead (one segment, e.g. 54 GB for 512^2 FP32 and 2000 steps):
 * the forward runs once and no step is recomputed.  The results do not depend on segment.  It returns J and dJ/dsigma_m (host, rlbm_num_modes values; may be NULL),
 * dJ/d(eta/s) (host, 1; may be NULL) and dJ/dF_body (host, 2; may be NULL; zero for the
 * eight-direction set, which has no force term), evaluated at
 * the current sigma, eta/s and body force.  FP64 and FP32 storage only (E_INVAL for the
 * 16-bit forms).  Syncs.
 * Workspace: rlbm_gradient_query_workspace bytes of caller-owned device memory, 256-byte
 * aligned, used only during the call.  Device errors of the run are latched as usual. */
RLBM_API rlbm_status rlbm_gradient_query_workspace(const rlbm_ctx *ctx, int64_t nsteps, int32_t segment,
                                                   size_t *bytes);
RLBM_API rlbm_status rlbm_gradient(rlbm_ctx *ctx, int64_t nsteps, int32_t segment, void *dev_workspace,
                                   size_t bytes, double *J, double *grad_sigma, double *grad_eta_over_s,
                                   double *grad_body_force);

/* Wait for queued work and report latched device errors. */
RLBM_API rlbm_status rlbm_sync(rlbm_ctx *ctx);

/* Self-test of the failure path (the paper has no counterpart).  Queues one kernel whose
 * thread waits on an mbarrier that nothing arrives on, with the bounded wait the step
 * kernels put on their TMA copies, for max_cycles SM clocks (1 <= max_cycles <= 2^31, about
 * 1 s at 2 GHz).  The wait runs out and latches the timeout in the context's device error
 * word, so the next syncing call returns RLBM_E_TIMEOUT and the context then accepts only
 * rlbm_free.  Nothing faults and nothing is left in flight.  Async. */
RLBM_API rlbm_status rlbm_wait_selftest(rlbm_ctx *ctx, int64_t max_cycles);

/* Number of steps taken since rlbm_init (or set by rlbm_set_state); -1 if ctx is NULL. */
RLBM_API int64_t rlbm_current_step(const rlbm_ctx *ctx);

/* Human-readable message of the last failing call on ctx, or of the last failing
 * rlbm_query_workspace / rlbm_init on this thread when ctx is NULL.  Never NULL. */
RLBM_API const char *rlbm_last_error(const rlbm_ctx *ctx);

/* Release the host context (does not free the caller's workspace).  NULL is a no-op. */
RLBM_API void rlbm_free(rlbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* RLBM_H */
