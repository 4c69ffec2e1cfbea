/*
 * ic.h -- C ABI of libic: one explicit time step of the inertial-coupling
 * (IC) method with particle compressibility (Balboa Usabiaga and
 * Delgado-Buscalioni, "A minimal model for acoustic forces on Brownian
 * particles", arXiv 1307.0702), on a single GPU.
 *
 * The step (App. A.2, substeps 1-7) couples compressible Landau-Lifshitz
 * fluctuating hydrodynamics on a periodic staggered grid (Sec. 4.2, Eqs.
 * (eq:consvDens), (eq:consvMom), (totp)), advanced by SSP-RK3 with the noise
 * combinations W_1..W_3 of App. A.2, to point particles through the 3-point
 * Peskin kernel (App. A.1): interpolation J (Eq. (Jdis)), spreading S (Eq.
 * (Sdis)), the no-slip impulse exchange (Eq. (eq:noSlip), substeps 4-6) and
 * the particle pressure pi = p(rho) + S Omega, Omega = epsilon V (J rho - rho0)
 * (Eqs. (eq:pressure), (omega)).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an ic_status; on failure ic_last_error(ctx) holds a
 *    one-line message.  A NULL ctx or a NULL required pointer gives
 *    IC_ERR_ARG.
 *  - Grid arrays are nx*ny*nz values indexed [z][y][x] (x fastest).  The
 *    alpha component of a vector field lives on the alpha-face r_i + h/2 e_alpha
 *    and is stored at the index of cell i.  Particle arrays are n*3 values
 *    (x, y, z per particle).
 *  - Host pointers passed in are only read (or written) during the call; the
 *    caller keeps ownership.  All device memory belongs to the context and is
 *    freed by ic_destroy.  It is obtained from params->alloc when given (e.g.
 *    PyTorch's caching allocator), else from cudaMalloc.
 *  - Work is ordered on params->stream (NULL: the library creates its own).
 *    ic_step only enqueues work; ic_sync, ic_forces, ic_time_average,
 *    ic_stats, ic_get_state and ic_checkpoint synchronise that stream and
 *    report device-side errors (non-finite state, neighbour-list overflow).
 *  - A context is not thread-safe.  Different contexts are independent.
 */
#ifndef IC_H
#define IC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ic_ctx ic_ctx;

typedef enum {
  IC_OK = 0,
  IC_ERR_ARG = -1,        /* invalid argument or parameter                  */
  IC_ERR_CUDA = -2,       /* a CUDA runtime call or kernel launch failed    */
  IC_ERR_OOM = -3,        /* device allocation failed                       */
  IC_ERR_NONFINITE = -4,  /* the state became NaN/Inf (e.g. CFL violated)   */
  IC_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up             */
  IC_ERR_STATE = -6,      /* call not valid in the current state            */
  IC_ERR_CAPACITY = -7    /* a fixed-size device table overflowed           */
} ic_status;

enum { IC_FP64 = 0, IC_FP32 = 1 };
/* Standing-wave drive.  MODE: body pressure P cos(k x) sin(omega t) with
 * P = 2 Gamma omega A that holds the k mode at density amplitude A.  PLANE:
 * the paper's drive, Eq. (pext): Delta p0 sin(omega t) on one grid plane with
 * Delta p0 = A N Gamma omega.  omega = (2c/h) sin(kh/2), Gamma = (4 eta/3 +
 * zeta)/(2 rho0), k = 2 pi nlambda / L along wave_axis; both drives use
 * sin(omega t + phi) with phi = wave_phase. */
enum { IC_FORCE_NONE = 0, IC_FORCE_MODE = 1, IC_FORCE_PLANE = 2 };

typedef struct {
  int nx, ny, nz;       /* cells per direction, each >= 6                      */
  double h;             /* grid spacing                                        */
  double rho0;          /* equilibrium density                                 */
  double c;             /* fluid speed of sound c_f, p = p0 + c^2 rho          */
  double eta, zeta;     /* shear and bulk viscosity                            */
  double kT;            /* temperature (0: deterministic, no stochastic stress) */
  double dt;            /* time step                                           */
  uint64_t seed;        /* Philox key of the stochastic stress                 */
  uint32_t box;         /* Philox counter word 3: independent replicas          */
  int precision;        /* IC_FP64 or IC_FP32 (accumulators are FP64 in both)  */
  int forcing;          /* IC_FORCE_*                                          */
  int wave_axis;        /* 0 = x, 1 = y, 2 = z                                 */
  double wave_amp;      /* density amplitude A of the driven mode              */
  int wave_nlambda;     /* wavelengths per box along wave_axis                 */
  int plane_index;      /* driven plane for IC_FORCE_PLANE                     */
  double wave_phase;    /* drive phase phi: sin(omega t + phi)                 */
  void *stream;         /* cudaStream_t or NULL                                */
  void *(*alloc)(size_t bytes, void *alloc_ctx);          /* NULL: cudaMalloc  */
  void (*free)(void *ptr, size_t bytes, void *alloc_ctx); /* NULL: cudaFree    */
  void *alloc_ctx;
} ic_grid_params;

/* Zero-copy device views of the current state, valid until the next call
 * that steps, restores or adds particles.  Fields hold delta rho = rho - rho0
 * (not rho) and g; element type is double (IC_FP64) or float (IC_FP32). */
typedef struct {
  void *drho, *gx, *gy, *gz;
  int precision;
  int n_particles;
  void *q;              /* n*3 device positions: FP64 length units (IC_FP64) or 64-bit
                           fixed point q/h in units of 2^-40 (IC_FP32) */
} ic_views;

/* Creates a context: validates params (IC_ERR_ARG), allocates the three
 * RK3 state buffers and sets rho = rho0, g = 0. */
ic_status ic_create_grid(const ic_grid_params *params, ic_ctx **out);

/* Uploads the fluid state from host arrays (density rho, not delta rho, and
 * face momenta g), each nx*ny*nz doubles.  Any of gx, gy, gz may be NULL (zero). */
ic_status ic_set_state(ic_ctx *ctx, const double *rho, const double *gx, const double *gy,
                       const double *gz);

/* Downloads the fluid state to host arrays of nx*ny*nz doubles (NULL skips). */
ic_status ic_get_state(ic_ctx *ctx, double *rho, double *gx, double *gy, double *gz);

/* Thermal initial state: draws delta rho ~ N(0, rho0 kT/(c^2 h^3)) and
 * g ~ N(0, rho0 kT/h^3) (the discrete Gibbs measure of the linearised fluid,
 * whose velocity variance kT/(rho0 h^3) is the equipartition of Sec. 4.5)
 * from Philox purpose 1, removes their means, and adds them to the current
 * state (add != 0) or replaces it (add == 0).  Call before ic_add_particles,
 * which sets particle velocities from the fluid. */
ic_status ic_init_thermal(ic_ctx *ctx, uint64_t seed, int add);

/* Appends n particles.  q: n*3 positions (wrapped into the box); u: n*3
 * velocities or NULL for u = J v at q (no-slip, Eq. (noslip)); m_e: n excess
 * masses (m_e > -m_f; Eq. (eq:particleMass)); kappa_ratio: n values of
 * kappa_p/kappa_f > 0, giving epsilon_pf = c^2 (kappa_f/kappa_p - 1) (Eqs.
 * (part_svel), (ke)); k_spring: n spring constants of a tether
 * F = -k_s (q - q_eq) with q_eq the initial position, or NULL (free).
 * *first_id (if not NULL) receives the index of the first new particle. */
ic_status ic_add_particles(ic_ctx *ctx, int n, const double *q, const double *u,
                           const double *m_e, const double *kappa_ratio,
                           const double *k_spring, int *first_id);

/* Advances nsteps time steps (App. A.2 substeps 1-7).  w: nsteps host
 * weights of the time averages (Sigma w F, Sigma w lambda, Sigma w A^2), or
 * NULL for weight 0.  Enqueues work only (a CUDA graph per buffer parity). */
ic_status ic_step(ic_ctx *ctx, int nsteps, const double *w);

/* Latest step's particle data to host n*3 arrays (NULL skips): lambda, the
 * fluid force on each particle (substep 4: dg = dt (lambda + F)); u; q. */
ic_status ic_forces(ic_ctx *ctx, double *lambda, double *u, double *q);

/* Pipelined read-back of lambda.  ic_forces_async queues on the stream a
 * copy of the latest step's lambda and of the device status word into the
 * context's pinned host slot (0 or 1) and returns without synchronising.
 * ic_forces_collect waits for that slot's copy alone (not for work queued
 * after it), writes lambda (n*3 doubles) to the host array (NULL skips) and
 * returns the device error the status word carried, as ic_forces does.
 * With both slots a caller reads every step's forces while the next step
 * runs.  IC_ERR_ARG for a slot other than 0 or 1; IC_ERR_STATE when the slot
 * holds no queued copy (each queued copy is collected once). */
ic_status ic_forces_async(ic_ctx *ctx, int slot);
ic_status ic_forces_collect(ic_ctx *ctx, int slot, double *lambda);

/* Kernel-averaged fluid density J rho^{n+1} at q^{n+1/2} of the latest step
 * (n values; m_f = V J rho, App. A.2 substep 4), to a host array.  Its
 * equilibrium variance is rho0 kT / (c_p^2 V) (Eq. (eq:densityVariance)). */
ic_status ic_particle_density(ic_ctx *ctx, double *jrho);

/* Weighted time averages since the last reset: spring force <F>_w and fluid
 * force <lambda>_w (n*3 each, NULL skips) and <A^2>_w of the driven-mode
 * density amplitude A(t) = (2/N) sum (rho - rho0) cos(k x).  The radiation
 * force of Sec. 6 is -<F>_w.  reset != 0 zeroes the sums after reading.
 * IC_ERR_STATE if the weights summed to 0. */
ic_status ic_time_average(ic_ctx *ctx, double *f_spring, double *lambda, double *a2, int reset);

/* Total momentum h^3 sum g + sum m_e u (3 doubles, Eq. (eq:totmom)), current
 * driven-mode amplitude A, and the step counter (each may be NULL). */
ic_status ic_stats(ic_ctx *ctx, double *p_total, double *mode_amp, int64_t *step);
/* Number of neighbour-list rebuilds the context's steps have made (App. A.1:
 * a particle's kernel touches the 27 cells around it, so two particles
 * interact only within 4h + skin on every axis; the lists are rebuilt, by a
 * counting sort of the particles into bins of whole cells, after a particle
 * has moved a quarter of the skin).  Synchronises the stream; IC_ERR_ARG for
 * a NULL count. */
ic_status ic_neighbour_rebuilds(ic_ctx *ctx, int64_t *count);

/* Index-check build.  libic_bounds.so is this library compiled with
 * -DIC_BOUNDS_CHECK: every grid, noise, neighbour-bin and particle index the
 * kernels form is checked against its array; one outside it raises a flag,
 * the access is redirected to the array's first element, and the next status
 * check (ic_step, ic_sync, ic_stats ...) returns IC_ERR_ARG naming the kernel
 * family.  A debug build: the flags are read back with a device
 * synchronisation.  ic_bounds_check_build returns 1 in that build, 0 in
 * libic.so.  ic_bounds_selftest launches (on the legacy default stream) a
 * kernel that passes an index equal to its extent to the check without
 * touching memory, and waits for it: IC_OK if the flag rose (it is cleared
 * again), IC_ERR_STATE in a build without the checks, IC_ERR_CUDA if the
 * launch fails. */
int ic_bounds_check_build(void);
ic_status ic_bounds_selftest(void);
/* The objective whose gradients the adjoint computes (Sec. 6 reads the
 * acoustic force as the time-averaged tether force):
 *   *phi = sum_p d_p . <F_p>_w,  <F_p>_w = sum_n w_n F_p^{n+1/2} / sum_n w_n
 * from the context's weighted sums (those of ic_time_average), summed over
 * the particles in index order.  direction: n x 3 doubles (host), or NULL for
 * the x axis of every particle.  reset != 0 zeroes the sums after reading.
 * Synchronises the stream; IC_ERR_ARG for a NULL phi, IC_ERR_STATE if the
 * weights sum to zero. */
ic_status ic_objective(ic_ctx *ctx, const double *direction, double *phi, int reset);

/* Synchronises the stream and reports device-side errors raised since the
 * last check (IC_ERR_NONFINITE, IC_ERR_CAPACITY). */
ic_status ic_sync(ic_ctx *ctx);

/* Serialises the complete state (fields, particles, accumulators, step
 * counter).  buf == NULL: *bytes receives the size needed.  Resuming from a
 * checkpoint reproduces the uninterrupted run bit for bit. */
ic_status ic_checkpoint(ic_ctx *ctx, void *buf, size_t *bytes);
/* Restores a checkpoint written by a context of the same grid and precision. */
ic_status ic_restore(ic_ctx *ctx, const void *buf, size_t bytes);

ic_status ic_device_views(ic_ctx *ctx, ic_views *out);

/* Batched ensemble: many independent boxes (distinct contexts on the current
 * device, e.g. different sizes, seeds or box ids) advanced together, the
 * observables of the method being ensemble averages (Sec. 6).  ic_batch_step
 * uploads the weights of every box, then launches each box's own step graph
 * on the box's stream, step by step across the ensemble, so that the boxes
 * advance independently (no ensemble-wide join between steps).  With
 * IC_BATCH_GRAPH=1 in the environment it instead captures the whole ensemble
 * step -- every box's kernels as a branch on the box's stream (boxes sharing
 * a stream run one after the other in it) -- into one CUDA graph per buffer
 * parity and launches that once per step.  Either way each box evolves
 * exactly as under its own ic_step.  The batch does not own the contexts;
 * modifying a context (adding particles, restoring) makes the batch
 * re-capture.  All boxes must be at the same step parity (stepped the same
 * number of times).  w: nsteps weights applied to every box, or NULL. */
typedef struct ic_batch ic_batch;
ic_status ic_batch_create(ic_ctx *const *ctxs, int n, ic_batch **out);
ic_status ic_batch_step(ic_batch *batch, int nsteps, const double *w);
void ic_batch_destroy(ic_batch *batch);

/* Stage-kernel tiling.  The paper has no counterpart: this is a performance
 * setting.  The RK3 stage kernel marches CTAs along z in runs of at least
 * zchunk planes, over one of two families of tiles:
 *   column tiles, tile_x 32 or 16 (tile_y follows: 13 or 8 in FP32, 6 or 4
 *     in FP64), each thread one cell, for any grid;
 *   whole rows, tile_x 0 (FP32 only, nx a multiple of 4 and at most 128):
 *     bands of whole x rows copied into shared memory by bulk copies, four
 *     cells per thread (ic_get_tile then reports tile_x = nx and the band
 *     height as tile_y).  With noise it stores the divergence of the stochastic
 *     stress for stages 2 and 3 instead of its normals.
 * Within a family every field, particle and force is bit for bit the same
 * under every tiling; only the driven-mode amplitude A(t) and <A^2>_w change,
 * by the rounding of their reduction order.  Between the families the same
 * holds at kT = 0; with noise results agree to the rounding of the stress
 * divergence.  A context starts on whole rows where it can, kT = 0 and the
 * band planner gives its CTAs runs of at least 8 planes (a large box), on
 * column tiles otherwise.
 * ic_set_tile: IC_ERR_ARG for tile_x not 0, 16 or 32, whole rows on a grid
 * that does not take them, or zchunk < 8 (unless it is at least nz).
 * ic_get_tile: the current tiling (each pointer may be NULL).
 * ic_autotune synchronises the stream, times the three stage kernels of every
 * candidate (column tiles: tile_x 32 with each staging mode of
 * ic_set_stage_copy that the grid allows, and 16; whole rows: the band
 * planner's choice; zchunk 32, 16 and 8, clipped to nz) of both families at
 * kT = 0, of the context's current family with noise (so that tuning never
 * changes a run's results), reps
 * repetitions each, on the context's scratch buffers (U^n is left untouched:
 * the state is unchanged) and keeps the fastest; choice[3] (or NULL) receives
 * tile_x, tile_y, zchunk (the staging mode is kept in the context).
 * ic_batch_autotune tunes one context of each distinct grid shape and
 * precision of the batch and gives the choice to the others. */
ic_status ic_set_tile(ic_ctx *ctx, int tile_x, int zchunk);
ic_status ic_get_tile(const ic_ctx *ctx, int *tile_x, int *tile_y, int *zchunk);
ic_status ic_autotune(ic_ctx *ctx, int reps, int *choice);
ic_status ic_batch_autotune(ic_batch *batch, int reps);

/* Loads of the FP32 wide-tile stage kernel (tile_x 32).  The paper has no
 * counterpart: this is a performance setting; every mode gives the same bits.
 *   IC_STAGE_COPY_THREAD: each thread copies its own values into shared
 *     memory (4-byte cp.async).  Works on every grid.
 *   IC_STAGE_COPY_BULK: each plane pair's tile rows (40 floats, x0 - 4 to
 *     x0 + 36) are copied by TMA bulk copies (cp.async.bulk, one or two per
 *     row), their completion tracked by an mbarrier.
 *   IC_STAGE_COPY_ROWS16: the same rows by 16-byte cp.async, one thread per
 *     row, signalling the same mbarrier.
 * The row modes need nx a multiple of 4 and at least 40, and 16-byte aligned
 * fields (always so for the context's own buffers unless a custom allocator
 * returns others); elsewhere the kernel falls back to IC_STAGE_COPY_THREAD.
 * ic_set_stage_copy: IC_ERR_ARG for an unknown mode.  ic_get_stage_copy:
 * the mode the next step's stage kernels use (after that fallback).  A row
 * copy that has not landed after about a second stops the kernel; the next
 * call that reads the device status returns IC_ERR_TIMEOUT.  ic_autotune
 * times every mode of the wide tile. */
enum { IC_STAGE_COPY_THREAD = 0, IC_STAGE_COPY_BULK = 1, IC_STAGE_COPY_ROWS16 = 2 };
ic_status ic_set_stage_copy(ic_ctx *ctx, int mode);
ic_status ic_get_stage_copy(const ic_ctx *ctx, int *mode);

/* Measurement helper (the paper has no counterpart): the FP64 fused
 * multiply-add rate of the current device, from one launch of eight
 * independent FMA chains per thread over 8 CTAs of 256 threads per SM, each
 * thread running iters iterations, timed by CUDA events on a stream of its
 * own (after a short warm-up launch).  *flops_per_s = 2 FLOP per FMA over the
 * measured time; *seconds (may be NULL) that time.  Synchronous; IC_ERR_ARG
 * for iters <= 0 or a NULL result pointer, IC_ERR_CUDA on a CUDA error.  It
 * allocates 8 bytes of device memory for the duration of the call. */
ic_status ic_fma64_rate(int iters, double *flops_per_s, double *seconds);

/* Verification entry point: the library's counter-based generator,
 * Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11), which draws the
 * stochastic stress (Sec. 4.2) and the thermal initial state, evaluated by
 * the same device code for n counter/key pairs.  in: n*6 host words (ctr0,
 * ctr1, ctr2, ctr3, key0, key1 per pair); out: n*4 host words.  Needs no
 * context: runs on the current device with its own temporary buffers and
 * synchronises it.  IC_ERR_ARG for n < 0, or a NULL array with n > 0;
 * IC_ERR_OOM, IC_ERR_CUDA on failure. */
ic_status ic_philox4x32_10(int n, const uint32_t *in, uint32_t *out);

/* Kernel timing for measurement.  While enabled, ic_step launches without
 * CUDA graphs and brackets every kernel (and ic_adjoint_step every adjoint
 * kernel) with CUDA events on the context's stream.  ic_profile_read
 * synchronises and returns, per kernel class (0: fluid RK3 stages, 1:
 * particle kernels, 2: end-of-step reduction, 3: adjoint of the RK3 stage
 * rates, 4: other adjoint grid kernels, 5: adjoint particle kernels), the
 * summed device milliseconds (ms[IC_PROFILE_CLASSES]) and launch counts
 * (launches[IC_PROFILE_CLASSES]) since the last reset. */
#define IC_PROFILE_CLASSES 6
ic_status ic_profile(ic_ctx *ctx, int enable);
ic_status ic_profile_read(ic_ctx *ctx, double *ms, int64_t *launches, int reset);

/* One SSP-RK3 step of the fluid alone (no particles) that allocates no
 * device memory.  The paper has no counterpart: this is for callers that
 * cannot allocate when they step -- code running inside another framework's
 * stream capture (cudaMalloc is not allowed there), hosts whose device memory
 * is all reserved by their own pool, plug-ins that may not allocate after
 * start-up.  params: as for ic_create_grid (stream is used; alloc, free and
 * alloc_ctx are ignored); in / out: device pointers to delta rho, g_x, g_y,
 * g_z of nx*ny*nz values each in the params' precision; no out array may
 * share a byte with an in array or with another out array (IC_ERR_ARG);
 * step: the step index n (Philox counter and drive phase).  The same
 * kernels as ic_step, without the particle terms.  Scratch lives in one static
 * device array of 5.5 MiB held by every GPU that loads the library, so
 * nx*ny*nz must not exceed IC_NOALLOC_MAX_CELLS (else IC_ERR_CAPACITY).  Its
 * device address is looked up on the first call in each CUDA context and
 * cached with the context's id, so a device reset (which ends the context)
 * makes the next call look it up again: make the first call in a context
 * before any stream capture.  Calls share the array (it keeps the last
 * call's contents), so calls that overlap on the GPU race.  Returns
 * IC_ERR_ARG on invalid parameters or pointers, IC_ERR_CUDA if the symbol
 * lookup or a launch fails; work is enqueued on params->stream. */
#define IC_NOALLOC_MAX_CELLS 32768
ic_status ic_fluid_step_noalloc(const ic_grid_params *params, const void *const in[4], void *const out[4],
                                int64_t step);

/* ------------------------------------------------------------------------
 * Adjoint of the deterministic step (kT = 0): reverse-mode gradients of
 *
 *   Phi = sum_n weight_n sum_p d_p . F_p^{n+1/2}
 *
 * (F = -k_s (q^{n+1/2} - q_eq) the tether force of App. A.2 substep 2 that
 * Sec. 6 reads the acoustic force from; d_p a direction per particle) with
 * respect to every particle's m_e and epsilon_pf, the drive amplitude A
 * (ic_grid_params.wave_amp) and the state (delta rho, g, q, u) at the start
 * of the reversed steps.  The reverse sweep is the transpose of substeps 7 to
 * 1 of App. A.2 with J and S swapping roles (they are adjoint, Eq. (adj)).
 *
 * Use: ic_adjoint_enable once the particles are in place; then, for the steps
 * n = N-1 down to 0: restore the state at the start of step n (for instance
 * with ic_snapshot_load), ic_step_record (step n forward, keeping the tape),
 * ic_adjoint_step(weight_n).  ic_adjoint_read returns the accumulated
 * gradients and the adjoint of the state at the start of the last reversed
 * step.  Gradients with respect to kappa_p/kappa_f follow from
 * epsilon_pf = c^2 (kappa_f/kappa_p - 1): dPhi/d(kappa_p/kappa_f) =
 * -c^2 / (kappa_p/kappa_f)^2 dPhi/d epsilon_pf.  The adjoint spreads with
 * atomic adds: it is reproducible to rounding, not bit for bit.
 *
 * ic_adjoint_enable allocates the tape and adjoint fields (29 grid fields in
 * the context's precision, 20 doubles per particle) and zeroes them; it
 * returns IC_ERR_STATE if kT > 0, IC_ERR_OOM if allocation fails.  Adding
 * particles afterwards makes the other calls return IC_ERR_STATE until it is
 * called again. */
ic_status ic_adjoint_enable(ic_ctx *ctx);
/* Zeroes the adjoint state and the gradients and sets the directions d_p
 * (n x 3 doubles, host; NULL: the x axis for every particle). */
ic_status ic_adjoint_reset(ic_ctx *ctx, const double *direction);
/* One forward step, as ic_step(ctx, 1, NULL), that keeps what the reverse
 * sweep of that step needs (q^n, u^n, the first RK stage and the momenta
 * before substep 6).  The time averages are not updated. */
ic_status ic_step_record(ic_ctx *ctx);
/* Reverses the step recorded last: the adjoint held by the context goes from
 * the state after that step to the state before it, and the gradients gain
 * the step's terms, weight * sum_p d_p . F_p included.  IC_ERR_STATE if no
 * step is recorded or the state has moved on since.  Enqueues work only: the
 * reverse step runs as a CUDA graph per set of recorded buffers (captured on
 * first use; the step's drive derivative and weight are rewritten in it
 * before each launch), or kernel by kernel while profiling or with the
 * environment variable IC_NO_GRAPH=1. */
ic_status ic_adjoint_step(ic_ctx *ctx, double weight);
/* Reads (each pointer may be NULL): grad_m_e[n], grad_eps[n], *grad_A, the
 * adjoint of delta rho and g (nx*ny*nz doubles each, [z][y][x]) and of q and u
 * (n x 3).  Synchronises the stream. */
ic_status ic_adjoint_read(ic_ctx *ctx, double *grad_m_e, double *grad_eps, double *grad_A, double *rho_bar,
                          double *gx_bar, double *gy_bar, double *gz_bar, double *q_bar, double *u_bar);

/* dPhi / d(kappa_p / kappa_f) of every particle (n doubles, host): the
 * epsilon gradient of ic_adjoint_read taken through epsilon_pf =
 * c_f^2 (kappa_f / kappa_p - 1) (Eqs. (part_svel), (ke)), with kappa_p / kappa_f
 * recovered from the context's epsilon.  Synchronises the stream; IC_ERR_ARG
 * for a NULL pointer, IC_ERR_STATE as ic_adjoint_read. */
ic_status ic_adjoint_read_kappa(ic_ctx *ctx, double *grad_kappa_ratio);

/* Step tapes: ic_step_record_tape runs ic_step_record and copies everything
 * the reverse sweep of that step reads (U^n, the first two RK stages, the
 * momenta before substep 6, U^{n+1}, and q^n, q^{n+1/2}, u^n, F, dg) into a
 * caller-owned device buffer of ic_tape_size bytes, 16-byte aligned
 * (IC_ERR_ARG otherwise); ic_adjoint_step_tape reverses the step of such a
 * tape, as ic_adjoint_step does for the step recorded last, whatever the
 * state has done since.  A rollout can so record a whole segment and then
 * reverse it without recomputing its steps.  A tape recorded by this
 * context is reversed without synchronising; one from elsewhere has its
 * header read back and checked (IC_ERR_ARG if it is of another grid,
 * precision or particle count). */
ic_status ic_tape_size(const ic_ctx *ctx, size_t *bytes);
ic_status ic_step_record_tape(ic_ctx *ctx, void *dev_buf);
ic_status ic_adjoint_step_tape(ic_ctx *ctx, const void *dev_buf, double weight);

/* Device snapshots of the state a rollout needs to restart a step (fields,
 * q, u, step counter): the caller owns dev_buf, device memory of
 * ic_snapshot_size bytes, 16-byte aligned (IC_ERR_ARG otherwise).  Save
 * enqueues device copies on the context's stream; load enqueues the copies
 * back (and the step's drive).  Neither synchronises when the buffer was last
 * saved by the same context (its header is remembered); a buffer from
 * elsewhere has its header read back and checked: IC_ERR_ARG if it is of
 * another grid, precision or particle count.  The time averages are not part
 * of a snapshot. */
ic_status ic_snapshot_size(const ic_ctx *ctx, size_t *bytes);
ic_status ic_snapshot_save(ic_ctx *ctx, void *dev_buf);
ic_status ic_snapshot_load(ic_ctx *ctx, const void *dev_buf);

const char *ic_last_error(const ic_ctx *ctx);
void ic_destroy(ic_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* IC_H */
