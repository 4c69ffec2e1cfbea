// Host-side context of libic and the launch interfaces between its files.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ic.h"

namespace ic {

// Programmatic dependent launch of the step's kernels: each may be
// scheduled while its predecessor in the stream drains, and waits for it
// (pdl_enter, ic_device.cuh) before its first access to global memory.  On
// inside ic_batch_step and with IC_PDL=1, off otherwise: on GB300 it made
// the 128^3 box with 10^4 particles 2 % slower per step and the 256-box
// ensemble 2 % faster.
extern thread_local bool t_pdl_scope;
bool pdl_enabled();

template <typename... K, typename... A>
cudaError_t launch_k(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream, A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

constexpr int kMaxNeighbours = 64;     // per-particle neighbour table width
constexpr double kSkin = 1.0;          // neighbour-list skin in units of h
constexpr int kStatusNonfinite = 1;    // device status bits
constexpr int kStatusNbrOverflow = 2;
constexpr int kStatusSkin = 4;
constexpr int kStatusStaging = 8;     // a bulk copy into shared memory did not land in time
// loads of the FP32 wide-tile stage kernel (IC_STAGE_COPY_THREAD / _BULK / _ROWS16)
constexpr int kDefaultStageCopy = 0;

// Per-stage constants of the fluid kernel, derived on the host in FP64 and
// handed to the kernel in its working precision.
template <typename real>
struct FluidConsts {
  int nx, ny, nz;
  real rho0, c2, inv_h, dt, eta, lam2;        // lam2 = zeta - 2 eta / 3
  real noise_diag, noise_trace, noise_edge;   // sqrt2 S, sqrt2 (B - S/3), S
  // The stage kernels carry the momentum fluxes scaled by 4 (so that the
  // advective products of two-point sums need no factor 1/4) and fold 1/h and
  // dt into these constants:
  real c2x4;                                  // 4 c^2
  real visc_d, visc_o;                        // 8 eta / h (diagonal), 4 eta / h (edges)
  real lam2x4_h;                              // 4 lam2 / h
  real noise_d4, noise_t4, noise_e4;          // 4 x the noise coefficients
  real out_flux, out_mass;                    // -dt / (4 h), -dt / h
  int forcing, wave_axis, plane_index;
  const real *cos_table;                      // cos(k x_i) along the wave axis
  const real *drive;                          // drive amplitude of each RK stage of the current step
  uint32_t k0, k1, box;                       // Philox key and box
  int noise;
};

// The constants of a grid, derived in FP64 and rounded once to real.
template <typename real>
FluidConsts<real> make_fluid_consts(const ic_grid_params &p, const real *cos_table, const real *drive) {
  FluidConsts<real> c{};
  c.nx = p.nx;
  c.ny = p.ny;
  c.nz = p.nz;
  c.rho0 = real(p.rho0);
  c.c2 = real(p.c * p.c);
  c.inv_h = real(1.0 / p.h);
  c.dt = real(p.dt);
  c.eta = real(p.eta);
  const double lam2 = p.zeta - 2.0 * p.eta / 3.0;
  c.lam2 = real(lam2);
  const double vol_dt = p.h * p.h * p.h * p.dt;
  const double S = std::sqrt(2.0 * p.eta * p.kT / vol_dt);
  const double B = std::sqrt(p.zeta * p.kT / (3.0 * vol_dt));
  c.noise_diag = real(std::sqrt(2.0) * S);
  c.noise_trace = real(std::sqrt(2.0) * (B - S / 3.0));
  c.noise_edge = real(S);
  c.c2x4 = real(4.0 * p.c * p.c);
  c.visc_d = real(8.0 * p.eta / p.h);
  c.visc_o = real(4.0 * p.eta / p.h);
  c.lam2x4_h = real(4.0 * lam2 / p.h);
  c.noise_d4 = real(4.0 * std::sqrt(2.0) * S);
  c.noise_t4 = real(4.0 * std::sqrt(2.0) * (B - S / 3.0));
  c.noise_e4 = real(4.0 * S);
  c.out_flux = real(-p.dt / (4.0 * p.h));
  c.out_mass = real(-p.dt / p.h);
  c.forcing = (p.wave_amp == 0.0) ? IC_FORCE_NONE : p.forcing;
  c.wave_axis = p.wave_axis;
  c.plane_index = p.plane_index;
  c.cos_table = cos_table;
  c.drive = drive;
  c.k0 = uint32_t(p.seed & 0xffffffffull);
  c.k1 = uint32_t(p.seed >> 32);
  c.box = p.box;
  c.noise = p.kT > 0.0;
  return c;
}

// Device pointers of the particle arrays; element type of the void* arrays
// is the context's real type (double or float).
struct ParticleStore {
  int n = 0, cap = 0;
  double *q = nullptr, *q_eq = nullptr, *q_build = nullptr, *q_half = nullptr;  // n*3
  double *acc = nullptr;     // n*6: sum w F, sum w lambda
  void *u = nullptr;         // n*3
  void *m_e = nullptr, *eps = nullptr, *k_s = nullptr;   // n
  void *w = nullptr;         // n*18: centre weights [axis][3], own-axis face weights [axis][3]
  void *jv_n = nullptr;      // n*3: J^{n+1/2} v^n
  void *force = nullptr;     // n*3: F^{n+1/2}
  void *dg = nullptr;        // n*3: impulse dg
  void *lam = nullptr;       // n*3: lambda
  void *jrho = nullptr;      // n: J rho^{n+1} at q^{n+1/2}
  int *base = nullptr;       // n*6: centre base (x,y,z), own-axis face base (x,y,z)
  int *nbr = nullptr;        // n*kMaxNeighbours, ascending indices
  int *nnbr = nullptr;       // n
  int *order = nullptr;      // n: particle indices grouped by neighbour bin
  int *bins = nullptr;       // 2 nbins + 1: first slot of each bin in order (nbins + 1), fill cursors
};

// Neighbour bins: the box cut into nb[a] slabs per axis of whole cells, each
// at least floor(cutoff / h) + 1 cells wide, so that two particles within the
// cutoff on every axis sit in the same or adjacent bins.  Returns nb[0] nb[1] nb[2].
int neighbour_bins(const ic_grid_params &p, int nb[3]);

struct Device {
  int64_t *step = nullptr;        // [0] step counter n, [1] step of weights[0], [2] number of weights
  double *weights = nullptr;      // averaging weights of the current ic_step call (0 outside)
  double *scalars = nullptr;      // [0] sum w, [1] sum w A^2, [2] A of the last step
  int *status = nullptr;          // error bits
  int *rebuild = nullptr;         // neighbour list must be rebuilt
  long long *rebuilds = nullptr;  // neighbour-list rebuilds so far
  int *bin_done = nullptr;        // CTAs of the running k_final that have finished (0 between launches)
  double *partials = nullptr;     // per-CTA partial sums
};

// Adjoint of the deterministic step: the tape of the last recorded step and
// the adjoint fields (allocated by ic_adjoint_enable).
struct AdjointStore {
  bool on = false;
  int np = 0;                          // particles when enabled
  void *tU1[4] = {}, *tG3[3] = {};     // tape: U_1 and g~ (the momenta before substep 6)
  void *tq = nullptr, *tu = nullptr;   // tape: q^n (8 bytes per component) and u^n
  int rec_cur = -1;                    // buffer of U^n of the recorded step (-1: none to reverse)
  int64_t rec_step = 0;
  // grid adjoint fields in the context's precision
  void *bar[4] = {}, *acc[4] = {}, *vbar[3] = {}, *gpart[3] = {}, *rfbar[3] = {}, *vel[3] = {};
  void *pibar = nullptr, *rhox = nullptr;
  // particle adjoints and gradients (FP64)
  double *qbar = nullptr, *ubar = nullptr, *qhbar = nullptr, *fbar = nullptr, *jvnh = nullptr;
  double *gme = nullptr, *geps = nullptr, *gA = nullptr, *dir = nullptr;
  void *grid_block = nullptr, *part_block = nullptr;
};


// A named NVTX range for the lifetime of the object (host-side tracing; a
// no-op unless a profiler is attached).
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

// A captured kernel node whose scalar arguments change between launches of
// its graph: the node, its launch configuration and byte copies of its
// arguments (kernelParams points into them).
struct KeptNode {
  cudaGraphNode_t node = nullptr;
  cudaKernelNodeParams p{};
  std::vector<std::vector<unsigned char>> arg;
  std::vector<void *> ptr;
  template <typename... A>
  void keep(cudaGraphNode_t n, const void *func, dim3 grid, dim3 block, size_t smem, const A &...a) {
    node = n;
    arg.clear();
    (arg.emplace_back(reinterpret_cast<const unsigned char *>(&a), reinterpret_cast<const unsigned char *>(&a) + sizeof(A)),
     ...);
    ptr.resize(arg.size());
    for (size_t i = 0; i < arg.size(); ++i) ptr[i] = arg[i].data();
    p.func = const_cast<void *>(func);
    p.gridDim = grid;
    p.blockDim = block;
    p.sharedMemBytes = static_cast<unsigned int>(smem);
    p.kernelParams = ptr.data();
    p.extra = nullptr;
  }
};

// The reverse sweep of one recorded step as a CUDA graph (one per tape, keyed
// by its U^n buffer): the stage transposes (whose drive derivative depends on
// the step) and the particles' start (the objective's weight) are updated
// before each launch.
struct AdjGraph {
  cudaGraph_t graph = nullptr;   // kept: the updated nodes belong to it
  cudaGraphExec_t exec = nullptr;
  KeptNode rates[3];   // by RK stage
  KeptNode start;
};

}  // namespace ic

struct ic_ctx {
  ic_grid_params p{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t cells = 0;
  size_t real_size = 8;
  void *U[3][4] = {};      // three state buffers (delta rho, gx, gy, gz)
  int cur = 0;             // buffer holding U^n (0 or 1); buffer 2 holds U^{n+1/2}
  ic::Device d{};
  ic::ParticleStore ps{};
  ic::AdjointStore adj{};
  std::unordered_map<uintptr_t, std::pair<int64_t, int>> snapshots;   // device snapshots saved: step, particles
  std::unordered_map<uintptr_t, std::pair<int64_t, int>> tapes;       // step tapes recorded: step, particles
  std::unordered_map<const void *, ic::AdjGraph> adj_graphs;           // reverse-step graphs by tape
  void *pp = nullptr;       // particle pressure S Omega at centres (zero outside particle stencils)
  void *noise[18] = {};     // kT > 0: W_2 and W_3 of the current step (6 components each), written by stage 1;
                            // FP64: also W_1 (12..17), all three drawn by k_draw_noise before stage 1
  bool any_spring = false;  // some particle is tethered: the stage force source is launched
  double *cos_table = nullptr;      // cos(k x_i) along the wave axis, FP64
  float *cos_table_f = nullptr;     // the same in FP32
  double *drive = nullptr;          // [0..2] FP64 drive amplitude of each RK stage of the current step
  float *drive_f = nullptr;         // [0..2] the same in FP32
  size_t n_partials = 0;
  int weights_cap = 0;
  int64_t host_step = 0;
  int64_t host_wcount = 0;          // weights count currently on the device
  double *staging = nullptr;        // pinned host staging for weights (cap + 3)
  cudaEvent_t staging_done = nullptr;
  unsigned char *download = nullptr;  // pinned host staging for per-step particle read-back
  size_t download_cap = 0;
  // pipelined read-back slots (ic_forces_async / ic_forces_collect)
  unsigned char *fetch[2] = {nullptr, nullptr};
  size_t fetch_cap[2] = {0, 0};
  cudaEvent_t fetch_done[2] = {nullptr, nullptr};
  int fetch_n[2] = {-1, -1};            // particles of the queued copy, -1: none
  cudaGraphExec_t graph[2] = {nullptr, nullptr};   // one step, per buffer parity
  uint64_t generation = 0;                          // bumped whenever the captured step changes
  int tile_variant = 0;    // stage-kernel tile: 0 = wide (32 x TY), 1 = narrow (16 x TY), 2 = whole rows
  int zchunk = 0;          // fewest z planes a stage-kernel CTA marches (0 = default)
  int stage_copy = ic::kDefaultStageCopy;   // FP32 wide-tile loads (IC_STAGE_COPY_*), where the grid allows
  int sm_count = 1;        // SMs of the context's device
  std::string err;
  double omega = 0, force_amp = 0, kwave = 0;
  // kernel timing (ic_profile): event pairs per kernel class
  bool profiling = false;
  struct Timed {
    cudaEvent_t a, b;
    int cls;
  };
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> event_pool;
  size_t event_next = 0;
  // every device allocation, for ic_destroy
  void *allocs[128] = {};
  size_t alloc_bytes[128] = {};
  int n_allocs = 0;
};

namespace ic {
void *dev_alloc(ic_ctx *ctx, size_t bytes);

// Kernel timing (ic_profile): an event from the context's pool.
inline cudaEvent_t pooled_event(ic_ctx *ctx) {
  if (ctx->event_next == ctx->event_pool.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    ctx->event_pool.push_back(ev);
  }
  return ctx->event_pool[ctx->event_next++];
}

// Launch `fn` and, while profiling, bracket it with events of class `cls`
// (the classes of ic_profile_read).
template <typename F>
cudaError_t timed_launch(ic_ctx *ctx, int cls, F &&fn) {
  if (!ctx->profiling) return fn();
  cudaEvent_t a = pooled_event(ctx), b = pooled_event(ctx);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaEventRecord(a, ctx->stream);
  const cudaError_t e = fn();
  cudaEventRecord(b, ctx->stream);
  ctx->timed.push_back({a, b, cls});
  return e;
}
void dev_free(ic_ctx *ctx, void *p);

// fluid (ic_fluid.cu)
void drive_amplitudes(const ic_ctx *ctx, int64_t step, double out[3]);
size_t fluid_num_partials(const ic_ctx *ctx);
cudaError_t launch_stage(const ic_ctx *ctx, int stage, void *const in_s[4], void *const in_n[4],
                         void *const out[4]);
cudaError_t launch_thermal(ic_ctx *ctx, uint64_t seed, int add);
cudaError_t launch_field_sums(ic_ctx *ctx, void *const state[4], double *dev_out4);
cudaError_t launch_end_of_step(ic_ctx *ctx);

// The end-of-step bookkeeping: the driven-mode amplitude A from the last
// stage's per-CTA partial sums, the weighted sums w and w A^2, the
// non-finite check, the step counter and the next step's drive amplitudes.
// A box with particles does it in the last CTA of its final particle
// substep (k_final), a box without in k_end_of_step.
struct EndArgs {
  const double *partials;
  int nb;
  double inv_cells;
  int has_mode;
  int64_t *step;
  const double *weights;
  double *scalars;
  int *status;
  double amp, omega, dt, phase;
  double *drive;
  float *drive_f;
};
EndArgs end_args(const ic_ctx *ctx);
// context-free stage launch (consts points to a FluidConsts<real> of the params' precision)
cudaError_t launch_stage_raw(const ic_grid_params &p, const void *consts, int stage, const void *const in_s[4],
                             const void *const in_n[4], void *const out[4], void *const noise[12],
                             const int64_t *step, double *partials, cudaStream_t stream);
size_t stage_ctas_raw(const ic_grid_params &p);
// stage-kernel tiling: variant 0 (32-wide) or 1 (16-wide) and the z chunk
constexpr int kMinZChunk = 8;
bool set_stage_tile(ic_ctx *ctx, int variant, int zchunk);
int stage_copy_active(const ic_ctx *ctx);   // the staging mode the next FP32 wide-tile launch uses
void stage_tile(const ic_ctx *ctx, int *tx, int *ty, int *zchunk);
bool rows_active(const ic_ctx *ctx);        // the next stage launch is the whole-row kernel

// whole-row FP32 stage kernel (ic_stage_rows.cu): tile variant 2
constexpr int kTileRows = 2;
bool rows_eligible(const ic_grid_params &p);
bool rows_buffers_aligned(const ic_ctx *ctx);
int rows_ctas(const ic_ctx *ctx, int stage);
// planes of z a CTA of the whole-row kernel marches per step on average (its
// runs start with a fill of the plane rings: short runs pay it often)
double rows_mean_run(const ic_grid_params &p, int sm_count);
void rows_tile(const ic_ctx *ctx, int *ty);
cudaError_t launch_stage_rows(const ic_ctx *ctx, int stage, void *const in_s[4], void *const in_n[4],
                              void *const out[4]);

// particles (ic_particles.cu)
// Index-check flags of the kernels of each source file, cleared on read
// (always 0 unless the library is built with -DIC_BOUNDS_CHECK).
unsigned bounds_flag_fluid();
unsigned bounds_flag_rows();
unsigned bounds_flag_particles();
unsigned bounds_flag_adjoint();
cudaError_t launch_bounds_probe(cudaStream_t stream);

enum ParticlePhase { kHalfStep = 0, kPressure = 1, kForce = 2, kImpulse = 3, kSpread = 4, kFinal = 5 };
// the counting sort into the neighbour bins, if a rebuild is flagged (after
// the host has changed positions outside a step)
cudaError_t launch_particle_bins(ic_ctx *ctx);
cudaError_t launch_particles(ic_ctx *ctx, ParticlePhase phase, int stage, void *const cur[4],
                             void *const tgt[4]);
cudaError_t launch_particle_velocity(ic_ctx *ctx, int first, int n, void *const state[4]);
cudaError_t launch_particle_momentum(ic_ctx *ctx, double *dev_out3);

// adjoint (ic_adjoint.cu): reverse sweep of one recorded step, whose states
// and particle arrays are read from these buffers (the context's own after
// ic_step_record, or a caller's tape after ic_step_record_tape)
struct AdjStepTape {
  void *Un[4], *U1[4], *U2[4], *G3[3], *Unew[4];   // U^n, U_1, U_2, g~, U^{n+1}
  const void *q_n, *q_half, *u_n, *force, *dg;
  int64_t step;
};
// cap: while capturing, the graph whose per-launch nodes are recorded
cudaError_t launch_adjoint_step(ic_ctx *ctx, const AdjStepTape &t, double weight, AdjGraph *cap = nullptr);
// rewrites the per-launch arguments of a captured reverse step for tape t
cudaError_t update_adjoint_graph(const ic_ctx *ctx, AdjGraph &g, const AdjStepTape &t, double weight);
void positions_to_device(const ic_ctx *ctx, const double *q, size_t n3, void *out);
void positions_to_host(const ic_ctx *ctx, const void *in, size_t n3, double *q);
}  // namespace ic
