// C ABI of libic (include/ic.h): context lifetime, host <-> device transfers,
// and the step driver that chains the fluid and particle kernels of one IC
// time step (App. A.2 substeps 1-7) on one stream, captured once per buffer
// parity into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <array>
#include <vector>

#include "ic_device.cuh"
#include "ic_internal.hpp"

namespace ic {

void *dev_alloc(ic_ctx *ctx, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (ctx->n_allocs >= 128) return nullptr;
  void *p = nullptr;
  if (ctx->p.alloc) {
    p = ctx->p.alloc(bytes, ctx->p.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    ctx->allocs[ctx->n_allocs] = p;
    ctx->alloc_bytes[ctx->n_allocs] = bytes;
    ++ctx->n_allocs;
  }
  return p;
}

void dev_free(ic_ctx *ctx, void *p) {
  if (!p) return;
  for (int i = 0; i < ctx->n_allocs; ++i) {
    if (ctx->allocs[i] == p) {
      if (ctx->p.free)
        ctx->p.free(p, ctx->alloc_bytes[i], ctx->p.alloc_ctx);
      else
        cudaFree(p);
      ctx->allocs[i] = ctx->allocs[ctx->n_allocs - 1];
      ctx->alloc_bytes[i] = ctx->alloc_bytes[ctx->n_allocs - 1];
      --ctx->n_allocs;
      return;
    }
  }
}

// set while ic_batch_step enqueues or captures its boxes' steps: the many
// small launches of an ensemble gain from programmatic dependent launch
thread_local bool t_pdl_scope = false;

bool pdl_enabled() {
  const char *v = std::getenv("IC_PDL");
  return t_pdl_scope || (v && v[0] == '1');
}

}  // namespace ic

namespace {

using ic::dev_alloc;
using ic::dev_free;

ic_status fail(ic_ctx *ctx, ic_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return st;
}

ic_status cuda_fail(ic_ctx *ctx, cudaError_t e, const char *where) {
  return fail(ctx, IC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define IC_CUDA(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

void drop_adj_graphs(ic_ctx *ctx) {
  for (auto &kv : ctx->adj_graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  ctx->adj_graphs.clear();
}

void invalidate_graphs(ic_ctx *ctx) {
  ++ctx->generation;
  for (int i = 0; i < 2; ++i)
    if (ctx->graph[i]) {
      cudaGraphExecDestroy(ctx->graph[i]);
      ctx->graph[i] = nullptr;
    }
  drop_adj_graphs(ctx);
}

using ic::timed_launch;

// Enqueue one full time step with U^n in buffer `cur`; U^{n+1} lands in 1 - cur.
// With `record`, the intermediates the adjoint needs and the step overwrites
// (q^n, u^n, U_1 and the momenta g~ before substep 6) are copied to the tape.
cudaError_t enqueue_step(ic_ctx *ctx, int cur, bool record = false) {
  void *const *U0 = ctx->U[cur];
  void *const *U1 = ctx->U[1 - cur];
  void *const *U2 = ctx->U[2];
  const bool parts = ctx->ps.n > 0;
  const size_t fb = size_t(ctx->cells) * ctx->real_size;
  cudaError_t e;
  auto tape = [&](void *const *dst, void *const *src, int n) {
    cudaError_t te = cudaSuccess;
    for (int j = 0; j < n && te == cudaSuccess; ++j)
      te = cudaMemcpyAsync(dst[j], src[j], fb, cudaMemcpyDeviceToDevice, ctx->stream);
    return te;
  };
  // trace names of the substeps (App. A.2)
  static const char *const kStageName[3] = {"IC RK3 stage 1", "IC RK3 stage 2", "IC RK3 stage 3"};
  static const char *const kPhaseName[6][3] = {
      {"IC substeps 1-2: half step, tether force, stencils", "", ""},
      {"IC particle pressure, stage 1", "IC particle pressure, stage 2", "IC particle pressure, stage 3"},
      {"IC tether source, stage 1", "IC tether source, stage 2", "IC tether source, stage 3"},
      {"IC substeps 4-5: impulse", "", ""},
      {"IC substep 6: momentum correction", "", ""},
      {"IC substep 7: positions, force sums", "", ""}};
  auto fluid = [&](int stage, void *const *s, void *const *n, void *const *o) {
    const ic::TraceRange tr(kStageName[stage]);
    return timed_launch(ctx, 0, [&] { return ic::launch_stage(ctx, stage, s, n, o); });
  };
  auto part = [&](ic::ParticlePhase ph, int stage, void *const *tgt) {
    const ic::TraceRange tr(kPhaseName[ph][stage]);
    return timed_launch(ctx, 1, [&] { return ic::launch_particles(ctx, ph, stage, U0, tgt); });
  };
#define IC_TRY(x)                           \
  do {                                      \
    if ((e = (x)) != cudaSuccess) return e; \
  } while (0)
  const bool springs = parts && ctx->any_spring;
  if (record && parts) {
    const size_t n = size_t(ctx->ps.n);
    IC_TRY(cudaMemcpyAsync(ctx->adj.tq, ctx->ps.q, 24 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    IC_TRY(cudaMemcpyAsync(ctx->adj.tu, ctx->ps.u, 3 * ctx->real_size * n, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  if (parts) IC_TRY(part(ic::kHalfStep, 0, U0));
  if (parts) IC_TRY(part(ic::kPressure, 0, U0));
  IC_TRY(fluid(0, U0, U0, U1));
  if (springs) IC_TRY(part(ic::kForce, 0, U1));
  if (record) IC_TRY(tape(ctx->adj.tU1, U1, 4));
  if (parts) IC_TRY(part(ic::kPressure, 1, U1));
  IC_TRY(fluid(1, U1, U0, U2));
  if (springs) IC_TRY(part(ic::kForce, 1, U2));
  if (parts) IC_TRY(part(ic::kPressure, 2, U2));
  IC_TRY(fluid(2, U2, U0, U1));
  if (springs) IC_TRY(part(ic::kForce, 2, U1));
  if (record) IC_TRY(tape(ctx->adj.tG3, U1 + 1, 3));
  if (parts) {
    IC_TRY(part(ic::kImpulse, 0, U1));
    IC_TRY(part(ic::kSpread, 0, U1));
    IC_TRY(part(ic::kFinal, 0, U1));
  }
  // with particles k_final's last CTA has done the end-of-step bookkeeping
  if (!parts) IC_TRY(timed_launch(ctx, 2, [&] { return ic::launch_end_of_step(ctx); }));
#undef IC_TRY
  return cudaSuccess;
}

bool graphs_enabled() {
  const char *v = std::getenv("IC_NO_GRAPH");
  return !(v && v[0] == '1');
}

constexpr size_t kMaxAdjGraphs = 256;

// The reverse sweep of one recorded step: its CUDA graph for this tape
// (captured on first use, its per-step arguments updated after that), or
// the kernels one by one while profiling.
cudaError_t run_adjoint_step(ic_ctx *ctx, const ic::AdjStepTape &t, double weight) {
  if (!graphs_enabled() || ctx->profiling) return ic::launch_adjoint_step(ctx, t, weight);
  const void *key = t.Un[0];
  auto it = ctx->adj_graphs.find(key);
  cudaError_t e = cudaSuccess;
  if (it == ctx->adj_graphs.end()) {
    if (ctx->adj_graphs.size() >= kMaxAdjGraphs) drop_adj_graphs(ctx);   // tapes at ever new addresses
    ic::AdjGraph g;
    e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = ic::launch_adjoint_step(ctx, t, weight, &g);
    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g.graph);
    e = le != cudaSuccess ? le : ce;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (e != cudaSuccess) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
      cudaGetLastError();
      return e;
    }
    it = ctx->adj_graphs.emplace(key, std::move(g)).first;
  } else {
    e = ic::update_adjoint_graph(ctx, it->second, t, weight);
    if (e != cudaSuccess) return e;
  }
  return cudaGraphLaunch(it->second.exec, ctx->stream);
}

template <typename real>
void to_real(const double *src, double offset, std::vector<unsigned char> &dst, size_t n) {
  dst.resize(n * sizeof(real));
  real *d = reinterpret_cast<real *>(dst.data());
  for (size_t i = 0; i < n; ++i) d[i] = real(src[i] - offset);
}

template <typename real>
void from_real(const unsigned char *src, double offset, double *dst, size_t n) {
  const real *s = reinterpret_cast<const real *>(src);
  for (size_t i = 0; i < n; ++i) dst[i] = double(s[i]) + offset;
}

ic_status upload_real(ic_ctx *ctx, void *dev, const double *host, double offset, size_t n) {
  std::vector<unsigned char> tmp;
  if (ctx->p.precision == IC_FP32)
    to_real<float>(host, offset, tmp, n);
  else
    to_real<double>(host, offset, tmp, n);
  IC_CUDA(ctx, cudaMemcpyAsync(dev, tmp.data(), tmp.size(), cudaMemcpyHostToDevice, ctx->stream));
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return IC_OK;
}

ic_status download_real(ic_ctx *ctx, double *host, const void *dev, double offset, size_t n) {
  std::vector<unsigned char> tmp(n * ctx->real_size);
  IC_CUDA(ctx, cudaMemcpyAsync(tmp.data(), dev, tmp.size(), cudaMemcpyDeviceToHost, ctx->stream));
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->p.precision == IC_FP32)
    from_real<float>(tmp.data(), offset, host, n);
  else
    from_real<double>(tmp.data(), offset, host, n);
  return IC_OK;
}

ic_status status_error(ic_ctx *ctx, int st);

ic_status check_device_status(ic_ctx *ctx) {
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int st = 0;
  IC_CUDA(ctx, cudaMemcpy(&st, ctx->d.status, sizeof(int), cudaMemcpyDeviceToHost));
  return status_error(ctx, st);
}

// The status word as read back with other data: IC_OK, or the error it flags
// (the flags are cleared).
ic_status status_error(ic_ctx *ctx, int st) {
#ifdef IC_BOUNDS_CHECK
  {  // the debug build's index checks: any index outside its array is an error
    const unsigned f[4] = {ic::bounds_flag_fluid(), ic::bounds_flag_rows(), ic::bounds_flag_particles(),
                           ic::bounds_flag_adjoint()};
    if (f[0] | f[1] | f[2] | f[3])
      return fail(ctx, IC_ERR_ARG, "index out of bounds in the kernels of (fluid, rows, particles, adjoint) = (%u, %u, %u, %u)",
                  f[0], f[1], f[2], f[3]);
  }
#endif
  if (st == 0) return IC_OK;
  IC_CUDA(ctx, cudaMemset(ctx->d.status, 0, sizeof(int)));
  if (st & ic::kStatusStaging)   // first: the stages it stopped leave the rest of the step undefined
    return fail(ctx, IC_ERR_TIMEOUT, "a bulk copy into a stage kernel's shared memory did not complete");
  if (st & ic::kStatusNonfinite)
    return fail(ctx, IC_ERR_NONFINITE, "state became non-finite (check the CFL numbers c dt/h and c_p dt/h)");
  if (st & ic::kStatusNbrOverflow)
    return fail(ctx, IC_ERR_CAPACITY, "more than %d particles within the neighbour cutoff of one particle",
                ic::kMaxNeighbours);
  return fail(ctx, IC_ERR_STATE, "a particle moved more than half the neighbour skin within one step");
}

// Particle arrays: (pointer slot, bytes per particle)
struct PArray {
  void **slot;
  size_t per;
};

std::vector<PArray> particle_arrays(ic_ctx *ctx) {
  ic::ParticleStore &s = ctx->ps;
  const size_t r = ctx->real_size;
  return {{(void **)&s.q, 24},       {(void **)&s.q_eq, 24},     {(void **)&s.q_build, 24},
          {(void **)&s.q_half, 24},  {(void **)&s.acc, 48},      {&s.u, 3 * r},
          {&s.m_e, r},               {&s.eps, r},                {&s.k_s, r},
          {&s.w, 18 * r},            {&s.jv_n, 3 * r},
          {&s.force, 3 * r},         {&s.dg, 3 * r},             {&s.lam, 3 * r},
          {&s.jrho, r},
          {(void **)&s.base, 6 * sizeof(int)},
          {(void **)&s.nbr, ic::kMaxNeighbours * sizeof(int)},
          {(void **)&s.nnbr, sizeof(int)},
          {(void **)&s.order, sizeof(int)}};
}

ic_status grow_particles(ic_ctx *ctx, int need) {
  ic::ParticleStore &s = ctx->ps;
  if (need <= s.cap) return IC_OK;
  const int cap = std::max(need, std::max(16, 2 * s.cap));
  if (!s.bins) {   // bin starts and fill cursors of the neighbour-list counting sort
    int nb[3];
    const size_t bytes = (2 * size_t(ic::neighbour_bins(ctx->p, nb)) + 1) * sizeof(int);
    s.bins = static_cast<int *>(dev_alloc(ctx, bytes));
    if (!s.bins) return fail(ctx, IC_ERR_OOM, "neighbour bin table allocation of %zu bytes failed", bytes);
  }
  // one spare particle slot per array: lambda's holds the copy of the status
  // word that the final substep leaves after the last particle's lambda
  for (PArray a : particle_arrays(ctx)) {
    void *fresh = dev_alloc(ctx, a.per * size_t(cap + 1));
    if (!fresh) return fail(ctx, IC_ERR_OOM, "particle buffer allocation of %zu bytes failed", a.per * (cap + 1));
    IC_CUDA(ctx, cudaMemsetAsync(fresh, 0, a.per * size_t(cap + 1), ctx->stream));
    if (*a.slot) {
      if (s.n > 0)
        IC_CUDA(ctx, cudaMemcpyAsync(fresh, *a.slot, a.per * size_t(s.n), cudaMemcpyDeviceToDevice, ctx->stream));
      IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      dev_free(ctx, *a.slot);
    }
    *a.slot = fresh;
  }
  s.cap = cap;
  invalidate_graphs(ctx);
  return IC_OK;
}

// Weights of the next nsteps steps (or none) through a pinned staging buffer
// (the caller's w is only read during the call).
ic_status upload_weights(ic_ctx *ctx, int nsteps, const double *w) {
  if (w && nsteps > ctx->weights_cap) {
    // the step counter, the weights' header and the weights share one block,
    // so that one copy uploads a call's header and weights
    int64_t *fresh = (int64_t *)dev_alloc(ctx, (3 + size_t(nsteps)) * sizeof(int64_t));
    if (!fresh) return fail(ctx, IC_ERR_OOM, "weights buffer");
    IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    IC_CUDA(ctx, cudaMemcpy(fresh, ctx->d.step, 3 * sizeof(int64_t), cudaMemcpyDeviceToDevice));
    dev_free(ctx, ctx->d.step);
    ctx->d.step = fresh;
    ctx->d.weights = reinterpret_cast<double *>(fresh + 3);
    cudaFreeHost(ctx->staging);
    ctx->staging = nullptr;
    IC_CUDA(ctx, cudaMallocHost(&ctx->staging, (size_t(nsteps) + 3) * sizeof(double)));
    ctx->weights_cap = nsteps;
    invalidate_graphs(ctx);
  }
  if (w || ctx->host_wcount != 0) {
    IC_CUDA(ctx, cudaEventSynchronize(ctx->staging_done));   // previous upload has left the staging buffer
    const int64_t hdr[2] = {ctx->host_step, w ? int64_t(nsteps) : 0};
    std::memcpy(ctx->staging, hdr, sizeof(hdr));
    size_t bytes = sizeof(hdr);
    if (w) {   // the weights follow the header in the device block too
      std::memcpy(ctx->staging + 2, w, size_t(nsteps) * sizeof(double));
      bytes += size_t(nsteps) * sizeof(double);
    }
    IC_CUDA(ctx, cudaMemcpyAsync(ctx->d.step + 1, ctx->staging, bytes, cudaMemcpyHostToDevice, ctx->stream));
    IC_CUDA(ctx, cudaEventRecord(ctx->staging_done, ctx->stream));
    ctx->host_wcount = w ? nsteps : 0;
  }
  return IC_OK;
}

ic_status upload_drive(ic_ctx *ctx, int64_t step) {
  double d[3];
  ic::drive_amplitudes(ctx, step, d);
  const float f[3] = {float(d[0]), float(d[1]), float(d[2])};
  IC_CUDA(ctx, cudaMemcpy(ctx->drive, d, sizeof(d), cudaMemcpyHostToDevice));
  IC_CUDA(ctx, cudaMemcpy(ctx->drive_f, f, sizeof(f), cudaMemcpyHostToDevice));
  return IC_OK;
}

// One step on the context's stream: its CUDA graph for the current buffer
// parity (captured on first use), or the kernels one by one while profiling.
ic_status launch_one_step(ic_ctx *ctx) {
  if (graphs_enabled() && !ctx->profiling) {
    cudaGraphExec_t &g = ctx->graph[ctx->cur];
    if (!g) {
      cudaGraph_t graph;
      IC_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      const cudaError_t le = enqueue_step(ctx, ctx->cur);
      const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
      if (le != cudaSuccess) return cuda_fail(ctx, le, "kernel launch during capture");
      if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
      const cudaError_t ie = cudaGraphInstantiate(&g, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) return cuda_fail(ctx, ie, "cudaGraphInstantiate");
    }
    IC_CUDA(ctx, cudaGraphLaunch(g, ctx->stream));
  } else {
    IC_CUDA(ctx, enqueue_step(ctx, ctx->cur));
  }
  ctx->cur = 1 - ctx->cur;
  return IC_OK;
}

// FP64 fused multiply-add throughput (ic_fma64_rate): eight independent FMA
// chains per thread, enough warps to fill every SM's FP64 units.
constexpr int kFmaChains = 8;
__global__ void k_fma64(double *sink, int iters, double b, double c) {
  double a[kFmaChains];
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) a[j] = 1e-3 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) s += a[j];
  if (s == 12345.6789) sink[0] = s;   // never true for these inputs; keeps the chains live
}

// Philox4x32-10 of n counter/key pairs (ic_philox4x32_10): the device code of
// the noise and thermal draws, evaluated on given inputs.
__global__ void k_philox_eval(int n, const uint32_t *in, uint32_t *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t *w = in + 6 * size_t(i);
  const uint4 r = ic::philox4x32_10(make_uint4(w[0], w[1], w[2], w[3]), w[4], w[5]);
  uint32_t *o = out + 4 * size_t(i);
  o[0] = r.x;
  o[1] = r.y;
  o[2] = r.z;
  o[3] = r.w;
}

}  // namespace

extern "C" {

ic_status ic_create_grid(const ic_grid_params *params, ic_ctx **out) {
  if (!params || !out) return IC_ERR_ARG;
  *out = nullptr;
  const ic_grid_params &p = *params;
  if (p.nx < 6 || p.ny < 6 || p.nz < 6) return IC_ERR_ARG;
  if (!(p.h > 0) || !(p.rho0 > 0) || !(p.c > 0) || !(p.dt > 0) || p.eta < 0 || p.zeta < 0 || p.kT < 0)
    return IC_ERR_ARG;
  if (p.precision != IC_FP64 && p.precision != IC_FP32) return IC_ERR_ARG;
  if (p.forcing < IC_FORCE_NONE || p.forcing > IC_FORCE_PLANE || p.wave_axis < 0 || p.wave_axis > 2)
    return IC_ERR_ARG;
  if ((int64_t)p.nx * p.ny * p.nz >= (int64_t(1) << 32)) return IC_ERR_ARG;   // Philox cell counter is 32-bit
  if ((p.alloc == nullptr) != (p.free == nullptr)) return IC_ERR_ARG;
  const int n_ax = p.wave_axis == 0 ? p.nx : (p.wave_axis == 1 ? p.ny : p.nz);
  if (p.wave_nlambda < 1 || p.plane_index < 0 || p.plane_index >= n_ax) return IC_ERR_ARG;

  ic_ctx *ctx = new ic_ctx();
  ctx->p = p;
  ctx->cells = int64_t(p.nx) * p.ny * p.nz;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        ctx->sm_count <= 0)
      ctx->sm_count = 1;
  }
  ctx->real_size = p.precision == IC_FP32 ? 4 : 8;
  auto bail = [&](ic_status st) {
    ic_destroy(ctx);
    return st;
  };
  if (p.stream) {
    ctx->stream = static_cast<cudaStream_t>(p.stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(IC_ERR_CUDA);
    ctx->own_stream = true;
  }
  // driven mode: k, discrete k~, omega = c k~, Gamma
  const double L = n_ax * p.h;
  ctx->kwave = 2.0 * M_PI * p.wave_nlambda / L;
  const double kd = (2.0 / p.h) * std::sin(0.5 * ctx->kwave * p.h);
  ctx->omega = p.c * kd;
  const double gamma = (4.0 * p.eta / 3.0 + p.zeta) / (2.0 * p.rho0);
  ctx->force_amp = p.forcing == IC_FORCE_MODE ? 2.0 * gamma * ctx->omega * p.wave_amp
                                              : p.wave_amp * n_ax * gamma * ctx->omega;

  const size_t fbytes = size_t(ctx->cells) * ctx->real_size;
  for (int b = 0; b < 3; ++b)
    for (int j = 0; j < 4; ++j) {
      ctx->U[b][j] = dev_alloc(ctx, fbytes);
      if (!ctx->U[b][j]) return bail(IC_ERR_OOM);
      if (cudaMemsetAsync(ctx->U[b][j], 0, fbytes, ctx->stream) != cudaSuccess) return bail(IC_ERR_CUDA);
    }
  ctx->pp = dev_alloc(ctx, fbytes);
  if (!ctx->pp) return bail(IC_ERR_OOM);
  if (p.kT > 0.0)
    for (int j = 0; j < (p.precision == IC_FP64 ? 18 : 12); ++j)
      if (!(ctx->noise[j] = dev_alloc(ctx, fbytes))) return bail(IC_ERR_OOM);
  if (cudaMemsetAsync(ctx->pp, 0, fbytes, ctx->stream) != cudaSuccess) return bail(IC_ERR_CUDA);
  ctx->n_partials = ic::fluid_num_partials(ctx);
  ctx->d.partials = (double *)dev_alloc(ctx, ctx->n_partials * sizeof(double));
  ctx->weights_cap = 1024;
  // [0] step counter, [1] step of weights[0], [2] number of weights, then the weights
  ctx->d.step = (int64_t *)dev_alloc(ctx, (3 + size_t(ctx->weights_cap)) * sizeof(int64_t));
  ctx->d.scalars = (double *)dev_alloc(ctx, 16 * sizeof(double));
  ctx->d.status = (int *)dev_alloc(ctx, 4 * sizeof(int));   // status, rebuild, bin_done, spare
  ctx->d.rebuilds = (long long *)dev_alloc(ctx, sizeof(long long));
  ctx->cos_table = (double *)dev_alloc(ctx, n_ax * sizeof(double));
  ctx->cos_table_f = (float *)dev_alloc(ctx, n_ax * sizeof(float));
  ctx->drive = (double *)dev_alloc(ctx, 3 * sizeof(double));
  ctx->drive_f = (float *)dev_alloc(ctx, 3 * sizeof(float));
  ctx->d.weights = ctx->d.step ? reinterpret_cast<double *>(ctx->d.step + 3) : nullptr;
  if (!ctx->d.partials || !ctx->d.step || !ctx->d.scalars || !ctx->d.status || !ctx->d.rebuilds || !ctx->cos_table ||
      !ctx->d.weights ||
      !ctx->cos_table_f || !ctx->drive || !ctx->drive_f)
    return bail(IC_ERR_OOM);
  if (cudaMallocHost(&ctx->staging, (ctx->weights_cap + 3) * sizeof(double)) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->staging_done, cudaEventDisableTiming) != cudaSuccess)
    return bail(IC_ERR_OOM);
  ctx->d.rebuild = ctx->d.status + 1;
  ctx->d.bin_done = ctx->d.status + 2;
  std::vector<double> tab(n_ax);
  std::vector<float> tab_f(n_ax);
  for (int i = 0; i < n_ax; ++i) {
    tab[i] = std::cos(ctx->kwave * i * p.h);
    tab_f[i] = float(tab[i]);
  }
  const int zero_rebuild[4] = {0, 1, 0, 0};
  if (upload_drive(ctx, 0) != IC_OK ||
      cudaMemcpyAsync(ctx->cos_table, tab.data(), n_ax * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) ||
      cudaMemcpyAsync(ctx->cos_table_f, tab_f.data(), n_ax * sizeof(float), cudaMemcpyHostToDevice, ctx->stream) ||
      cudaMemsetAsync(ctx->d.step, 0, (3 + size_t(ctx->weights_cap)) * sizeof(int64_t), ctx->stream) ||
      cudaMemsetAsync(ctx->d.scalars, 0, 16 * sizeof(double), ctx->stream) ||
      cudaMemsetAsync(ctx->d.rebuilds, 0, sizeof(long long), ctx->stream) ||
      cudaMemcpyAsync(ctx->d.status, zero_rebuild, sizeof(zero_rebuild), cudaMemcpyHostToDevice, ctx->stream) ||
      cudaStreamSynchronize(ctx->stream))
    return bail(IC_ERR_CUDA);
  // Deterministic FP32 boxes whose rows the whole-row stage kernel takes start
  // on it when its CTAs march runs of at least 8 planes (measured faster at
  // 128^3, 13 planes a CTA; slower at 64^3, 3); with noise the column-tile
  // kernels are the default
  if (p.kT == 0.0 && ic::rows_eligible(p) && ic::rows_buffers_aligned(ctx) &&
      ic::rows_mean_run(p, ctx->sm_count) >= 8.0)
    ctx->tile_variant = ic::kTileRows;
  // a state of rho = rho0 is delta rho = 0: the buffers are already zero
  *out = ctx;
  return IC_OK;
}

ic_status ic_set_state(ic_ctx *ctx, const double *rho, const double *gx, const double *gy, const double *gz) {
  if (!ctx || !rho) return IC_ERR_ARG;
  const size_t n = size_t(ctx->cells);
  ic_status st = upload_real(ctx, ctx->U[ctx->cur][0], rho, ctx->p.rho0, n);
  if (st) return st;
  const double *g[3] = {gx, gy, gz};
  for (int a = 0; a < 3; ++a) {
    if (g[a]) {
      st = upload_real(ctx, ctx->U[ctx->cur][1 + a], g[a], 0.0, n);
      if (st) return st;
    } else {
      IC_CUDA(ctx, cudaMemsetAsync(ctx->U[ctx->cur][1 + a], 0, n * ctx->real_size, ctx->stream));
    }
  }
  return IC_OK;
}

ic_status ic_get_state(ic_ctx *ctx, double *rho, double *gx, double *gy, double *gz) {
  if (!ctx) return IC_ERR_ARG;
  const size_t n = size_t(ctx->cells);
  double *dst[4] = {rho, gx, gy, gz};
  for (int j = 0; j < 4; ++j) {
    if (!dst[j]) continue;
    ic_status st = download_real(ctx, dst[j], ctx->U[ctx->cur][j], j == 0 ? ctx->p.rho0 : 0.0, n);
    if (st) return st;
  }
  return check_device_status(ctx);
}

ic_status ic_init_thermal(ic_ctx *ctx, uint64_t seed, int add) {
  if (!ctx) return IC_ERR_ARG;
  if (!(ctx->p.kT > 0)) return fail(ctx, IC_ERR_STATE, "ic_init_thermal needs kT > 0");
  IC_CUDA(ctx, ic::launch_thermal(ctx, seed, add));
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return IC_OK;
}

ic_status ic_add_particles(ic_ctx *ctx, int n, const double *q, const double *u, const double *m_e,
                           const double *kappa_ratio, const double *k_spring, int *first_id) {
  if (!ctx || n < 0 || (n > 0 && (!q || !m_e || !kappa_ratio))) return IC_ERR_ARG;
  if (n == 0) return IC_OK;
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const ic_grid_params &p = ctx->p;
  const double L[3] = {p.nx * p.h, p.ny * p.h, p.nz * p.h};
  for (int i = 0; i < n; ++i) {
    if (!(kappa_ratio[i] > 0)) return fail(ctx, IC_ERR_ARG, "kappa_ratio[%d] must be > 0", i);
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(q[3 * i + a])) return fail(ctx, IC_ERR_ARG, "q[%d] is not finite", i);
  }
  const int first = ctx->ps.n;
  ic_status st = grow_particles(ctx, first + n);
  if (st) return st;
  ic::ParticleStore &s = ctx->ps;
  std::vector<double> qw(3 * n), eps(n), ks(n, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      double x = std::fmod(q[3 * i + a], L[a]);
      if (x < 0) x += L[a];
      if (x >= L[a]) x -= L[a];
      qw[3 * i + a] = x;
    }
    eps[i] = p.c * p.c * (1.0 / kappa_ratio[i] - 1.0);   // epsilon_pf, Eqs. (part_svel), (ke)
    if (k_spring) ks[i] = k_spring[i];
    if (ks[i] != 0.0) ctx->any_spring = true;
  }
  const size_t r = ctx->real_size;
  std::vector<long long> qdev(3 * size_t(n));   // 8 bytes per component in both representations
  ic::positions_to_device(ctx, qw.data(), 3 * size_t(n), qdev.data());
  IC_CUDA(ctx, cudaMemcpy((char *)s.q + 24 * size_t(first), qdev.data(), 24 * size_t(n), cudaMemcpyHostToDevice));
  IC_CUDA(ctx, cudaMemcpy((char *)s.q_eq + 24 * size_t(first), qdev.data(), 24 * size_t(n), cudaMemcpyHostToDevice));
  IC_CUDA(ctx, cudaMemcpy((char *)s.q_build + 24 * size_t(first), qdev.data(), 24 * size_t(n),
                          cudaMemcpyHostToDevice));
  st = upload_real(ctx, (char *)s.m_e + r * first, m_e, 0.0, n);
  if (!st) st = upload_real(ctx, (char *)s.eps + r * first, eps.data(), 0.0, n);
  if (!st) st = upload_real(ctx, (char *)s.k_s + r * first, ks.data(), 0.0, n);
  if (!st && u) st = upload_real(ctx, (char *)s.u + 3 * r * first, u, 0.0, 3 * size_t(n));
  if (st) return st;
  s.n = first + n;
  if (!u) {
    IC_CUDA(ctx, ic::launch_particle_velocity(ctx, first, n, ctx->U[ctx->cur]));
  }
  const int one = 1;
  IC_CUDA(ctx, cudaMemcpyAsync(ctx->d.rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  IC_CUDA(ctx, ic::launch_particle_bins(ctx));
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  invalidate_graphs(ctx);
  if (first_id) *first_id = first;
  return IC_OK;
}

ic_status ic_step(ic_ctx *ctx, int nsteps, const double *w) {
  if (!ctx || nsteps < 0) return IC_ERR_ARG;
  if (nsteps == 0) return IC_OK;
  const ic::TraceRange tr("ic_step");
  {
    const ic_status st = upload_weights(ctx, nsteps, w);
    if (st) return st;
  }
  for (int i = 0; i < nsteps; ++i) {
    const ic_status st = launch_one_step(ctx);
    if (st) return st;
  }
  ctx->host_step += nsteps;
  return IC_OK;
}

ic_status ic_sync(ic_ctx *ctx) {
  if (!ctx) return IC_ERR_ARG;
  return check_device_status(ctx);
}

ic_status ic_forces(ic_ctx *ctx, double *lambda, double *u, double *q) {
  if (!ctx) return IC_ERR_ARG;
  // one pinned staging area, all copies queued, one synchronisation
  const size_t n3 = 3 * size_t(ctx->ps.n), rb = n3 * ctx->real_size, need = 2 * rb + 8 * n3 + sizeof(int);
  if (need > ctx->download_cap) {
    if (ctx->download) cudaFreeHost(ctx->download);
    ctx->download = nullptr;
    ctx->download_cap = 0;
    IC_CUDA(ctx, cudaMallocHost(&ctx->download, need));
    ctx->download_cap = need;
  }
  unsigned char *h_lam = ctx->download, *h_u = h_lam + rb, *h_q = h_u + rb, *h_st = h_q + 8 * n3;
  if (n3) {
    if (lambda) IC_CUDA(ctx, cudaMemcpyAsync(h_lam, ctx->ps.lam, rb, cudaMemcpyDeviceToHost, ctx->stream));
    if (u) IC_CUDA(ctx, cudaMemcpyAsync(h_u, ctx->ps.u, rb, cudaMemcpyDeviceToHost, ctx->stream));
    if (q) IC_CUDA(ctx, cudaMemcpyAsync(h_q, ctx->ps.q, 8 * n3, cudaMemcpyDeviceToHost, ctx->stream));
  }
  IC_CUDA(ctx, cudaMemcpyAsync(h_st, ctx->d.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (n3) {
    for (int j = 0; j < 2; ++j) {
      double *dst = j == 0 ? lambda : u;
      const unsigned char *src = j == 0 ? h_lam : h_u;
      if (!dst) continue;
      if (ctx->p.precision == IC_FP32)
        from_real<float>(src, 0.0, dst, n3);
      else
        from_real<double>(src, 0.0, dst, n3);
    }
    if (q) ic::positions_to_host(ctx, h_q, n3, q);
  }
  int st = 0;
  std::memcpy(&st, h_st, sizeof(int));
  return status_error(ctx, st);
}

ic_status ic_forces_async(ic_ctx *ctx, int slot) {
  if (!ctx || slot < 0 || slot > 1) return IC_ERR_ARG;
  const size_t n3 = 3 * size_t(ctx->ps.n), rb = n3 * ctx->real_size, need = rb + sizeof(int);
  if (!ctx->fetch_done[slot]) IC_CUDA(ctx, cudaEventCreateWithFlags(&ctx->fetch_done[slot], cudaEventDisableTiming));
  if (need > ctx->fetch_cap[slot]) {
    IC_CUDA(ctx, cudaEventSynchronize(ctx->fetch_done[slot]));   // an earlier copy into the old buffer
    if (ctx->fetch[slot]) cudaFreeHost(ctx->fetch[slot]);
    ctx->fetch[slot] = nullptr;
    ctx->fetch_cap[slot] = 0;
    IC_CUDA(ctx, cudaMallocHost(&ctx->fetch[slot], need));
    ctx->fetch_cap[slot] = need;
  }
  // with particles one copy: lambda and, after it, the status word as the
  // last step's final substep left it
  if (n3)
    IC_CUDA(ctx, cudaMemcpyAsync(ctx->fetch[slot], ctx->ps.lam, rb + sizeof(int), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  else
    IC_CUDA(ctx, cudaMemcpyAsync(ctx->fetch[slot] + rb, ctx->d.status, sizeof(int), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  IC_CUDA(ctx, cudaEventRecord(ctx->fetch_done[slot], ctx->stream));
  ctx->fetch_n[slot] = ctx->ps.n;
  return IC_OK;
}

ic_status ic_forces_collect(ic_ctx *ctx, int slot, double *lambda) {
  if (!ctx || slot < 0 || slot > 1) return IC_ERR_ARG;
  if (ctx->fetch_n[slot] < 0) return fail(ctx, IC_ERR_STATE, "no read-back queued in slot %d", slot);
  IC_CUDA(ctx, cudaEventSynchronize(ctx->fetch_done[slot]));
  const size_t n3 = 3 * size_t(ctx->fetch_n[slot]), rb = n3 * ctx->real_size;
  ctx->fetch_n[slot] = -1;
  if (lambda && n3) {
    if (ctx->p.precision == IC_FP32)
      from_real<float>(ctx->fetch[slot], 0.0, lambda, n3);
    else
      from_real<double>(ctx->fetch[slot], 0.0, lambda, n3);
  }
  int st = 0;
  std::memcpy(&st, ctx->fetch[slot] + rb, sizeof(int));
  return status_error(ctx, st);
}

ic_status ic_fma64_rate(int iters, double *flops_per_s, double *seconds) {
  if (iters <= 0 || !flops_per_s) return IC_ERR_ARG;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return IC_ERR_CUDA;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return IC_ERR_CUDA;
  double *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ic_status rc = IC_OK;
  const int blocks = 8 * sms, threads = 256;
  float ms = 0.0f;
  if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = IC_ERR_CUDA;
  } else {
    k_fma64<<<blocks, threads, 0, st>>>(sink, iters / 8 + 1, 1.0000001, 1e-9);   // warm-up
    cudaEventRecord(e0, st);
    k_fma64<<<blocks, threads, 0, st>>>(sink, iters, 1.0000001, 1e-9);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f)
      rc = IC_ERR_CUDA;
  }
  if (rc == IC_OK) {
    const double flops = 2.0 * kFmaChains * double(iters) * blocks * threads;
    *flops_per_s = flops / (1e-3 * ms);
    if (seconds) *seconds = 1e-3 * ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  cudaStreamDestroy(st);
  return rc;
}

ic_status ic_philox4x32_10(int n, const uint32_t *in, uint32_t *out) {
  if (n < 0 || (n > 0 && (!in || !out))) return IC_ERR_ARG;
  if (n == 0) return IC_OK;
  uint32_t *d_in = nullptr, *d_out = nullptr;
  if (cudaMalloc(&d_in, size_t(n) * 6 * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&d_out, size_t(n) * 4 * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_in);
    return IC_ERR_OOM;
  }
  cudaError_t e = cudaMemcpy(d_in, in, size_t(n) * 6 * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_philox_eval<<<(n + 127) / 128, 128>>>(n, d_in, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, size_t(n) * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_out);
  return e == cudaSuccess ? IC_OK : IC_ERR_CUDA;
}

ic_status ic_particle_density(ic_ctx *ctx, double *jrho) {
  if (!ctx || !jrho) return IC_ERR_ARG;
  if (ctx->ps.n > 0) {
    ic_status st = download_real(ctx, jrho, ctx->ps.jrho, 0.0, size_t(ctx->ps.n));
    if (st) return st;
  }
  return check_device_status(ctx);
}

ic_status ic_time_average(ic_ctx *ctx, double *f_spring, double *lambda, double *a2, int reset) {
  if (!ctx) return IC_ERR_ARG;
  double sc[2];
  IC_CUDA(ctx, cudaMemcpyAsync(sc, ctx->d.scalars, sizeof(sc), cudaMemcpyDeviceToHost, ctx->stream));
  const size_t n = size_t(ctx->ps.n);
  std::vector<double> acc(6 * n);
  if (n) IC_CUDA(ctx, cudaMemcpyAsync(acc.data(), ctx->ps.acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                      ctx->stream));
  ic_status st = check_device_status(ctx);
  if (st) return st;
  if (!(sc[0] != 0.0)) return fail(ctx, IC_ERR_STATE, "time-average weights sum to zero");
  for (size_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      if (f_spring) f_spring[3 * i + a] = acc[6 * i + a] / sc[0];
      if (lambda) lambda[3 * i + a] = acc[6 * i + 3 + a] / sc[0];
    }
  if (a2) *a2 = sc[1] / sc[0];
  if (reset) {
    IC_CUDA(ctx, cudaMemsetAsync(ctx->d.scalars, 0, 2 * sizeof(double), ctx->stream));
    if (n) IC_CUDA(ctx, cudaMemsetAsync(ctx->ps.acc, 0, acc.size() * sizeof(double), ctx->stream));
    IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return IC_OK;
}

ic_status ic_objective(ic_ctx *ctx, const double *direction, double *phi, int reset) {
  if (!ctx || !phi) return IC_ERR_ARG;
  const size_t n = size_t(ctx->ps.n);
  std::vector<double> f(3 * n);
  const ic_status st = ic_time_average(ctx, n ? f.data() : nullptr, nullptr, nullptr, reset);
  if (st) return st;
  // Phi = sum_p d_p . <F_p>_w, particles in index order, components x, y, z
  double s = 0.0;
  for (size_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) s += (direction ? direction[3 * i + a] : (a == 0 ? 1.0 : 0.0)) * f[3 * i + a];
  *phi = s;
  return IC_OK;
}

int ic_bounds_check_build(void) {
#ifdef IC_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

ic_status ic_bounds_selftest(void) {
  ic::bounds_flag_fluid();   // clear
  if (ic::launch_bounds_probe(nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return IC_ERR_CUDA;
  const unsigned f = ic::bounds_flag_fluid();
  return ic_bounds_check_build() && f == 1u ? IC_OK : IC_ERR_STATE;
}

ic_status ic_neighbour_rebuilds(ic_ctx *ctx, int64_t *count) {
  if (!ctx || !count) return IC_ERR_ARG;
  long long v = 0;
  IC_CUDA(ctx, cudaMemcpyAsync(&v, ctx->d.rebuilds, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *count = v;
  return IC_OK;
}

ic_status ic_stats(ic_ctx *ctx, double *p_total, double *mode_amp, int64_t *step) {
  if (!ctx) return IC_ERR_ARG;
  double *sums = ctx->d.scalars + 8;
  IC_CUDA(ctx, ic::launch_field_sums(ctx, ctx->U[ctx->cur], sums));
  IC_CUDA(ctx, cudaMemsetAsync(ctx->d.scalars + 12, 0, 3 * sizeof(double), ctx->stream));
  if (ctx->ps.n > 0) IC_CUDA(ctx, ic::launch_particle_momentum(ctx, ctx->d.scalars + 12));
  double h[7];
  IC_CUDA(ctx, cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  ic_status st = check_device_status(ctx);
  if (st) return st;
  const double vol = ctx->p.h * ctx->p.h * ctx->p.h;
  if (p_total)
    for (int a = 0; a < 3; ++a) p_total[a] = vol * h[a] + h[4 + a];
  if (mode_amp) *mode_amp = 2.0 * h[3] / double(ctx->cells);
  if (step) *step = ctx->host_step;
  return IC_OK;
}

// ----------------------------------------------------------- checkpointing
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version, precision, nx, ny, nz, np;
  int64_t step;
  double scalars[3];
};

size_t ckpt_size_for(const ic_ctx *ctx, size_t n) {
  const size_t r = ctx->real_size;
  return sizeof(CkptHeader) + 4 * size_t(ctx->cells) * r + n * (24 + 24 + 48) + n * r * (3 + 1 + 1 + 1 + 3 + 3);
}
size_t ckpt_size(const ic_ctx *ctx) { return ckpt_size_for(ctx, size_t(ctx->ps.n)); }
}  // namespace

ic_status ic_checkpoint(ic_ctx *ctx, void *buf, size_t *bytes) {
  if (!ctx || !bytes) return IC_ERR_ARG;
  const size_t need = ckpt_size(ctx);
  if (!buf) {
    *bytes = need;
    return IC_OK;
  }
  if (*bytes < need) return fail(ctx, IC_ERR_ARG, "checkpoint buffer too small (%zu < %zu)", *bytes, need);
  ic_status st = check_device_status(ctx);
  if (st) return st;
  CkptHeader hd{};
  std::memcpy(hd.magic, "ICCKPT1", 8);
  hd.version = 1;
  hd.precision = ctx->p.precision;
  hd.nx = ctx->p.nx;
  hd.ny = ctx->p.ny;
  hd.nz = ctx->p.nz;
  hd.np = ctx->ps.n;
  hd.step = ctx->host_step;
  IC_CUDA(ctx, cudaMemcpy(hd.scalars, ctx->d.scalars, sizeof(hd.scalars), cudaMemcpyDeviceToHost));
  char *out = static_cast<char *>(buf);
  std::memcpy(out, &hd, sizeof(hd));
  out += sizeof(hd);
  const size_t r = ctx->real_size, fb = size_t(ctx->cells) * r, n = size_t(ctx->ps.n);
  for (int j = 0; j < 4; ++j, out += fb) IC_CUDA(ctx, cudaMemcpy(out, ctx->U[ctx->cur][j], fb, cudaMemcpyDeviceToHost));
  const ic::ParticleStore &s = ctx->ps;
  struct Item {
    const void *src;
    size_t len;
  } items[] = {{s.q, 24 * n},     {s.q_eq, 24 * n},  {s.acc, 48 * n},   {s.u, 3 * r * n}, {s.m_e, r * n},
               {s.eps, r * n},    {s.k_s, r * n},    {s.force, 3 * r * n}, {s.lam, 3 * r * n}};
  for (const Item &it : items) {
    if (it.len) IC_CUDA(ctx, cudaMemcpy(out, it.src, it.len, cudaMemcpyDeviceToHost));
    out += it.len;
  }
  *bytes = need;
  return IC_OK;
}

ic_status ic_restore(ic_ctx *ctx, const void *buf, size_t bytes) {
  if (!ctx || !buf || bytes < sizeof(CkptHeader)) return IC_ERR_ARG;
  CkptHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, "ICCKPT1", 8) != 0 || hd.version != 1)
    return fail(ctx, IC_ERR_ARG, "not a libic checkpoint");
  if (hd.precision != ctx->p.precision || hd.nx != ctx->p.nx || hd.ny != ctx->p.ny || hd.nz != ctx->p.nz)
    return fail(ctx, IC_ERR_ARG, "checkpoint grid or precision differs from this context");
  // checked before anything of the context changes: a rejected blob leaves it as it was
  if (hd.np < 0 || bytes < ckpt_size_for(ctx, size_t(hd.np))) return fail(ctx, IC_ERR_ARG, "checkpoint truncated");
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int n_before = ctx->ps.n;
  ctx->ps.n = 0;
  ic_status st = grow_particles(ctx, hd.np);
  if (st) {
    ctx->ps.n = n_before;
    return st;
  }
  ctx->ps.n = hd.np;
  const char *in = static_cast<const char *>(buf) + sizeof(hd);
  ctx->cur = 0;
  const size_t r = ctx->real_size, fb = size_t(ctx->cells) * r, n = size_t(hd.np);
  for (int j = 0; j < 4; ++j, in += fb) IC_CUDA(ctx, cudaMemcpy(ctx->U[0][j], in, fb, cudaMemcpyHostToDevice));
  ic::ParticleStore &s = ctx->ps;
  struct Item {
    void *dst;
    size_t len;
  } items[] = {{s.q, 24 * n},     {s.q_eq, 24 * n},  {s.acc, 48 * n},   {s.u, 3 * r * n}, {s.m_e, r * n},
               {s.eps, r * n},    {s.k_s, r * n},    {s.force, 3 * r * n}, {s.lam, 3 * r * n}};
  for (const Item &it : items) {
    if (it.len) IC_CUDA(ctx, cudaMemcpy(it.dst, in, it.len, cudaMemcpyHostToDevice));
    in += it.len;
  }
  if (n) IC_CUDA(ctx, cudaMemcpy(s.q_build, s.q, 24 * n, cudaMemcpyDeviceToDevice));
  IC_CUDA(ctx, cudaMemset(ctx->pp, 0, fb));
  {
    // a tether anywhere switches the stage force source on
    const char *ks = static_cast<const char *>(buf) + sizeof(hd) + 4 * fb + n * (24 + 24 + 48) + n * r * (3 + 1 + 1);
    ctx->any_spring = false;
    for (size_t i = 0; i < n; ++i) {
      double v = (r == 4) ? double(reinterpret_cast<const float *>(ks)[i]) : reinterpret_cast<const double *>(ks)[i];
      if (v != 0.0) ctx->any_spring = true;
    }
  }
  ctx->host_step = hd.step;
  ctx->host_wcount = 0;
  const int64_t steps[3] = {hd.step, hd.step, 0};
  IC_CUDA(ctx, cudaMemcpy(ctx->d.step, steps, sizeof(steps), cudaMemcpyHostToDevice));
  IC_CUDA(ctx, cudaMemcpy(ctx->d.scalars, hd.scalars, sizeof(hd.scalars), cudaMemcpyHostToDevice));
  {
    const ic_status st3 = upload_drive(ctx, hd.step);
    if (st3) return st3;
  }
  const int st2[2] = {0, 1};
  IC_CUDA(ctx, cudaMemcpy(ctx->d.status, st2, sizeof(st2), cudaMemcpyHostToDevice));
  IC_CUDA(ctx, ic::launch_particle_bins(ctx));
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  invalidate_graphs(ctx);
  return IC_OK;
}

}  // extern "C"

// ------------------------------------------------------------- adjoint
namespace {

// FP64 words per particle of the adjoint's particle block: qbar, ubar, qhbar,
// fbar, jvnh and the objective direction (3 each), the m_e and epsilon
// gradients (1 each); one word more holds the amplitude gradient.
constexpr size_t kAdjWordsPerParticle = 6 * 3 + 2;

ic_status adjoint_zero(ic_ctx *ctx, const double *direction) {
  ic::AdjointStore &A = ctx->adj;
  const size_t fb = size_t(ctx->cells) * ctx->real_size, n = size_t(A.np);
  for (int j = 0; j < 4; ++j) IC_CUDA(ctx, cudaMemsetAsync(A.bar[j], 0, fb, ctx->stream));
  IC_CUDA(ctx, cudaMemsetAsync(A.part_block, 0, (kAdjWordsPerParticle * n + 1) * sizeof(double), ctx->stream));
  std::vector<double> dir(3 * n, 0.0);
  for (size_t i = 0; i < n; ++i) {
    if (direction)
      for (int a = 0; a < 3; ++a) dir[3 * i + a] = direction[3 * i + a];
    else
      dir[3 * i] = 1.0;
  }
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (n) IC_CUDA(ctx, cudaMemcpy(A.dir, dir.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice));
  A.rec_cur = -1;
  return IC_OK;
}

ic_status adjoint_ready(ic_ctx *ctx) {
  if (!ctx->adj.on) return fail(ctx, IC_ERR_STATE, "ic_adjoint_enable has not been called");
  if (ctx->adj.np != ctx->ps.n)
    return fail(ctx, IC_ERR_STATE, "particles were added after ic_adjoint_enable; enable it again");
  return IC_OK;
}

constexpr uint64_t kSnapMagic = 0x31504e53434943ull;   // "ICSNP1"

struct SnapHeader {
  uint64_t magic;
  int64_t step;
  int32_t np, precision, nx, ny, nz, pad;
  uint64_t pad2[3];
};
static_assert(sizeof(SnapHeader) == 64, "snapshot header is 64 bytes");

__global__ void k_snapshot_header(SnapHeader *out, uint64_t magic, int64_t step, int np, int precision, int nx,
                                  int ny, int nz) {
  SnapHeader h{};
  h.magic = magic;
  h.step = step;
  h.np = np;
  h.precision = precision;
  h.nx = nx;
  h.ny = ny;
  h.nz = nz;
  *out = h;
}

__global__ void k_snapshot_restart(int64_t *step, int64_t n, int *rebuild, double *drive, float *drive_f, double d0,
                                   double d1, double d2) {
  step[0] = n;
  step[1] = n;
  step[2] = 0;
  *rebuild = 1;
  drive[0] = d0;
  drive[1] = d1;
  drive[2] = d2;
  drive_f[0] = float(d0);
  drive_f[1] = float(d1);
  drive_f[2] = float(d2);
}

constexpr uint64_t kTapeMagic = 0x31504154434943ull;   // "ICTAP1"

// Up to kMaxCopies device-to-device copies in one launch (lengths multiples
// of 4 bytes, addresses 4-byte aligned): block y takes copy y, its threads
// stride over the 4-byte words, 16 bytes at a time where both ends allow.
constexpr int kMaxCopies = 32;
struct CopyList {
  const char *src[kMaxCopies];
  char *dst[kMaxCopies];
  size_t len[kMaxCopies];
  int n;
};

__global__ void k_copy_list(CopyList L) {
  const int c = blockIdx.y;
  if (c >= L.n) return;
  const char *src = L.src[c];
  char *dst = L.dst[c];
  const size_t len = L.len[c];
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  const size_t t0 = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  size_t done = 0;
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    const size_t n16 = len / 16;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (size_t i = t0; i < n16; i += stride) d4[i] = s4[i];
    done = n16 * 16;
  }
  const size_t n4 = (len - done) / 4;
  const uint32_t *s1 = reinterpret_cast<const uint32_t *>(src + done);
  uint32_t *d1 = reinterpret_cast<uint32_t *>(dst + done);
  for (size_t i = t0; i < n4; i += stride) d1[i] = s1[i];
}

// The context's own buffers as the tape of the step recorded last.
ic::AdjStepTape context_tape(ic_ctx *ctx) {
  ic::AdjStepTape t{};
  const ic::AdjointStore &A = ctx->adj;
  for (int j = 0; j < 4; ++j) {
    t.Un[j] = ctx->U[A.rec_cur][j];
    t.U1[j] = A.tU1[j];
    t.U2[j] = ctx->U[2][j];
    t.Unew[j] = ctx->U[1 - A.rec_cur][j];
  }
  for (int a = 0; a < 3; ++a) t.G3[a] = A.tG3[a];
  t.q_n = A.tq;
  t.q_half = ctx->ps.q_half;
  t.u_n = A.tu;
  t.force = ctx->ps.force;
  t.dg = ctx->ps.dg;
  t.step = A.rec_step;
  return t;
}

// A caller's step tape: a 64-byte header, the 19 fields (U^n, U_1, U_2, g~,
// U^{n+1}), then q^n, q^{n+1/2}, u^n, F, dg, each 16-byte aligned.
struct TapeLayout {
  ic::AdjStepTape t;
  size_t bytes;
};

TapeLayout tape_layout(const ic_ctx *ctx, void *base) {
  const size_t fb = size_t(ctx->cells) * ctx->real_size, fs = (fb + 15) / 16 * 16, n = size_t(ctx->ps.n);
  const size_t qs = (24 * n + 15) / 16 * 16, vs = (3 * ctx->real_size * n + 15) / 16 * 16;
  char *p = static_cast<char *>(base);
  TapeLayout L{};
  size_t off = sizeof(SnapHeader);
  auto take = [&](size_t len) {
    void *at = p ? p + off : nullptr;
    off += len;
    return at;
  };
  for (int j = 0; j < 4; ++j) L.t.Un[j] = take(fs);
  for (int j = 0; j < 4; ++j) L.t.U1[j] = take(fs);
  for (int j = 0; j < 4; ++j) L.t.U2[j] = take(fs);
  for (int a = 0; a < 3; ++a) L.t.G3[a] = take(fs);
  for (int j = 0; j < 4; ++j) L.t.Unew[j] = take(fs);
  L.t.q_n = take(qs);
  L.t.q_half = take(qs);
  L.t.u_n = take(vs);
  L.t.force = take(vs);
  L.t.dg = take(vs);
  L.bytes = off;
  return L;
}

size_t snapshot_bytes(const ic_ctx *ctx) {
  const size_t fb = size_t(ctx->cells) * ctx->real_size, n = size_t(ctx->ps.n);
  return sizeof(SnapHeader) + 4 * ((fb + 15) / 16 * 16) + (24 * n + 15) / 16 * 16 + 3 * ctx->real_size * n;
}

}  // namespace

extern "C" {

ic_status ic_adjoint_enable(ic_ctx *ctx) {
  if (!ctx) return IC_ERR_ARG;
  if (ctx->p.kT != 0.0) return fail(ctx, IC_ERR_STATE, "the adjoint covers the deterministic step (kT = 0)");
  ic::AdjointStore &A = ctx->adj;
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  invalidate_graphs(ctx);   // the reverse-step graphs point at the buffers freed here
  dev_free(ctx, A.grid_block);
  dev_free(ctx, A.part_block);
  A = ic::AdjointStore{};
  const size_t fb = size_t(ctx->cells) * ctx->real_size, n = size_t(ctx->ps.n);
  const size_t fstride = (fb + 255) / 256 * 256;
  constexpr int kFields = 29;
  const size_t tape_q = (24 * n + 255) / 256 * 256;
  char *g = static_cast<char *>(dev_alloc(ctx, kFields * fstride + tape_q + 3 * ctx->real_size * n));
  double *pd = static_cast<double *>(dev_alloc(ctx, (kAdjWordsPerParticle * n + 1) * sizeof(double)));
  if (!g || !pd) {
    dev_free(ctx, g);
    dev_free(ctx, pd);
    return fail(ctx, IC_ERR_OOM, "adjoint buffers");
  }
  IC_CUDA(ctx, cudaMemsetAsync(g, 0, kFields * fstride, ctx->stream));
  A.grid_block = g;
  A.part_block = pd;
  void **slots[kFields] = {&A.tU1[0], &A.tU1[1], &A.tU1[2], &A.tU1[3], &A.tG3[0], &A.tG3[1], &A.tG3[2],
                           &A.bar[0], &A.bar[1], &A.bar[2], &A.bar[3], &A.acc[0], &A.acc[1], &A.acc[2],
                           &A.acc[3], &A.vbar[0], &A.vbar[1], &A.vbar[2], &A.gpart[0], &A.gpart[1],
                           &A.gpart[2], &A.rfbar[0], &A.rfbar[1], &A.rfbar[2], &A.pibar, &A.rhox,
                           &A.vel[0],  &A.vel[1],  &A.vel[2]};
  for (int k = 0; k < kFields; ++k) *slots[k] = g + k * fstride;
  A.tq = g + kFields * fstride;
  A.tu = g + kFields * fstride + tape_q;
  double **ps[8] = {&A.qbar, &A.ubar, &A.qhbar, &A.fbar, &A.jvnh, &A.dir, &A.gme, &A.geps};
  const size_t len[8] = {3 * n, 3 * n, 3 * n, 3 * n, 3 * n, 3 * n, n, n};
  size_t off = 0;
  for (int k = 0; k < 8; ++k) {
    *ps[k] = pd + off;
    off += len[k];
  }
  A.gA = pd + off;
  if (off != kAdjWordsPerParticle * n) return fail(ctx, IC_ERR_STATE, "adjoint particle block layout");
  A.np = int(n);
  A.on = true;
  return adjoint_zero(ctx, nullptr);
}

ic_status ic_adjoint_reset(ic_ctx *ctx, const double *direction) {
  if (!ctx) return IC_ERR_ARG;
  const ic_status st = adjoint_ready(ctx);
  if (st) return st;
  return adjoint_zero(ctx, direction);
}

ic_status ic_step_record(ic_ctx *ctx) {
  const ic::TraceRange tr("ic_step_record");
  if (!ctx) return IC_ERR_ARG;
  ic_status st = adjoint_ready(ctx);
  if (st) return st;
  st = upload_weights(ctx, 1, nullptr);
  if (st) return st;
  const int cur = ctx->cur;
  IC_CUDA(ctx, enqueue_step(ctx, cur, true));
  ctx->adj.rec_cur = cur;
  ctx->adj.rec_step = ctx->host_step;
  ctx->cur = 1 - cur;
  ctx->host_step += 1;
  return IC_OK;
}

ic_status ic_adjoint_step(ic_ctx *ctx, double weight) {
  const ic::TraceRange tr("ic_adjoint_step");
  if (!ctx) return IC_ERR_ARG;
  const ic_status st = adjoint_ready(ctx);
  if (st) return st;
  if (ctx->adj.rec_cur < 0) return fail(ctx, IC_ERR_STATE, "no recorded step to reverse (call ic_step_record)");
  if (ctx->adj.rec_cur != 1 - ctx->cur)
    return fail(ctx, IC_ERR_STATE, "the state moved on after ic_step_record; record the step again");
  IC_CUDA(ctx, run_adjoint_step(ctx, context_tape(ctx), weight));
  ctx->adj.rec_cur = -1;
  return IC_OK;
}

ic_status ic_tape_size(const ic_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return IC_ERR_ARG;
  *bytes = tape_layout(ctx, nullptr).bytes;
  return IC_OK;
}

ic_status ic_step_record_tape(ic_ctx *ctx, void *dev_buf) {
  const ic::TraceRange tr("ic_step_record_tape");
  if (!ctx || !dev_buf || (reinterpret_cast<uintptr_t>(dev_buf) & 15)) return IC_ERR_ARG;
  ic_status st = ic_step_record(ctx);
  if (st) return st;
  // the recorded step's states and particle arrays, copied out before the next step overwrites them
  const ic::AdjStepTape src = context_tape(ctx);
  const TapeLayout L = tape_layout(ctx, dev_buf);
  const size_t fb = size_t(ctx->cells) * ctx->real_size, n = size_t(ctx->ps.n), r = ctx->real_size;
  // all 24 copies in one launch (the host issues one call instead of 24)
  CopyList cl{};
  auto cp = [&](void *dst, const void *from, size_t len) {
    if (!len) return;
    cl.src[cl.n] = static_cast<const char *>(from);
    cl.dst[cl.n] = static_cast<char *>(dst);
    cl.len[cl.n] = len;
    ++cl.n;
  };
  for (int j = 0; j < 4; ++j) {
    cp(L.t.Un[j], src.Un[j], fb);
    cp(L.t.U1[j], src.U1[j], fb);
    cp(L.t.U2[j], src.U2[j], fb);
    cp(L.t.Unew[j], src.Unew[j], fb);
  }
  for (int a = 0; a < 3; ++a) cp(L.t.G3[a], src.G3[a], fb);
  cp(const_cast<void *>(L.t.q_n), src.q_n, 24 * n);
  cp(const_cast<void *>(L.t.q_half), src.q_half, 24 * n);
  cp(const_cast<void *>(L.t.u_n), src.u_n, 3 * r * n);
  cp(const_cast<void *>(L.t.force), src.force, 3 * r * n);
  cp(const_cast<void *>(L.t.dg), src.dg, 3 * r * n);
  {
    const size_t words = (fb + 15) / 16;
    const unsigned bx = unsigned(std::min<size_t>((words + 255) / 256, 64));
    k_copy_list<<<dim3(bx, unsigned(cl.n)), 256, 0, ctx->stream>>>(cl);
    IC_CUDA(ctx, cudaGetLastError());
  }
  k_snapshot_header<<<1, 1, 0, ctx->stream>>>(static_cast<SnapHeader *>(dev_buf), kTapeMagic, src.step, ctx->ps.n,
                                              ctx->p.precision, ctx->p.nx, ctx->p.ny, ctx->p.nz);
  IC_CUDA(ctx, cudaGetLastError());
  ctx->tapes[reinterpret_cast<uintptr_t>(dev_buf)] = {src.step, ctx->ps.n};
  return IC_OK;
}

ic_status ic_adjoint_step_tape(ic_ctx *ctx, const void *dev_buf, double weight) {
  const ic::TraceRange tr("ic_adjoint_step_tape");
  if (!ctx || !dev_buf || (reinterpret_cast<uintptr_t>(dev_buf) & 15)) return IC_ERR_ARG;
  ic_status st = adjoint_ready(ctx);
  if (st) return st;
  TapeLayout L = tape_layout(ctx, const_cast<void *>(dev_buf));
  const auto known = ctx->tapes.find(reinterpret_cast<uintptr_t>(dev_buf));
  if (known != ctx->tapes.end() && known->second.second == ctx->ps.n) {
    L.t.step = known->second.first;   // recorded by this context: its header is known
  } else {
    SnapHeader hd{};
    IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    IC_CUDA(ctx, cudaMemcpy(&hd, dev_buf, sizeof(hd), cudaMemcpyDeviceToHost));
    if (hd.magic != kTapeMagic || hd.precision != ctx->p.precision || hd.nx != ctx->p.nx || hd.ny != ctx->p.ny ||
        hd.nz != ctx->p.nz || hd.np != ctx->ps.n)
      return fail(ctx, IC_ERR_ARG, "not a step tape of this context's grid and particles");
    L.t.step = hd.step;
  }
  IC_CUDA(ctx, run_adjoint_step(ctx, L.t, weight));
  return IC_OK;
}

ic_status ic_adjoint_read(ic_ctx *ctx, double *grad_m_e, double *grad_eps, double *grad_A, double *rho_bar,
                          double *gx_bar, double *gy_bar, double *gz_bar, double *q_bar, double *u_bar) {
  if (!ctx) return IC_ERR_ARG;
  ic_status st = adjoint_ready(ctx);
  if (st) return st;
  const ic::AdjointStore &A = ctx->adj;
  const size_t n = size_t(A.np);
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double *fields[4] = {rho_bar, gx_bar, gy_bar, gz_bar};
  for (int j = 0; j < 4; ++j)
    if (fields[j]) {
      st = download_real(ctx, fields[j], A.bar[j], 0.0, size_t(ctx->cells));
      if (st) return st;
    }
  if (grad_m_e && n) IC_CUDA(ctx, cudaMemcpy(grad_m_e, A.gme, n * sizeof(double), cudaMemcpyDeviceToHost));
  if (grad_eps && n) IC_CUDA(ctx, cudaMemcpy(grad_eps, A.geps, n * sizeof(double), cudaMemcpyDeviceToHost));
  if (grad_A) IC_CUDA(ctx, cudaMemcpy(grad_A, A.gA, sizeof(double), cudaMemcpyDeviceToHost));
  if (q_bar && n) IC_CUDA(ctx, cudaMemcpy(q_bar, A.qbar, 3 * n * sizeof(double), cudaMemcpyDeviceToHost));
  if (u_bar && n) IC_CUDA(ctx, cudaMemcpy(u_bar, A.ubar, 3 * n * sizeof(double), cudaMemcpyDeviceToHost));
  return check_device_status(ctx);
}

ic_status ic_adjoint_read_kappa(ic_ctx *ctx, double *grad_kappa_ratio) {
  if (!ctx || !grad_kappa_ratio) return IC_ERR_ARG;
  ic_status st = adjoint_ready(ctx);
  if (st) return st;
  const size_t n = size_t(ctx->adj.np);
  if (!n) return IC_OK;
  std::vector<double> geps(n), eps(n);
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  IC_CUDA(ctx, cudaMemcpy(geps.data(), ctx->adj.geps, n * sizeof(double), cudaMemcpyDeviceToHost));
  st = download_real(ctx, eps.data(), ctx->ps.eps, 0.0, n);
  if (st) return st;
  // epsilon = c^2 (kappa_f / kappa_p - 1) (Eqs. (part_svel), (ke)), so with
  // r = kappa_p / kappa_f = c^2 / (epsilon + c^2): d epsilon / d r = -c^2 / r^2
  const double c2 = ctx->p.c * ctx->p.c;
  for (size_t i = 0; i < n; ++i) {
    const double r = c2 / (eps[i] + c2);
    grad_kappa_ratio[i] = geps[i] * (-c2 / (r * r));
  }
  return check_device_status(ctx);
}

ic_status ic_snapshot_size(const ic_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return IC_ERR_ARG;
  *bytes = snapshot_bytes(ctx);
  return IC_OK;
}

ic_status ic_snapshot_save(ic_ctx *ctx, void *dev_buf) {
  if (!ctx || !dev_buf || (reinterpret_cast<uintptr_t>(dev_buf) & 15)) return IC_ERR_ARG;
  const size_t fb = size_t(ctx->cells) * ctx->real_size, fs = (fb + 15) / 16 * 16, n = size_t(ctx->ps.n);
  char *out = static_cast<char *>(dev_buf);
  // the header by a one-thread kernel: stream-ordered, no host synchronisation
  k_snapshot_header<<<1, 1, 0, ctx->stream>>>(reinterpret_cast<SnapHeader *>(out), kSnapMagic, ctx->host_step,
                                              ctx->ps.n, ctx->p.precision, ctx->p.nx, ctx->p.ny, ctx->p.nz);
  IC_CUDA(ctx, cudaGetLastError());
  out += sizeof(SnapHeader);
  for (int j = 0; j < 4; ++j, out += fs)
    IC_CUDA(ctx, cudaMemcpyAsync(out, ctx->U[ctx->cur][j], fb, cudaMemcpyDeviceToDevice, ctx->stream));
  if (n) {
    IC_CUDA(ctx, cudaMemcpyAsync(out, ctx->ps.q, 24 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    out += (24 * n + 15) / 16 * 16;
    IC_CUDA(ctx, cudaMemcpyAsync(out, ctx->ps.u, 3 * ctx->real_size * n, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  ctx->snapshots[reinterpret_cast<uintptr_t>(dev_buf)] = {ctx->host_step, ctx->ps.n};
  return IC_OK;
}

ic_status ic_snapshot_load(ic_ctx *ctx, const void *dev_buf) {
  if (!ctx || !dev_buf || (reinterpret_cast<uintptr_t>(dev_buf) & 15)) return IC_ERR_ARG;
  int64_t step = 0;
  const auto known = ctx->snapshots.find(reinterpret_cast<uintptr_t>(dev_buf));
  if (known != ctx->snapshots.end() && known->second.second == ctx->ps.n) {
    step = known->second.first;     // saved by this context: its header is known
  } else {
    SnapHeader hd{};
    IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    IC_CUDA(ctx, cudaMemcpy(&hd, dev_buf, sizeof(hd), cudaMemcpyDeviceToHost));
    if (hd.magic != kSnapMagic || hd.precision != ctx->p.precision || hd.nx != ctx->p.nx || hd.ny != ctx->p.ny ||
        hd.nz != ctx->p.nz || hd.np != ctx->ps.n)
      return fail(ctx, IC_ERR_ARG, "not a snapshot of this context's grid and particles");
    step = hd.step;
  }
  const size_t fb = size_t(ctx->cells) * ctx->real_size, fs = (fb + 15) / 16 * 16, n = size_t(ctx->ps.n);
  const char *in = static_cast<const char *>(dev_buf) + sizeof(SnapHeader);
  for (int j = 0; j < 4; ++j, in += fs)
    IC_CUDA(ctx, cudaMemcpyAsync(ctx->U[ctx->cur][j], in, fb, cudaMemcpyDeviceToDevice, ctx->stream));
  if (n) {
    IC_CUDA(ctx, cudaMemcpyAsync(ctx->ps.q, in, 24 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    IC_CUDA(ctx, cudaMemcpyAsync(ctx->ps.q_build, in, 24 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    in += (24 * n + 15) / 16 * 16;
    IC_CUDA(ctx, cudaMemcpyAsync(ctx->ps.u, in, 3 * ctx->real_size * n, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  // step counter (no weights), neighbour-list rebuild and the step's drive, stream-ordered
  double d[3];
  ic::drive_amplitudes(ctx, step, d);
  k_snapshot_restart<<<1, 1, 0, ctx->stream>>>(ctx->d.step, step, ctx->d.rebuild, ctx->drive, ctx->drive_f, d[0],
                                                d[1], d[2]);
  IC_CUDA(ctx, cudaGetLastError());
  IC_CUDA(ctx, ic::launch_particle_bins(ctx));
  ctx->host_step = step;
  ctx->host_wcount = 0;
  ctx->adj.rec_cur = -1;
  return IC_OK;
}

}  // extern "C"


struct ic_batch {
  std::vector<ic_ctx *> ctxs;
  cudaStream_t main = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::vector<uint64_t> gens[2];
};

namespace {
// IC_BATCH_GRAPH=1: capture the whole ensemble step into one graph per step
// (fork to every box's stream, join back) instead of launching the boxes'
// own step graphs
bool batch_one_graph() {
  const char *v = std::getenv("IC_BATCH_GRAPH");
  return v && v[0] == '1';
}

void batch_drop_graphs(ic_batch *b) {
  for (int i = 0; i < 2; ++i)
    if (b->graph[i]) {
      cudaGraphExecDestroy(b->graph[i]);
      b->graph[i] = nullptr;
    }
}
}  // namespace

extern "C" {

ic_status ic_batch_create(ic_ctx *const *ctxs, int n, ic_batch **out) {
  if (!ctxs || n <= 0 || !out) return IC_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return IC_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return IC_ERR_ARG;   // a box appears once
  }
  ic_batch *b = new ic_batch();
  b->ctxs.assign(ctxs, ctxs + n);
  // the boxes' step graphs are captured again inside ic_batch_step, with
  // programmatic dependent launch between their kernels
  for (int i = 0; i < n; ++i) invalidate_graphs(ctxs[i]);
  b->joins.resize(n, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < n; ++i) ok = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    ic_batch_destroy(b);
    return IC_ERR_CUDA;
  }
  *out = b;
  return IC_OK;
}

ic_status ic_batch_step(ic_batch *b, int nsteps, const double *w) {
  const ic::TraceRange tr("ic_batch_step");
  if (!b || nsteps < 0) return IC_ERR_ARG;
  struct PdlScope {
    PdlScope() { ic::t_pdl_scope = true; }
    ~PdlScope() { ic::t_pdl_scope = false; }
  } pdl_scope;
  if (nsteps == 0) return IC_OK;
  const int parity = b->ctxs[0]->cur;
  for (ic_ctx *c : b->ctxs) {
    if (c->cur != parity || c->profiling) return fail(c, IC_ERR_STATE, "batched boxes must share the step parity");
    const ic_status st = upload_weights(c, nsteps, w);
    if (st) return st;
  }
  if (!batch_one_graph()) {
    // every box's own step graph on its stream, step-major over the boxes:
    // boxes advance independently, with no ensemble-wide join between steps
    for (int s = 0; s < nsteps; ++s)
      for (ic_ctx *c : b->ctxs) {
        const ic_status st = launch_one_step(c);
        if (st) return st;
      }
    for (ic_ctx *c : b->ctxs) c->host_step += nsteps;
    return IC_OK;
  }
  // the boxes' own work (weight uploads, earlier steps) precedes the batch graph
  for (ic_ctx *c : b->ctxs) {
    if (cudaEventRecord(b->joins[0], c->stream) != cudaSuccess ||
        cudaStreamWaitEvent(b->main, b->joins[0], 0) != cudaSuccess)
      return IC_ERR_CUDA;
  }
  for (int s = 0; s < nsteps; ++s) {
    const int par = b->ctxs[0]->cur;
    bool stale = !b->graph[par] || b->gens[par].size() != b->ctxs.size();
    for (size_t i = 0; !stale && i < b->ctxs.size(); ++i) stale = b->gens[par][i] != b->ctxs[i]->generation;
    if (stale) {
      if (b->graph[par]) {
        cudaGraphExecDestroy(b->graph[par]);
        b->graph[par] = nullptr;
      }
      cudaGraph_t graph;
      if (cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return IC_ERR_CUDA;
      cudaError_t e = cudaEventRecord(b->fork, b->main);
      for (size_t i = 0; e == cudaSuccess && i < b->ctxs.size(); ++i) {
        ic_ctx *c = b->ctxs[i];
        e = cudaStreamWaitEvent(c->stream, b->fork, 0);
        if (e == cudaSuccess) e = enqueue_step(c, c->cur);
        if (e == cudaSuccess) e = cudaEventRecord(b->joins[i], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->joins[i], 0);
      }
      const cudaError_t ce = cudaStreamEndCapture(b->main, &graph);
      if (e != cudaSuccess || ce != cudaSuccess) return IC_ERR_CUDA;
      const cudaError_t ie = cudaGraphInstantiate(&b->graph[par], graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) return IC_ERR_CUDA;
      b->gens[par].clear();
      for (ic_ctx *c : b->ctxs) b->gens[par].push_back(c->generation);
    }
    if (cudaGraphLaunch(b->graph[par], b->main) != cudaSuccess) return IC_ERR_CUDA;
    for (ic_ctx *c : b->ctxs) c->cur = 1 - c->cur;
  }
  // later calls on any box are ordered after the batch
  if (cudaEventRecord(b->fork, b->main) != cudaSuccess) return IC_ERR_CUDA;
  for (ic_ctx *c : b->ctxs) {
    if (cudaStreamWaitEvent(c->stream, b->fork, 0) != cudaSuccess) return IC_ERR_CUDA;
    c->host_step += nsteps;
  }
  return IC_OK;
}

ic_status ic_set_tile(ic_ctx *ctx, int tile_x, int zchunk) {
  if (!ctx || (tile_x != 0 && tile_x != 16 && tile_x != 32)) return IC_ERR_ARG;
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int variant = tile_x == 0 ? ic::kTileRows : (tile_x == 16 ? 1 : 0);
  if (variant == ic::kTileRows && !(ic::rows_eligible(ctx->p) && ic::rows_buffers_aligned(ctx)))
    return fail(ctx, IC_ERR_ARG, "the whole-row stage kernel needs FP32, nx a multiple of 4 and at most 128");
  if (!ic::set_stage_tile(ctx, variant, zchunk)) return fail(ctx, IC_ERR_ARG, "zchunk below 8");
  invalidate_graphs(ctx);
  return IC_OK;
}

ic_status ic_set_stage_copy(ic_ctx *ctx, int mode) {
  if (!ctx || mode < IC_STAGE_COPY_THREAD || mode > IC_STAGE_COPY_ROWS16) return IC_ERR_ARG;
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->stage_copy = mode;
  invalidate_graphs(ctx);
  return IC_OK;
}

ic_status ic_get_stage_copy(const ic_ctx *ctx, int *mode) {
  if (!ctx || !mode) return IC_ERR_ARG;
  *mode = ic::stage_copy_active(ctx);
  return IC_OK;
}

ic_status ic_get_tile(const ic_ctx *ctx, int *tile_x, int *tile_y, int *zchunk) {
  if (!ctx) return IC_ERR_ARG;
  int t[3];
  ic::stage_tile(ctx, &t[0], &t[1], &t[2]);
  if (tile_x) *tile_x = t[0];
  if (tile_y) *tile_y = t[1];
  if (zchunk) *zchunk = t[2];
  return IC_OK;
}

ic_status ic_autotune(ic_ctx *ctx, int reps, int *choice) {
  const ic::TraceRange tr("ic_autotune");
  if (!ctx || reps <= 0) return IC_ERR_ARG;
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // the stage kernels of one step, U^n (buffer cur) only read: stage 1 writes
  // the other state buffer, stage 2 the half-step buffer, stage 3 the other
  // state buffer again (all three, the noise and the partials are scratch
  // until the next step rewrites them)
  void *const *U0 = ctx->U[ctx->cur];
  void *const *U1 = ctx->U[1 - ctx->cur];
  void *const *U2 = ctx->U[2];
  auto stages = [&]() {
    cudaError_t e = ic::launch_stage(ctx, 0, U0, U0, U1);
    if (e == cudaSuccess) e = ic::launch_stage(ctx, 1, U1, U0, U2);
    if (e == cudaSuccess) e = ic::launch_stage(ctx, 2, U2, U0, U1);
    return e;
  };
  cudaEvent_t e0, e1;
  IC_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx, IC_ERR_CUDA, "cudaEventCreate");
  }
  int best_v = ctx->tile_variant, best_z = ctx->zchunk, best_copy = ctx->stage_copy;
  float best_ms = -1.0f;
  cudaError_t err = cudaSuccess;
  // candidates: the wide tile with each staging mode (the row modes where the
  // grid allows them), the narrow tile; zchunk 32, 16, 8 each
  const int v_in = ctx->tile_variant, copy_in = ctx->stage_copy;
  ctx->tile_variant = 0;
  ctx->stage_copy = IC_STAGE_COPY_ROWS16;
  const bool rows_ok = ic::stage_copy_active(ctx) != IC_STAGE_COPY_THREAD;
  ctx->tile_variant = v_in;
  ctx->stage_copy = copy_in;
  // With noise a context on the whole-row kernel is tuned among its z chunks
  // only, one on the column-tile kernels among those: the two families round
  // the stress divergence differently, and tuning must not change a run's
  // results.  Without noise they give the same bits and all are candidates
  // (the whole-row kernel where its layout allows it).
  const bool whole_rows = ic::rows_active(ctx);
  const bool any_family = ctx->p.kT == 0.0;
  const bool rows_layout = ic::rows_eligible(ctx->p) && ic::rows_buffers_aligned(ctx);
  for (int cand = 0; cand < 5 && err == cudaSuccess; ++cand) {
    const int v = cand == 4 ? ic::kTileRows : (cand == 3 ? 1 : 0), copy = cand >= 3 ? IC_STAGE_COPY_THREAD : cand;
    if (copy != IC_STAGE_COPY_THREAD && !rows_ok) continue;
    if (!any_family && (v == ic::kTileRows) != whole_rows) continue;
    if (v == ic::kTileRows && !rows_layout) continue;
    ctx->stage_copy = copy;
    int last = -1;
    for (int z : {32, 16, 8}) {
      const int zc = std::min(z, ctx->p.nz);
      if (zc == last || !ic::set_stage_tile(ctx, v, zc)) continue;
      last = zc;
      err = stages();   // warm-up
      if (err == cudaSuccess) err = cudaEventRecord(e0, ctx->stream);
      for (int r = 0; r < reps && err == cudaSuccess; ++r) err = stages();
      if (err == cudaSuccess) err = cudaEventRecord(e1, ctx->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err != cudaSuccess) break;
      if (best_ms < 0.0f || ms < best_ms) {
        best_ms = ms;
        best_v = v;
        best_z = zc;
        best_copy = copy;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->stage_copy = best_copy;
  ic::set_stage_tile(ctx, best_v, best_z);
  invalidate_graphs(ctx);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "autotune");
  if (choice) ic::stage_tile(ctx, &choice[0], &choice[1], &choice[2]);
  return IC_OK;
}

ic_status ic_batch_autotune(ic_batch *b, int reps) {
  if (!b || reps <= 0) return IC_ERR_ARG;
  std::vector<std::array<int, 6>> keys;
  std::vector<ic_ctx *> tuned;
  for (ic_ctx *c : b->ctxs) {
    const std::array<int, 6> key{c->p.nx, c->p.ny, c->p.nz, c->p.precision, c->p.kT > 0.0 ? 1 : 0,
                                 c->ps.n > 0 ? 1 : 0};
    size_t j = 0;
    while (j < keys.size() && keys[j] != key) ++j;
    if (j == keys.size()) {
      const ic_status st = ic_autotune(c, reps, nullptr);
      if (st) return st;
      keys.push_back(key);
      tuned.push_back(c);
    } else {
      IC_CUDA(c, cudaStreamSynchronize(c->stream));
      c->stage_copy = tuned[j]->stage_copy;
      ic::set_stage_tile(c, tuned[j]->tile_variant, tuned[j]->zchunk);
      invalidate_graphs(c);
    }
  }
  return IC_OK;
}

void ic_batch_destroy(ic_batch *b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  batch_drop_graphs(b);
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->main) cudaStreamDestroy(b->main);
  delete b;
}

ic_status ic_device_views(ic_ctx *ctx, ic_views *out) {
  if (!ctx || !out) return IC_ERR_ARG;
  out->drho = ctx->U[ctx->cur][0];
  out->gx = ctx->U[ctx->cur][1];
  out->gy = ctx->U[ctx->cur][2];
  out->gz = ctx->U[ctx->cur][3];
  out->precision = ctx->p.precision;
  out->n_particles = ctx->ps.n;
  out->q = ctx->ps.q;
  return IC_OK;
}

ic_status ic_profile(ic_ctx *ctx, int enable) {
  if (!ctx) return IC_ERR_ARG;
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->profiling = enable != 0;
  ctx->timed.clear();
  ctx->event_next = 0;
  return IC_OK;
}

ic_status ic_profile_read(ic_ctx *ctx, double *ms, int64_t *launches, int reset) {
  if (!ctx) return IC_ERR_ARG;
  IC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double acc[IC_PROFILE_CLASSES] = {};
  int64_t cnt[IC_PROFILE_CLASSES] = {};
  for (const auto &t : ctx->timed) {
    float v = 0.f;
    IC_CUDA(ctx, cudaEventElapsedTime(&v, t.a, t.b));
    acc[t.cls] += v;
    ++cnt[t.cls];
  }
  for (int i = 0; i < IC_PROFILE_CLASSES; ++i) {
    if (ms) ms[i] = acc[i];
    if (launches) launches[i] = cnt[i];
  }
  if (reset) {
    ctx->timed.clear();
    ctx->event_next = 0;
  }
  return IC_OK;
}

const char *ic_last_error(const ic_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void ic_destroy(ic_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  invalidate_graphs(ctx);
  for (cudaEvent_t ev : ctx->event_pool) cudaEventDestroy(ev);
  if (ctx->staging_done) cudaEventDestroy(ctx->staging_done);
  if (ctx->staging) cudaFreeHost(ctx->staging);
  if (ctx->download) cudaFreeHost(ctx->download);
  for (int j = 0; j < 2; ++j) {
    if (ctx->fetch_done[j]) cudaEventDestroy(ctx->fetch_done[j]);
    if (ctx->fetch[j]) cudaFreeHost(ctx->fetch[j]);
  }
  while (ctx->n_allocs > 0) dev_free(ctx, ctx->allocs[ctx->n_allocs - 1]);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

}  // extern "C"
