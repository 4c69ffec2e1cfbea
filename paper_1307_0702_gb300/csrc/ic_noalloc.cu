// ic_fluid_step_noalloc: one SSP-RK3 fluid step between caller-owned device
// arrays, using no device allocation at all.
//
// Some callers cannot allocate device memory at the time they want to step
// the fluid: code that runs inside another framework's stream capture (where
// cudaMalloc is not allowed), hosts whose device memory is entirely reserved
// by their own pool or arena, and plug-ins that may not allocate once the
// host application has started.  For them this entry point keeps its scratch
// (the two intermediate RK3 states, the stored stage noise, the per-CTA
// partial sums and a few tables) in one file-scope device array of fixed
// size, kNoallocScratchBytes = 5.5 MiB, which every GPU that loads the library
// holds until the process exits.  It therefore accepts grids of at most
// IC_NOALLOC_MAX_CELLS = 32768 cells and rejects larger ones.
//
// The array's host-side name is only a stand-in for the device symbol: the
// device address is looked up with cudaGetSymbolAddress the first time the
// entry point runs in a CUDA context and cached with that context's unique id
// (cuCtxGetId, reached through the runtime's driver entry points so that the
// library does not link the driver).  A device reset ends the context, the
// next call sees a new id and looks the address up again.  The first call in
// each context should therefore come before any stream capture.  Every call shares the one array and it keeps the last
// call's contents; nothing in it has to start at zero (each buffer is fully
// written before it is read within a call).  Calls whose work overlaps on the
// GPU (different streams, or several host threads) race on the array.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "ic_device.cuh"
#include "ic_internal.hpp"

namespace {

constexpr size_t kNoallocScratchBytes = 5767168;   // 5.5 MiB
constexpr int kMaxCells = IC_NOALLOC_MAX_CELLS;
constexpr size_t kMaxPartials = 4096;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char ic_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mutex;
void *g_scratch[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The per-call tables: step counter, drive amplitudes of the three stages and
// cos(k x_i) along the wave axis, computed on the device from the call's
// parameters (so that nothing is copied from host memory).
template <typename real>
__global__ void k_noalloc_tables(int64_t *step_out, int64_t step, real *drive, real *cos_table, int n_ax,
                                 double kwave, double h, double amp, double omega, double dt, double phase) {
  const int t = threadIdx.x;
  if (t == 0) step_out[0] = step;
  if (t < 3) {
    const double frac = t == 0 ? 0.0 : (t == 1 ? 1.0 : 0.5);
    drive[t] = real(amp * sin(omega * ((double(step) + frac) * dt) + phase));
  }
  for (int i = t; i < n_ax; i += blockDim.x) cos_table[i] = real(cos(kwave * i * h));
}

template <typename real>
ic::FluidConsts<real> consts_from(const ic_grid_params &p, const real *cos_table, const real *drive) {
  return ic::make_fluid_consts<real>(p, cos_table, drive);
}

template <typename real>
ic_status step_noalloc(const ic_grid_params &p, const void *const in[4], void *const out[4], int64_t step,
                       unsigned char *scratch) {
  const cudaStream_t stream = static_cast<cudaStream_t>(p.stream);
  const size_t cells = size_t(p.nx) * p.ny * p.nz;
  const size_t fb = align256(cells * sizeof(real));
  unsigned char *cur = scratch;
  void *u1[4], *u2[4], *noise[12];
  for (int j = 0; j < 4; ++j, cur += fb) u1[j] = cur;
  for (int j = 0; j < 4; ++j, cur += fb) u2[j] = cur;
  for (int j = 0; j < 12; ++j, cur += fb) noise[j] = cur;
  double *partials = reinterpret_cast<double *>(cur);
  cur += align256(kMaxPartials * sizeof(double));
  const int n_ax = p.wave_axis == 0 ? p.nx : (p.wave_axis == 1 ? p.ny : p.nz);
  real *cos_table = reinterpret_cast<real *>(cur);
  cur += align256(size_t(n_ax) * sizeof(real));
  real *drive = reinterpret_cast<real *>(cur);
  cur += 256;
  int64_t *stepd = reinterpret_cast<int64_t *>(cur);
  cur += 256;
  if (size_t(cur - scratch) > kNoallocScratchBytes || ic::stage_ctas_raw(p) > kMaxPartials) return IC_ERR_CAPACITY;

  // the driven mode (as in ic_create_grid)
  const double kwave = 2.0 * M_PI * p.wave_nlambda / (n_ax * p.h);
  const double omega = p.c * (2.0 / p.h) * std::sin(0.5 * kwave * p.h);
  const double gamma = (4.0 * p.eta / 3.0 + p.zeta) / (2.0 * p.rho0);
  double amp = p.forcing == IC_FORCE_MODE ? 2.0 * gamma * omega * p.wave_amp : p.wave_amp * n_ax * gamma * omega;
  if (p.wave_amp == 0.0 || p.forcing == IC_FORCE_NONE) amp = 0.0;
  k_noalloc_tables<real><<<1, 256, 0, stream>>>(stepd, step, drive, cos_table, n_ax, kwave, p.h, amp, omega, p.dt,
                                                p.wave_phase);
  if (cudaGetLastError() != cudaSuccess) return IC_ERR_CUDA;
  const ic::FluidConsts<real> c = consts_from<real>(p, cos_table, drive);
  const void *const in_u1[4] = {u1[0], u1[1], u1[2], u1[3]};
  const void *const in_u2[4] = {u2[0], u2[1], u2[2], u2[3]};
  if (ic::launch_stage_raw(p, &c, 0, in, in, u1, noise, stepd, partials, stream) != cudaSuccess ||
      ic::launch_stage_raw(p, &c, 1, in_u1, in, u2, noise, stepd, partials, stream) != cudaSuccess ||
      ic::launch_stage_raw(p, &c, 2, in_u2, in, out, noise, stepd, partials, stream) != cudaSuccess)
    return IC_ERR_CUDA;
  return IC_OK;
}

// unique id of the current CUDA context (0 if it cannot be had)
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(f1);
      get_id = reinterpret_cast<GetId>(f2);
    }
    cudaGetLastError();
    looked_up = true;
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// device address of the scratch array in the current context: looked up once
// per context, again after a device reset has replaced the context
unsigned char *scratch_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_mutex);
  const unsigned long long id = current_context_id();
  if (!g_scratch[dev] || id == 0 || id != g_ctx_id[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, ic_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch[dev] = ptr;
    g_ctx_id[dev] = current_context_id();   // the lookup made the context current if it was not
  }
  return static_cast<unsigned char *>(g_scratch[dev]);
}

// [a, a + bytes) and [b, b + bytes) share a byte
bool overlap(const void *a, const void *b, uint64_t bytes) {
  const uint64_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

}  // namespace

extern "C" ic_status ic_fluid_step_noalloc(const ic_grid_params *params, const void *const in[4], void *const out[4],
                                           int64_t step) {
  if (!params || !in || !out) return IC_ERR_ARG;
  const ic_grid_params &p = *params;
  if (p.nx < 6 || p.ny < 6 || p.nz < 6) return IC_ERR_ARG;
  if (!(p.h > 0) || !(p.rho0 > 0) || !(p.c > 0) || !(p.dt > 0) || p.eta < 0 || p.zeta < 0 || p.kT < 0)
    return IC_ERR_ARG;
  if (p.precision != IC_FP64 && p.precision != IC_FP32) return IC_ERR_ARG;
  if (p.forcing < IC_FORCE_NONE || p.forcing > IC_FORCE_PLANE || p.wave_axis < 0 || p.wave_axis > 2) return IC_ERR_ARG;
  const int n_ax = p.wave_axis == 0 ? p.nx : (p.wave_axis == 1 ? p.ny : p.nz);
  if (p.wave_nlambda < 1 || p.plane_index < 0 || p.plane_index >= n_ax) return IC_ERR_ARG;
  // no output may share a byte with an input (stage 3 reads U^n while it
  // writes U^{n+1}) or with another output
  const uint64_t bytes = uint64_t(p.nx) * uint64_t(p.ny) * uint64_t(p.nz) * (p.precision == IC_FP32 ? 4u : 8u);
  for (int j = 0; j < 4; ++j) {
    if (!in[j] || !out[j]) return IC_ERR_ARG;
    for (int k = 0; k < 4; ++k) {
      if (overlap(in[k], out[j], bytes)) return IC_ERR_ARG;
      if (k < j && overlap(out[k], out[j], bytes)) return IC_ERR_ARG;
    }
  }
  if (int64_t(p.nx) * p.ny * p.nz > kMaxCells) return IC_ERR_CAPACITY;
  unsigned char *scratch = scratch_for_current_device();
  if (!scratch) return IC_ERR_CUDA;
  return p.precision == IC_FP32 ? step_noalloc<float>(p, in, out, step, scratch)
                                : step_noalloc<double>(p, in, out, step, scratch);
}
