// Particle kernels of libic: the particle substeps of App. A.2 coupled to the
// grid through the 3-point kernel (App. A.1).  One warp per particle; lanes
// 0..26 own the 27 points of a location set.
//
// Per step (the fluid stages run in ic_fluid.cu between these launches):
//   kHalfStep        substeps 1-2: J^n v^n at q^n -> q^{n+1/2}; F^{n+1/2};
//                    stencils at q^{n+1/2}; J^{n+1/2} v^n; Omega of stage 1
//   kStageCorrection after each RK stage s: adds b_s dt times the particle
//                    part of the momentum rate, -(1/h) grad(S Omega_s) + S F,
//                    to the stage output, then gathers Omega_{s+1}
//   kImpulse         substeps 4-5: dg, u^{n+1}, lambda from J v~^{n+1}
//   kSpread          substep 6: g^{n+1} = g~^{n+1} - S dg
//   kFinal           substep 7: q^{n+1}; weighted force sums
//
// Spreading is deterministic and free of atomics: each grid face near
// particles is updated by exactly one particle (its "owner": the lowest
// index among the particles whose footprint holds the face), which sums the
// contributions of itself and its neighbours in ascending index order.  The
// footprint of a particle is the 4 x 3 x 3 block of a-faces around its centre
// stencil for each axis a: every face that its pressure gradient, its force
// or its impulse can reach.  Neighbour lists (|dq_a| < 4h + skin on every
// axis) are rebuilt when a particle has moved more than a quarter skin.
#include <cuda_runtime.h>

#include <cmath>

#include "ic_device.cuh"
#include "ic_internal.hpp"

namespace ic {
namespace {

constexpr int kWarpsPerBlock = 8;

struct PConsts {
  int n[3];
  double h, inv_h, L[3], dt, rho0, vol;
  double cutoff;      // neighbour cutoff per axis
  double rebuild_at;  // displacement since build that triggers a rebuild
  double skin_limit;  // displacement at which a list is no longer valid
};

template <typename real>
struct PV {
  int n;
  double *q, *q_eq, *q_build, *q_half, *acc;
  real *u, *m_e, *eps, *k_s, *w, *jv_n, *omega, *force, *dg, *lam;
  int *base, *nbr, *nnbr;
};

template <typename real>
PV<real> view(const ParticleStore &s) {
  PV<real> v;
  v.n = s.n;
  v.q = s.q;
  v.q_eq = s.q_eq;
  v.q_build = s.q_build;
  v.q_half = s.q_half;
  v.acc = s.acc;
  v.u = (real *)s.u;
  v.m_e = (real *)s.m_e;
  v.eps = (real *)s.eps;
  v.k_s = (real *)s.k_s;
  v.w = (real *)s.w;
  v.jv_n = (real *)s.jv_n;
  v.omega = (real *)s.omega;
  v.force = (real *)s.force;
  v.dg = (real *)s.dg;
  v.lam = (real *)s.lam;
  v.base = s.base;
  v.nbr = s.nbr;
  v.nnbr = s.nnbr;
  return v;
}

template <typename real>
struct Grid4 {
  real *f[4];   // delta rho, g_x, g_y, g_z
};

__device__ __forceinline__ double wrap_pos(double x, double L) {
  double r = fmod(x, L);
  if (r < 0.0) r += L;
  if (r >= L) r -= L;
  return r;
}

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

// Stencil of a particle at q: centre base and weights, own-axis face base and weights.
template <typename real>
__device__ void stencil_at(const double q[3], const PConsts &pc, int base[6], real w[18]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double s = q[a] / pc.h;
    const double fc = floor(s + 0.5);
    peskin3(real(s - fc), &w[3 * a]);
    base[a] = wrap(int(fc), pc.n[a]);
    const double sf = s - 0.5;
    const double ff = floor(sf + 0.5);
    peskin3(real(sf - ff), &w[9 + 3 * a]);
    base[3 + a] = wrap(int(ff), pc.n[a]);
  }
}

__device__ __forceinline__ size_t cell_index(int x, int y, int z, const PConsts &pc) {
  return size_t(x) + size_t(pc.n[0]) * (size_t(y) + size_t(pc.n[1]) * size_t(z));
}

__device__ __forceinline__ int step_coord(int b, int d, int n) {
  int v = b + d;
  if (v < 0) v += n;
  if (v >= n) v -= n;
  return v;
}

// Warp gather at one stencil: J delta rho (out[0]) and J v^a (out[1+a]).
template <typename real>
__device__ void gather(const Grid4<real> &G, const int base[6], const real w[18], const PConsts &pc,
                       int lane, bool want_rho, bool want_v, real out[4]) {
  real acc[4] = {real(0), real(0), real(0), real(0)};
  if (lane < 27) {
    const int d[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
    int cc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) cc[a] = step_coord(base[a], d[a], pc.n[a]);
    if (want_rho)
      acc[0] = w[d[0] + 1] * w[3 + d[1] + 1] * w[6 + d[2] + 1] * G.f[0][cell_index(cc[0], cc[1], cc[2], pc)];
    if (want_v) {
      const real rho0 = real(pc.rho0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int fc[3] = {cc[0], cc[1], cc[2]};
        fc[a] = step_coord(base[3 + a], d[a], pc.n[a]);
        real wt = w[9 + 3 * a + d[a] + 1];
#pragma unroll
        for (int b = 0; b < 3; ++b)
          if (b != a) wt *= w[3 * b + d[b] + 1];
        const size_t i = cell_index(fc[0], fc[1], fc[2], pc);
        int up[3] = {fc[0], fc[1], fc[2]};
        up[a] = (up[a] + 1 == pc.n[a]) ? 0 : up[a] + 1;
        const size_t iu = cell_index(up[0], up[1], up[2], pc);
        const real rf = rho0 + real(0.5) * (G.f[0][i] + G.f[0][iu]);
        acc[1 + a] = wt * (G.f[1 + a][i] / rf);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) out[j] = warp_sum(acc[j]);
}

template <typename real>
__device__ __forceinline__ void load_stencil(const PV<real> &P, int p, int base[6], real w[18]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) base[j] = P.base[6 * p + j];
#pragma unroll
  for (int j = 0; j < 18; ++j) w[j] = P.w[18 * p + j];
}

// centre-set weight of particle m at cell c (0 outside its stencil)
template <typename real>
__device__ __forceinline__ real centre_weight(const PV<real> &P, int m, const int c[3], const PConsts &pc) {
  real wt = real(1);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int d = ring_delta(c[b], P.base[6 * m + b], pc.n[b]);
    if (d < -1 || d > 1) return real(0);
    wt *= P.w[18 * m + 3 * b + d + 1];
  }
  return wt;
}

// a-face weight of particle m at face f (0 outside its stencil)
template <typename real>
__device__ __forceinline__ real face_weight(const PV<real> &P, int m, int a, const int f[3], const PConsts &pc) {
  real wt = real(1);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int bb = (b == a) ? 3 + b : b;
    const int d = ring_delta(f[b], P.base[6 * m + bb], pc.n[b]);
    if (d < -1 || d > 1) return real(0);
    wt *= P.w[18 * m + (b == a ? 9 : 0) + 3 * b + d + 1];
  }
  return wt;
}

template <typename real>
__device__ __forceinline__ bool in_footprint(const PV<real> &P, int m, int a, const int f[3], const PConsts &pc) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int d = ring_delta(f[b], P.base[6 * m + b], pc.n[b]);
    if (b == a ? (d < -2 || d > 1) : (d < -1 || d > 1)) return false;
  }
  return true;
}

// The owner-computes face update.  KIND 0: stage correction
// coef * [-(Omega_m / h^4)(W_c(c+) - W_c(c-)) + W_a(f) F_m / h^3];
// KIND 1: impulse, -W_a(f) dg_m / h^3.
template <typename real, int KIND>
__device__ void update_owned_faces(const PV<real> &P, const Grid4<real> &G, int p, int lane,
                                   const real *omega, real coef, const PConsts &pc) {
  const int nn = P.nnbr[p];
  const int *nb = P.nbr + size_t(p) * kMaxNeighbours;
  const real inv_h3 = real(pc.inv_h * pc.inv_h * pc.inv_h);
  const real inv_h4 = inv_h3 * real(pc.inv_h);
  for (int t = lane; t < 108; t += 32) {
    const int a = t / 36, r = t % 36;
    const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    int f[3];
    f[a] = step_coord(P.base[6 * p + a], r % 4 - 2, pc.n[a]);
    f[b1] = step_coord(P.base[6 * p + b1], (r / 4) % 3 - 1, pc.n[b1]);
    f[b2] = step_coord(P.base[6 * p + b2], r / 12 - 1, pc.n[b2]);
    bool owner = true;
    for (int j = 0; j < nn && owner; ++j) {
      const int m = nb[j];
      if (m >= p) break;
      if (in_footprint(P, m, a, f, pc)) owner = false;
    }
    if (!owner) continue;
    int cp[3] = {f[0], f[1], f[2]};
    cp[a] = (cp[a] + 1 == pc.n[a]) ? 0 : cp[a] + 1;
    // contributions of p and its neighbours, in ascending particle index
    real total = real(0);
    bool self_done = false;
    int j = 0;
    while (true) {
      int m;
      if (!self_done && (j >= nn || nb[j] > p)) {
        m = p;
        self_done = true;
      } else if (j < nn) {
        m = nb[j++];
      } else {
        break;
      }
      if (KIND == 0) {
        const real wp = centre_weight(P, m, cp, pc), wm = centre_weight(P, m, f, pc);
        const real wf = face_weight(P, m, a, f, pc);
        total += -(omega[m] * inv_h4) * (wp - wm) + wf * P.force[3 * m + a] * inv_h3;
      } else {
        const real wf = face_weight(P, m, a, f, pc);
        total += -wf * P.dg[3 * m + a] * inv_h3;
      }
    }
    const size_t i = cell_index(f[0], f[1], f[2], pc);
    G.f[1 + a][i] += coef * total;
  }
}

// ------------------------------------------------------------------ kernels
template <typename real>
__global__ void k_half_step(PV<real> P, Grid4<real> G, PConsts pc, int *rebuild, int *status) {
  const int p = blockIdx.x * kWarpsPerBlock + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= P.n) return;
  double q[3] = {P.q[3 * p], P.q[3 * p + 1], P.q[3 * p + 2]};

  if (*rebuild) {
    // neighbour list from q^n, in ascending index order
    int count = 0;
    for (int j0 = 0; j0 < P.n; j0 += 32) {
      const int j = j0 + lane;
      bool hit = false;
      if (j < P.n && j != p) {
        hit = true;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          hit = hit && fabs(min_image(P.q[3 * j + a] - q[a], pc.L[a])) < pc.cutoff;
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int slot = count + __popc(m & ((1u << lane) - 1u));
        if (slot < kMaxNeighbours) P.nbr[size_t(p) * kMaxNeighbours + slot] = j;
      }
      count += __popc(m);
    }
    if (lane == 0) {
      if (count > kMaxNeighbours) atomicOr(status, kStatusNbrOverflow);
      P.nnbr[p] = min(count, kMaxNeighbours);
      for (int a = 0; a < 3; ++a) P.q_build[3 * p + a] = q[a];
    }
  }

  // substep 1: q^{n+1/2} = q^n + dt/2 J^n v^n
  int base[6];
  real w[18];
  stencil_at(q, pc, base, w);
  real g4[4];
  gather(G, base, w, pc, lane, false, true, g4);
  double qh[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) qh[a] = wrap_pos(q[a] + 0.5 * pc.dt * double(g4[1 + a]), pc.L[a]);

  // substep 2: tether force at q^{n+1/2}
  real F[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) F[a] = real(-double(P.k_s[p]) * min_image(qh[a] - P.q_eq[3 * p + a], pc.L[a]));

  // stencil at q^{n+1/2}; J^{n+1/2} v^n and J^{n+1/2} rho^n
  stencil_at(qh, pc, base, w);
  gather(G, base, w, pc, lane, true, true, g4);
  if (lane == 0) {
    for (int a = 0; a < 3; ++a) {
      P.q_half[3 * p + a] = qh[a];
      P.force[3 * p + a] = F[a];
      P.jv_n[3 * p + a] = g4[1 + a];
      const double d = fabs(min_image(qh[a] - P.q_build[3 * p + a], pc.L[a]));
      if (d > pc.skin_limit) atomicOr(status, kStatusSkin);
    }
    for (int j = 0; j < 6; ++j) P.base[6 * p + j] = base[j];
    for (int j = 0; j < 18; ++j) P.w[18 * p + j] = w[j];
    P.omega[p] = P.eps[p] * real(pc.vol) * g4[0];   // Omega = eps V (J rho - rho0)
  }
}

template <typename real>
__global__ void k_stage_correction(PV<real> P, Grid4<real> G, PConsts pc, int stage, real coef,
                                   int *rebuild) {
  const int p = blockIdx.x * kWarpsPerBlock + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (stage == 0 && blockIdx.x == 0 && threadIdx.x == 0) *rebuild = 0;
  if (p >= P.n) return;
  const real *om = P.omega + size_t(stage & 1) * P.n;
  update_owned_faces<real, 0>(P, G, p, lane, om, coef, pc);
  if (stage < 2) {
    int base[6];
    real w[18];
    load_stencil(P, p, base, w);
    real g4[4];
    gather(G, base, w, pc, lane, true, false, g4);
    if (lane == 0) P.omega[size_t((stage + 1) & 1) * P.n + p] = P.eps[p] * real(pc.vol) * g4[0];
  }
}

template <typename real>
__global__ void k_impulse(PV<real> P, Grid4<real> G, PConsts pc) {
  const int p = blockIdx.x * kWarpsPerBlock + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= P.n) return;
  int base[6];
  real w[18];
  load_stencil(P, p, base, w);
  real g4[4];
  gather(G, base, w, pc, lane, true, true, g4);
  if (lane == 0) {
    const real mf = real(pc.vol) * (real(pc.rho0) + g4[0]);   // m_f = V J rho^{n+1}
    const real me = P.m_e[p];
    for (int a = 0; a < 3; ++a) {
      const real u = P.u[3 * p + a];
      const real rel = g4[1 + a] - u;
      const real dg = me * mf / (me + mf) * rel;
      P.dg[3 * p + a] = dg;
      P.u[3 * p + a] = u + mf / (me + mf) * rel;
      P.lam[3 * p + a] = dg / real(pc.dt) - P.force[3 * p + a];
    }
  }
}

template <typename real>
__global__ void k_spread(PV<real> P, Grid4<real> G, PConsts pc) {
  const int p = blockIdx.x * kWarpsPerBlock + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= P.n) return;
  update_owned_faces<real, 1>(P, G, p, lane, nullptr, real(1), pc);
}

template <typename real>
__global__ void k_final(PV<real> P, Grid4<real> G, PConsts pc, const int64_t *step, const double *weights,
                        int *rebuild) {
  const int p = blockIdx.x * kWarpsPerBlock + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= P.n) return;
  int base[6];
  real w[18];
  load_stencil(P, p, base, w);
  real g4[4];
  gather(G, base, w, pc, lane, false, true, g4);
  if (lane == 0) {
    const int64_t jw = step[0] - step[1];
    const double wt = (jw >= 0 && jw < step[2]) ? weights[jw] : 0.0;
    bool move = false;
    for (int a = 0; a < 3; ++a) {
      const double qn = wrap_pos(P.q[3 * p + a] + 0.5 * pc.dt * (double(g4[1 + a]) + double(P.jv_n[3 * p + a])),
                                 pc.L[a]);
      P.q[3 * p + a] = qn;
      P.acc[6 * p + a] += wt * double(P.force[3 * p + a]);
      P.acc[6 * p + 3 + a] += wt * double(P.lam[3 * p + a]);
      if (fabs(min_image(qn - P.q_build[3 * p + a], pc.L[a])) > pc.rebuild_at) move = true;
    }
    if (move) *rebuild = 1;
  }
}

template <typename real>
__global__ void k_init_velocity(PV<real> P, Grid4<real> G, PConsts pc, int first, int n) {
  const int p = first + blockIdx.x * kWarpsPerBlock + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= first + n) return;
  double q[3] = {P.q[3 * p], P.q[3 * p + 1], P.q[3 * p + 2]};
  int base[6];
  real w[18];
  stencil_at(q, pc, base, w);
  real g4[4];
  gather(G, base, w, pc, lane, false, true, g4);
  if (lane == 0)
    for (int a = 0; a < 3; ++a) P.u[3 * p + a] = g4[1 + a];
}

template <typename real>
__global__ void k_particle_momentum(PV<real> P, double *out3) {
  __shared__ double s[3][256];
  double acc[3] = {0, 0, 0};
  for (int p = threadIdx.x; p < P.n; p += blockDim.x)
    for (int a = 0; a < 3; ++a) acc[a] += double(P.m_e[p]) * double(P.u[3 * p + a]);
  for (int a = 0; a < 3; ++a) s[a][threadIdx.x] = acc[a];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int a = 0; a < 3; ++a) s[a][threadIdx.x] += s[a][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) out3[a] = s[a][0];
}

PConsts particle_consts(const ic_ctx *ctx) {
  const ic_grid_params &p = ctx->p;
  PConsts c{};
  c.n[0] = p.nx;
  c.n[1] = p.ny;
  c.n[2] = p.nz;
  c.h = p.h;
  c.inv_h = 1.0 / p.h;
  c.L[0] = p.nx * p.h;
  c.L[1] = p.ny * p.h;
  c.L[2] = p.nz * p.h;
  c.dt = p.dt;
  c.rho0 = p.rho0;
  c.vol = 8.0 * p.h * p.h * p.h;   // V = 1 / (J S) = 8 h^3 (Eq. (kvol))
  c.cutoff = (4.0 + kSkin) * p.h;
  c.rebuild_at = 0.25 * kSkin * p.h;
  c.skin_limit = 0.5 * kSkin * p.h;
  return c;
}

template <typename real>
Grid4<real> grid4(void *const U[4]) {
  Grid4<real> g;
  for (int j = 0; j < 4; ++j) g.f[j] = static_cast<real *>(U[j]);
  return g;
}

template <typename real>
cudaError_t launch_particles_t(ic_ctx *ctx, ParticlePhase phase, int stage, void *const cur[4],
                               void *const tgt[4]) {
  const PV<real> P = view<real>(ctx->ps);
  if (P.n == 0) return cudaSuccess;
  const PConsts pc = particle_consts(ctx);
  const dim3 grid((P.n + kWarpsPerBlock - 1) / kWarpsPerBlock), block(32 * kWarpsPerBlock);
  static const double kCoef[3] = {1.0, 0.25, 2.0 / 3.0};
  switch (phase) {
    case kHalfStep:
      k_half_step<real><<<grid, block, 0, ctx->stream>>>(P, grid4<real>(cur), pc, ctx->d.rebuild, ctx->d.status);
      break;
    case kStageCorrection:
      k_stage_correction<real><<<grid, block, 0, ctx->stream>>>(P, grid4<real>(tgt), pc, stage,
                                                                real(kCoef[stage] * ctx->p.dt), ctx->d.rebuild);
      break;
    case kImpulse:
      k_impulse<real><<<grid, block, 0, ctx->stream>>>(P, grid4<real>(tgt), pc);
      break;
    case kSpread:
      k_spread<real><<<grid, block, 0, ctx->stream>>>(P, grid4<real>(tgt), pc);
      break;
    case kFinal:
      k_final<real><<<grid, block, 0, ctx->stream>>>(P, grid4<real>(tgt), pc, ctx->d.step, ctx->d.weights,
                                                     ctx->d.rebuild);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_particles(ic_ctx *ctx, ParticlePhase phase, int stage, void *const cur[4],
                             void *const tgt[4]) {
  if (ctx->p.precision == IC_FP32) return launch_particles_t<float>(ctx, phase, stage, cur, tgt);
  return launch_particles_t<double>(ctx, phase, stage, cur, tgt);
}

cudaError_t launch_particle_velocity(ic_ctx *ctx, int first, int n, void *const state[4]) {
  const PConsts pc = particle_consts(ctx);
  const dim3 grid((n + kWarpsPerBlock - 1) / kWarpsPerBlock), block(32 * kWarpsPerBlock);
  if (ctx->p.precision == IC_FP32)
    k_init_velocity<float><<<grid, block, 0, ctx->stream>>>(view<float>(ctx->ps), grid4<float>(state), pc,
                                                            first, n);
  else
    k_init_velocity<double><<<grid, block, 0, ctx->stream>>>(view<double>(ctx->ps), grid4<double>(state), pc,
                                                             first, n);
  return cudaGetLastError();
}

cudaError_t launch_particle_momentum(ic_ctx *ctx, double *dev_out3) {
  if (ctx->p.precision == IC_FP32)
    k_particle_momentum<float><<<1, 256, 0, ctx->stream>>>(view<float>(ctx->ps), dev_out3);
  else
    k_particle_momentum<double><<<1, 256, 0, ctx->stream>>>(view<double>(ctx->ps), dev_out3);
  return cudaGetLastError();
}

}  // namespace ic
