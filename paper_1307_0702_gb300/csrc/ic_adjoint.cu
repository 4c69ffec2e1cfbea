// Adjoint kernels of libic: the reverse-mode derivative of one deterministic
// IC step (App. A.2 substeps 1-7, kT = 0), for gradients of the weighted time
// average of the tether forces (the force of Sec. 6) with respect to each
// particle's excess mass m_e, its epsilon_pf (Eqs. (part_svel), (ke)), the
// drive amplitude and the state at the start of the step.
//
// The reverse sweep takes the step's substeps in reverse order:
//   substep 7  q^{n+1} = q^n + dt/2 (J v^{n+1} + J v^n) at q^{n+1/2}
//   substep 6  g^{n+1} = g~ - S dg
//   substeps 4-5  dg = mu (J v~ - u^n), u^{n+1} = u^n + r (J v~ - u^n),
//              m_f = V (rho0 + J rho^{n+1})
//   substep 3  the three SSP-RK3 stages, each U_{s+1} = a_s U^n +
//              b_s (U_s + dt R(U_s, pi_s, S F)) with pi_s = c^2 rho_s + p_ext +
//              S Omega_s and Omega_s = epsilon V J rho_s (Eqs. (eq:pressure), (omega))
//   substeps 1-2  q^{n+1/2} = q^n + dt/2 J^n v^n, F = -k (q^{n+1/2} - q_eq)
// Interpolation J and spreading S swap roles (they are adjoint, Eq. (adj)):
// the adjoint of a gather is a spread of the same weights and vice versa.
// Positions enter through the weights of the 3-point function (App. A.1),
// whose derivative is written out in dpeskin3 below.
//
// Grid kernels are one thread per cell and gather every term they need, so
// they write each output once.  Particle kernels are one warp per particle
// (lane t < 27 holds stencil point t; sums by warp reduction) and spread
// with atomic adds (the adjoint is therefore reproducible to rounding, not
// bit for bit).  The grid adjoint fields are in the context's
// precision; the particle adjoints and the gradients are FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ic_device.cuh"
#include "ic_internal.hpp"
#include "ic_particle_common.cuh"

namespace ic {
namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjParticleThreads = 128;   // one warp per particle
// kernel classes of ic_profile_read
constexpr int kClassStage = 3, kClassGrid = 4, kClassParticles = 5;

// SSP-RK3 coefficients: U_{s+1} = a_s U^n + b_s (U_s + dt R(U_s))
constexpr double kA[3] = {0.0, 0.75, 1.0 / 3.0};
constexpr double kB[3] = {1.0, 0.25, 2.0 / 3.0};
// time of each stage's flux evaluation in units of dt after t^n
constexpr double kStageTimes[3] = {0.0, 1.0, 0.5};

// periodic coordinate for offsets of at most one box length
__device__ __forceinline__ int pw(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

struct Geo {
  int nx, ny, nz;
  __device__ __forceinline__ size_t at(int x, int y, int z) const {
    return size_t(IC_CHK(pw(x, nx), nx)) +
           size_t(nx) * (size_t(IC_CHK(pw(y, ny), ny)) + size_t(ny) * size_t(IC_CHK(pw(z, nz), nz)));
  }
};

// unit offset along axis a
__device__ __forceinline__ int ex(int a) { return a == 0; }
__device__ __forceinline__ int ey(int a) { return a == 1; }
__device__ __forceinline__ int ez(int a) { return a == 2; }

template <typename real>
struct State {
  const real *d;      // delta rho
  const real *g[3];   // face momenta
};

template <typename real>
State<real> state_of(void *const U[4]) {
  return {static_cast<const real *>(U[0]),
          {static_cast<const real *>(U[1]), static_cast<const real *>(U[2]), static_cast<const real *>(U[3])}};
}

// face density and velocity v^a = g^a / (rho0 + (drho_i + drho_{i+a}) / 2) of the a-face of cell (x, y, z)
template <typename real>
__device__ __forceinline__ real face_rho(const State<real> &U, const Geo &G, real rho0, int a, int x, int y, int z) {
  return rho0 + real(0.5) * (U.d[G.at(x, y, z)] + U.d[G.at(x + ex(a), y + ey(a), z + ez(a))]);
}
template <typename real>
__device__ __forceinline__ real face_v(const State<real> &U, const Geo &G, real rho0, int a, int x, int y, int z) {
  return U.g[a][G.at(x, y, z)] / face_rho(U, G, rho0, a, x, y, z);
}

template <typename real>
__device__ __forceinline__ void grid_coords(size_t i, const Geo &G, int &x, int &y, int &z) {
  x = int(i % size_t(G.nx));
  const size_t r = i / size_t(G.nx);
  y = int(r % size_t(G.ny));
  z = int(r / size_t(G.ny));
}

// ---------------------------------------------------------------- V^T
// Adds the transpose of the velocity map v = V(drho, g) applied to vbar:
//   gbar_a(i) += vbar_a(i) / rho^a_i,
//   rhobar(i) += 1/2 sum_a (rfbar_a(i) + rfbar_a(i - a)), rfbar_a = -vbar_a v_a / rho^a.
template <typename real>
__global__ void __launch_bounds__(kAdjThreads) k_adj_velocity_T(State<real> U, Geo G, real rho0,
                                                                 const real *__restrict__ vb0, const real *__restrict__ vb1,
                                                                 const real *__restrict__ vb2, real *bar0, real *bar1,
                                                                 real *bar2, real *bar3) {
  const real *vb[3] = {vb0, vb1, vb2};
  real *bg[3] = {bar1, bar2, bar3};
  const size_t cells = size_t(G.nx) * G.ny * G.nz;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < cells; i += size_t(gridDim.x) * blockDim.x) {
    int x, y, z;
    grid_coords<real>(i, G, x, y, z);
    real dr = real(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const real rf = face_rho(U, G, rho0, a, x, y, z);
      const real v = vb[a][i];
      bg[a][i] += v / rf;
      dr -= real(0.5) * v * U.g[a][i] / (rf * rf);
      const int xm = x - ex(a), ym = y - ey(a), zm = z - ez(a);
      const size_t im = G.at(xm, ym, zm);
      const real rfm = face_rho(U, G, rho0, a, xm, ym, zm);
      dr -= real(0.5) * vb[a][im] * U.g[a][im] / (rfm * rfm);
    }
    bar0[i] += dr;
  }
}

// ---------------------------------------------------------------- stage
struct StageAdjConsts {
  double coef;          // b_s dt: lambda = coef * (adjoint of U_{s+1})
  double inv_h, eta, lam2, rho0;
  int forcing, wave_axis, plane_index;
  double dpdA;          // d (drive amplitude of this stage) / d A
};

// Face velocities v^a = g^a / rho^a of the stage state U_s, read many times
// by the stage adjoint below.
template <typename real>
__global__ void __launch_bounds__(kAdjThreads) k_adj_face_velocity(State<real> U, Geo G, real rho0, real *v0, real *v1,
                                                                    real *v2) {
  real *v[3] = {v0, v1, v2};
  const size_t cells = size_t(G.nx) * G.ny * G.nz;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < cells; i += size_t(gridDim.x) * blockDim.x) {
    int x, y, z;
    grid_coords<real>(i, G, x, y, z);
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a][i] = U.g[a][i] / face_rho(U, G, rho0, a, x, y, z);
  }
}

template <typename real>
struct StageIn {
  const real *lam[4];   // adjoint of U_{s+1} (delta rho, g_x, g_y, g_z), scaled by coef when read
  const real *v[3];     // face velocities of U_s
  State<real> U;        // U_s
};

// Transpose of the rates R(U_s, pi) applied to lambda = coef * (adjoint of
// U_{s+1}) (App. A.2 flux form), for the A-faces of cell i:
//   Tbar_a(c)  = (lambda_a(c) - lambda_a(c - a)) / h        diagonal flux at centre c
//   Fbar_ab(c) = (lambda_a(c + b) - lambda_a(c)) / h        a-momentum flux along b on c's edge
// gathered into
//   gp = gbar_A(i) + vbar_A(i) / rho^A_i  (the advective momenta, the mass flux and V^T),
//   rf = -vbar_A(i) v_A(i) / rho^A_i      (for the density part, summed by the next kernel),
//   T0 = Tbar_A(i)                        (its sum over A is the adjoint of the centre pressure).
// The arrays of In may be global fields or a block's shared-memory tile;
// Idx maps an offset (dx, dy, dz) in {-1, 0, 1}^3 from the cell to an index
// of them, and i is the cell's own index.
template <typename real, int A, typename Idx>
__device__ __forceinline__ void stage_face(const StageIn<real> &In, const Idx &at, real coef, real inv_h, real eta,
                                           real lam2, real rho0, uint32_t i, real &gp, real &rf, real &T0) {
  constexpr int ax = A == 0, ay = A == 1, az = A == 2;
  constexpr int x = 0, y = 0, z = 0;   // offsets are relative to the cell
  const auto L = [&](int a, int xx, int yy, int zz) { return coef * In.lam[1 + a][at(xx, yy, zz)]; };
  const auto Tb = [&](int a, int xx, int yy, int zz) {
    return (L(a, xx, yy, zz) - L(a, xx - (a == 0), yy - (a == 1), zz - (a == 2))) * inv_h;
  };
  const auto Fb = [&](int a, int b, int xx, int yy, int zz) {
    return (L(a, xx + (b == 0), yy + (b == 1), zz + (b == 2)) - L(a, xx, yy, zz)) * inv_h;
  };
  const auto V = [&](int a, int xx, int yy, int zz) { return In.v[a][at(xx, yy, zz)]; };
  const auto Gm = [&](int a, int xx, int yy, int zz) { return In.U.g[a][at(xx, yy, zz)]; };
  // dvbar_A(c) = -2 eta Tbar_A(c) - lam2 sum_a Tbar_a(c)
  const auto DV = [&](int xx, int yy, int zz) {
    const real t0 = Tb(0, xx, yy, zz), t1 = Tb(1, xx, yy, zz), t2 = Tb(2, xx, yy, zz);
    return real(-2) * eta * (A == 0 ? t0 : (A == 1 ? t1 : t2)) - lam2 * (t0 + t1 + t2);
  };
  // diagonal fluxes at the centres i and i + A
  T0 = Tb(A, x, y, z);
  const real T1 = Tb(A, x + ax, y + ay, z + az);
  const real vm = V(A, x - ax, y - ay, z - az), v0 = In.v[A][i], vp = V(A, x + ax, y + ay, z + az);
  const real gm = Gm(A, x - ax, y - ay, z - az), g0 = In.U.g[A][i], gpl = Gm(A, x + ax, y + ay, z + az);
  real gb = real(0.25) * (T0 * (vm + v0) + T1 * (v0 + vp));
  real vb = real(0.25) * (T0 * (gm + g0) + T1 * (g0 + gpl));
  vb += (DV(x, y, z) - DV(x + ax, y + ay, z + az)) * inv_h;
  // edge fluxes on the edges of i and i - B
#pragma unroll
  for (int B = 0; B < 3; ++B) {
    if (B == A) continue;
    const int bx = B == 0, by = B == 1, bz = B == 2;
    const real Fab0 = Fb(A, B, x, y, z), Fab1 = Fb(A, B, x - bx, y - by, z - bz);
    const real Fba0 = Fb(B, A, x, y, z), Fba1 = Fb(B, A, x - bx, y - by, z - bz);
    gb += real(0.25) * (Fab0 * (V(B, x, y, z) + V(B, x + ax, y + ay, z + az)) +
                        Fab1 * (V(B, x - bx, y - by, z - bz) + V(B, x - bx + ax, y - by + ay, z - bz + az)));
    vb += real(0.25) * (Fba0 * (Gm(B, x, y, z) + Gm(B, x + ax, y + ay, z + az)) +
                        Fba1 * (Gm(B, x - bx, y - by, z - bz) + Gm(B, x - bx + ax, y - by + ay, z - bz + az)));
    // the viscous part of the (A, B) edge flux, shared by F_AB and F_BA
    vb += eta * inv_h * ((Fab0 + Fba0) - (Fab1 + Fba1));
  }
  // mass flux: d rho/dt = -(1/h) sum_a (g_a(i) - g_a(i - a))
  const uint32_t iA = at(x + ax, y + ay, z + az);
  gb -= coef * (In.lam[0][i] - In.lam[0][iA]) * inv_h;
  const real rfv = rho0 + real(0.5) * (In.U.d[i] + In.U.d[iA]);
  gp = gb + vb / rfv;
  rf = -vb * v0 / rfv;
}

// The stage adjoint's grid part for every cell (stage_face of the three
// face sets), and dpdA * sum_i pibar(i) profile(i) added to *gA (the drive is
// linear in A).  A block takes an 8 x 8 x 4 box of cells: it stages the 11
// fields the gathers read (the adjoint of U_{s+1}, the face velocities and
// momenta, delta rho) on the box and its one-cell periodic halo in shared
// memory, then each thread gathers its cell's ~100 neighbour values from
// there.
constexpr int kTileX = 8, kTileY = 8, kTileZ = 4;
constexpr int kHaloX = kTileX + 2, kHaloY = kTileY + 2, kHaloZ = kTileZ + 2;
constexpr int kHaloCells = kHaloX * kHaloY * kHaloZ;
constexpr int kTileFields = 11;
static_assert(kTileX * kTileY * kTileZ == kAdjThreads, "one thread per cell of the box");

template <typename real>
__global__ void __launch_bounds__(kAdjThreads) k_adj_stage_rates(StageIn<real> In, Geo G, StageAdjConsts k,
                                                                  const real *__restrict__ cos_table, real *gp0,
                                                                  real *gp1, real *gp2, real *rf0, real *rf1,
                                                                  real *rf2, real *pibar, double *gA) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *tile = reinterpret_cast<real *>(smem_raw);   // [kTileFields][kHaloCells]
  const real coef = real(k.coef), inv_h = real(k.inv_h), eta = real(k.eta), lam2 = real(k.lam2),
             rho0 = real(k.rho0);
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY, z0 = blockIdx.z * kTileZ;
  for (int h = threadIdx.x; h < kHaloCells; h += blockDim.x) {
    const int hx = h % kHaloX, hy = (h / kHaloX) % kHaloY, hz = h / (kHaloX * kHaloY);
    const size_t gi = G.at(x0 + hx - 1, y0 + hy - 1, z0 + hz - 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) tile[j * kHaloCells + h] = In.lam[j][gi];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      tile[(4 + a) * kHaloCells + h] = In.v[a][gi];
      tile[(7 + a) * kHaloCells + h] = In.U.g[a][gi];
    }
    tile[10 * kHaloCells + h] = In.U.d[gi];
  }
  __syncthreads();
  const int tx = threadIdx.x % kTileX, ty = (threadIdx.x / kTileX) % kTileY, tz = threadIdx.x / (kTileX * kTileY);
  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  double acc_A = 0.0;
  if (x < G.nx && y < G.ny && z < G.nz) {
    StageIn<real> T;
#pragma unroll
    for (int j = 0; j < 4; ++j) T.lam[j] = tile + j * kHaloCells;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T.v[a] = tile + (4 + a) * kHaloCells;
      T.U.g[a] = tile + (7 + a) * kHaloCells;
    }
    T.U.d = tile + 10 * kHaloCells;
    const int c = (tx + 1) + kHaloX * ((ty + 1) + kHaloY * (tz + 1));
    const auto at = [c](int dx, int dy, int dz) { return uint32_t(c + dx + kHaloX * (dy + kHaloY * dz)); };
    real g0, r0, t0, g1, r1, t1, g2, r2, t2;
    stage_face<real, 0>(T, at, coef, inv_h, eta, lam2, rho0, uint32_t(c), g0, r0, t0);
    stage_face<real, 1>(T, at, coef, inv_h, eta, lam2, rho0, uint32_t(c), g1, r1, t1);
    stage_face<real, 2>(T, at, coef, inv_h, eta, lam2, rho0, uint32_t(c), g2, r2, t2);
    const size_t i = size_t(IC_CHK(x, G.nx)) + size_t(G.nx) * (size_t(IC_CHK(y, G.ny)) + size_t(G.ny) * size_t(IC_CHK(z, G.nz)));
    gp0[i] = g0;
    gp1[i] = g1;
    gp2[i] = g2;
    rf0[i] = r0;
    rf1[i] = r1;
    rf2[i] = r2;
    const real pb = t0 + t1 + t2;
    pibar[i] = pb;
    const int cw = k.wave_axis == 0 ? x : (k.wave_axis == 1 ? y : z);
    if (k.forcing == IC_FORCE_MODE)
      acc_A = double(pb) * double(cos_table[cw]);
    else if (k.forcing == IC_FORCE_PLANE && cw == k.plane_index)
      acc_A = double(pb);
  }
  if (k.forcing != IC_FORCE_NONE) {
    acc_A = warp_sum(acc_A);
    __shared__ double red[kAdjThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc_A;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < int(blockDim.x) / 32; ++w) sum += red[w];
      atomicAdd(gA, k.dpdA * sum);
    }
  }
}

// Adjoint of U_s from the adjoint of U_{s+1}:
//   rhobar_s(i) = b_s rhobar(i) + c^2 pibar(i) + 1/2 sum_a (rfbar_a(i) + rfbar_a(i - a)) + rhox(i)
//   gbar_s,a(i) = b_s gbar_a(i) + gpart_a(i)
// with rhox the particle-pressure part (spread by the particle kernel; cleared
// here).  a_s times the adjoint of U_{s+1} goes to the U^n accumulator; after
// the first stage (s = 0, whose U_s is U^n) the accumulator is folded in.
template <typename real>
__global__ void __launch_bounds__(kAdjThreads) k_adj_stage_combine(Geo G, real a_s, real b_s, real c2, int last,
                                                                    real *b0, real *b1, real *b2, real *b3, real *c0,
                                                                    real *c1, real *c2a, real *c3,
                                                                    const real *__restrict__ gp0, const real *__restrict__ gp1,
                                                                    const real *__restrict__ gp2, const real *__restrict__ rf0,
                                                                    const real *__restrict__ rf1, const real *__restrict__ rf2,
                                                                    const real *__restrict__ pibar, real *rhox) {
  real *bar[4] = {b0, b1, b2, b3};
  real *acc[4] = {c0, c1, c2a, c3};
  const real *gp[3] = {gp0, gp1, gp2};
  const real *rf[3] = {rf0, rf1, rf2};
  const size_t cells = size_t(G.nx) * G.ny * G.nz;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < cells; i += size_t(gridDim.x) * blockDim.x) {
    int x, y, z;
    grid_coords<real>(i, G, x, y, z);
    real nr = b_s * bar[0][i] + c2 * pibar[i] + rhox[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) nr += real(0.5) * (rf[a][i] + rf[a][G.at(x - ex(a), y - ey(a), z - ez(a))]);
    real nv[4] = {nr, b_s * bar[1][i] + gp[0][i], b_s * bar[2][i] + gp[1][i], b_s * bar[3][i] + gp[2][i]};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (a_s != real(0)) acc[j][i] += a_s * bar[j][i];
      bar[j][i] = last ? nv[j] + acc[j][i] : nv[j];
    }
    rhox[i] = real(0);
  }
}

// ---------------------------------------------------------------- particles
// d/dr of the three 1D weights of peskin3 (r = s - i0), times 1/h for d/dq:
// with S = sqrt(1 - 3 r^2), dS/dr = -3 r / S, so
//   d/dr (2 - 3r - S)/6 = (r/S - 1)/2, d/dr (1 + S)/3 = -r/S, d/dr (2 + 3r - S)/6 = (r/S + 1)/2.
template <typename real>
__device__ __forceinline__ void dpeskin3(real r, real inv_h, real dw[3]) {
  const real rs = r / sqrt(real(1) - real(3) * r * r);
  dw[0] = real(0.5) * (rs - real(1)) * inv_h;
  dw[1] = -rs * inv_h;
  dw[2] = real(0.5) * (rs + real(1)) * inv_h;
}

// Stencil of one position: for the centre set (0) and the own-axis face set
// (1) of each axis, the base index, the three 1D weights and their
// derivatives with respect to q along that axis.
template <typename real>
struct Sten {
  int b[2][3];
  real w[2][3][3], dw[2][3][3];
};

template <typename real>
__device__ void stencil_at(const typename Pos<real>::T *q, const PConsts<real> &pc, Sten<real> &S) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int bc, bf;
    real rc, rf;
    Pos<real>::axis(q[a], pc, a, bc, rc, bf, rf);
    S.b[0][a] = bc;
    S.b[1][a] = bf;
    peskin3(rc, S.w[0][a]);
    peskin3(rf, S.w[1][a]);
    dpeskin3(rc, pc.inv_h, S.dw[0][a]);
    dpeskin3(rf, pc.inv_h, S.dw[1][a]);
  }
}

// One warp per particle: lane t < 27 holds point t = (t % 3, (t / 3) % 3,
// t / 9) - 1 of a location set (0 centre, 1 + a the a-faces).  Returns false
// on the other lanes; else the cell, its coordinates, the weight and its
// gradient with respect to q.
template <typename real>
__device__ __forceinline__ bool point_of(const Sten<real> &S, int set, const Geo &G, int lane, size_t &i, int &x,
                                         int &y, int &z, real &w, real dw[3]) {
  if (lane >= 27) return false;
  const int dx = lane % 3, dy = (lane / 3) % 3, dz = lane / 9;
  const int sx = set == 1, sy = set == 2, sz = set == 3;
  const real wx = S.w[sx][0][dx], wy = S.w[sy][1][dy], wz = S.w[sz][2][dz];
  x = pw(S.b[sx][0] + dx - 1, G.nx);
  y = pw(S.b[sy][1] + dy - 1, G.ny);
  z = pw(S.b[sz][2] + dz - 1, G.nz);
  i = G.at(x, y, z);
  w = wx * wy * wz;
  dw[0] = S.dw[sx][0][dx] * wy * wz;
  dw[1] = wx * S.dw[sy][1][dy] * wz;
  dw[2] = wx * wy * S.dw[sz][2][dz];
  return true;
}

// warp sum, the same value (lane 0's) on every lane
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// J f (FP64 sum) and its gradient with respect to q; val(i, x, y, z) gives f
template <typename real, typename Val>
__device__ __forceinline__ void interp_grad(const Sten<real> &S, int set, const Geo &G, int lane, Val val, double &J,
                                            double dJ[3]) {
  double j = 0.0, a = 0.0, b = 0.0, c = 0.0;
  size_t i;
  int x, y, z;
  real w, dw[3];
  if (point_of<real>(S, set, G, lane, i, x, y, z, w, dw)) {
    const double f = double(val(i, x, y, z));
    j = double(w) * f;
    a = double(dw[0]) * f;
    b = double(dw[1]) * f;
    c = double(dw[2]) * f;
  }
  J = wsum(j);
  dJ[0] = wsum(a);
  dJ[1] = wsum(b);
  dJ[2] = wsum(c);
}

// transpose of J: point i of set `set` receives w_i * value
template <typename real>
__device__ __forceinline__ void spread_T(const Sten<real> &S, int set, const Geo &G, int lane, real *field,
                                         double value) {
  size_t i;
  int x, y, z;
  real w, dw[3];
  if (point_of<real>(S, set, G, lane, i, x, y, z, w, dw)) atomicAdd(field + i, real(double(w) * value));
}

template <typename real>
struct AdjParticles {
  int n;
  const typename Pos<real>::T *q_half, *q_n;
  const real *u_n, *m_e, *eps, *k_s, *force, *dg;
  double *qbar, *ubar, *qhbar, *fbar, *jvnh, *gme, *geps;
  const double *dir;
};

template <typename real>
AdjParticles<real> adj_particles(const ic_ctx *ctx, const AdjStepTape &t) {
  using T = typename Pos<real>::T;
  const ParticleStore &s = ctx->ps;
  const AdjointStore &A = ctx->adj;
  AdjParticles<real> P;
  P.n = s.n;
  P.q_half = (const T *)t.q_half;
  P.q_n = (const T *)t.q_n;
  P.u_n = (const real *)t.u_n;
  P.m_e = (const real *)s.m_e;
  P.eps = (const real *)s.eps;
  P.k_s = (const real *)s.k_s;
  P.force = (const real *)t.force;
  P.dg = (const real *)t.dg;
  P.qbar = A.qbar;
  P.ubar = A.ubar;
  P.qhbar = A.qhbar;
  P.fbar = A.fbar;
  P.jvnh = A.jvnh;
  P.gme = A.gme;
  P.geps = A.geps;
  P.dir = A.dir;
  return P;
}

// v^a of the face (x, y, z) of a state
template <typename real>
struct FaceV {
  State<real> U;
  Geo G;
  real rho0;
  int a;
  __device__ __forceinline__ real operator()(size_t i, int x, int y, int z) const {
    return U.g[a][i] / (rho0 + real(0.5) * (U.d[i] + U.d[G.at(x + ex(a), y + ey(a), z + ez(a))]));
  }
};

// plain field values
template <typename real>
struct FieldV {
  const real *f;
  real scale;
  __device__ __forceinline__ real operator()(size_t i, int, int, int) const { return scale * f[i]; }
};

template <typename real>
struct Fields3 {
  real *f[3];
};

__device__ __forceinline__ int warp_particle() { return int((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }

// Substep 7 reversed: jv_new_bar = jv_nh_bar = dt/2 qbar (kept for the last
// kernel); vbar_a += J^T jv_new_bar_a at q^{n+1/2};
// qhbar = sum_a jv_new_bar_a d(J v^{n+1}_a)/dq; fbar = 0.
template <typename real>
__global__ void __launch_bounds__(kAdjParticleThreads) k_adj_p_final(AdjParticles<real> P, State<real> Unew, Geo G,
                                                                      PConsts<real> pc, Fields3<real> vb) {
  const int p = warp_particle(), lane = threadIdx.x & 31;
  if (p >= P.n) return;
  Sten<real> S;
  stencil_at<real>(P.q_half + 3 * p, pc, S);
  // every gather before any spread, so that the loads are not held behind
  // the atomics (the arithmetic is the same, in the same order)
  double J[3], dJ[3][3], jb[3];
  for (int a = 0; a < 3; ++a) {
    jb[a] = 0.5 * double(pc.dt) * P.qbar[3 * p + a];
    interp_grad<real>(S, 1 + a, G, lane, FaceV<real>{Unew, G, pc.rho0, a}, J[a], dJ[a]);
  }
  double qh[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) qh[c] += jb[a] * dJ[a][c];
  for (int a = 0; a < 3; ++a) {
    spread_T<real>(S, 1 + a, G, lane, vb.f[a], jb[a]);
    if (lane == 0) {
      P.jvnh[3 * p + a] = jb[a];
      P.fbar[3 * p + a] = 0.0;
    }
  }
  if (lane == 0)
    for (int c = 0; c < 3; ++c) P.qhbar[3 * p + c] = qh[c];
}

// Substeps 6, 5 and 4 reversed (after V^T of v^{n+1} has been added to bar):
//   dg_bar_a = -(1/h^3) J_a gbar_a                       (g^{n+1} = g~ - S dg)
//   jvt_bar = r ubar + mu dg_bar, u^n_bar = (1 - r) ubar - mu dg_bar
//   m_f_bar, m_e gradient from r = m_f / (m_e + m_f), mu = m_e r
//   rhobar += V m_f_bar J_c^T                              (m_f = V (rho0 + J_c rho^{n+1}))
//   vbar_a += J_a^T jvt_bar_a                              (J v~ at q^{n+1/2})
// plus every term's gradient with respect to q^{n+1/2}.
template <typename real>
__global__ void __launch_bounds__(kAdjParticleThreads) k_adj_p_impulse(AdjParticles<real> P, State<real> U3, Geo G,
                                                                        PConsts<real> pc, Fields3<real> vb,
                                                                        const real *gbar0, const real *gbar1,
                                                                        const real *gbar2, real *rhobar) {
  const int p = warp_particle(), lane = threadIdx.x & 31;
  if (p >= P.n) return;
  const real *gb[3] = {gbar0, gbar1, gbar2};
  Sten<real> S;
  stencil_at<real>(P.q_half + 3 * p, pc, S);
  const double inv_h3 = double(pc.inv_h3), vol = double(pc.vol);
  double qh[3] = {P.qhbar[3 * p], P.qhbar[3 * p + 1], P.qhbar[3 * p + 2]};
  double dgb[3], jvt[3], djvt[3][3];
  for (int a = 0; a < 3; ++a) {
    double J, dJ[3];
    interp_grad<real>(S, 1 + a, G, lane, FieldV<real>{gb[a], real(1)}, J, dJ);
    dgb[a] = -J * inv_h3;
    const double dga = double(P.dg[3 * p + a]);
    for (int c = 0; c < 3; ++c) qh[c] -= dga * inv_h3 * dJ[c];
    interp_grad<real>(S, 1 + a, G, lane, FaceV<real>{U3, G, pc.rho0, a}, jvt[a], djvt[a]);
  }
  double Jr, dJr[3];
  interp_grad<real>(S, 0, G, lane, FieldV<real>{U3.d, real(1)}, Jr, dJr);
  const double me = double(P.m_e[p]), mf = vol * (double(pc.rho0) + Jr), tot = me + mf;
  const double r = mf / tot, mu = me * r;
  double su = 0.0, sg = 0.0, jvtb[3], ub_new[3];
  for (int a = 0; a < 3; ++a) {
    const double ub = P.ubar[3 * p + a], d = jvt[a] - double(P.u_n[3 * p + a]);
    jvtb[a] = r * ub + mu * dgb[a];
    ub_new[a] = (1.0 - r) * ub - mu * dgb[a];
    su += ub * d;
    sg += dgb[a] * d;
  }
  const double mfb = me / (tot * tot) * su + me * me / (tot * tot) * sg;
  spread_T<real>(S, 0, G, lane, rhobar, vol * mfb);
  for (int c = 0; c < 3; ++c) qh[c] += vol * mfb * dJr[c];
  for (int a = 0; a < 3; ++a) {
    for (int c = 0; c < 3; ++c) qh[c] += jvtb[a] * djvt[a][c];
    spread_T<real>(S, 1 + a, G, lane, vb.f[a], jvtb[a]);
  }
  if (lane == 0) {
    P.gme[p] += -mf / (tot * tot) * su + mf * mf / (tot * tot) * sg;
    for (int c = 0; c < 3; ++c) {
      P.ubar[3 * p + c] = ub_new[c];
      P.qhbar[3 * p + c] = qh[c];
    }
  }
}

// The particle terms of one RK stage reversed (before the stage's combine):
//   Omega_bar = J_c pibar / h^3, Omega = eps V J_c rho_s            (pi += S_c Omega)
//   eps gradient += V (J_c rho_s) Omega_bar; rhox += eps V Omega_bar J_c^T
//   F_bar_a += J_a lambda_a / h^3 with lambda = coef * gbar           (the source S F)
// plus their gradients with respect to q^{n+1/2}.
template <typename real>
__global__ void __launch_bounds__(kAdjParticleThreads) k_adj_p_stage(AdjParticles<real> P, State<real> Us, Geo G,
                                                                      PConsts<real> pc, const real *pibar,
                                                                      const real *gbar0, const real *gbar1,
                                                                      const real *gbar2, real coef, real *rhox) {
  const int p = warp_particle(), lane = threadIdx.x & 31;
  if (p >= P.n) return;
  const real *gb[3] = {gbar0, gbar1, gbar2};
  Sten<real> S;
  stencil_at<real>(P.q_half + 3 * p, pc, S);
  const double inv_h3 = double(pc.inv_h3), vol = double(pc.vol), eps = double(P.eps[p]);
  double qh[3] = {P.qhbar[3 * p], P.qhbar[3 * p + 1], P.qhbar[3 * p + 2]};
  // every gather before the spread (the arithmetic is the same, in the same order)
  double Jp, dJp[3], Jr, dJr[3], Jf[3], dJf[3][3];
  interp_grad<real>(S, 0, G, lane, FieldV<real>{pibar, real(1)}, Jp, dJp);
  interp_grad<real>(S, 0, G, lane, FieldV<real>{Us.d, real(1)}, Jr, dJr);
  for (int a = 0; a < 3; ++a) interp_grad<real>(S, 1 + a, G, lane, FieldV<real>{gb[a], coef}, Jf[a], dJf[a]);
  const double ob = Jp * inv_h3, om = eps * vol * Jr;
  for (int c = 0; c < 3; ++c) qh[c] += om * inv_h3 * dJp[c] + eps * vol * ob * dJr[c];
  double fb[3];
  for (int a = 0; a < 3; ++a) {
    fb[a] = Jf[a] * inv_h3;
    const double Fa = double(P.force[3 * p + a]);
    for (int c = 0; c < 3; ++c) qh[c] += Fa * inv_h3 * dJf[a][c];
  }
  spread_T<real>(S, 0, G, lane, rhox, eps * vol * ob);
  if (lane == 0) {
    P.geps[p] += vol * Jr * ob;
    for (int c = 0; c < 3; ++c) {
      P.fbar[3 * p + c] += fb[c];
      P.qhbar[3 * p + c] = qh[c];
    }
  }
}

// Substeps 2 and 1 reversed, with the objective's own term:
//   F_bar += weight * d_p; qhbar -= k_s F_bar                     (F = -k_s (q^{n+1/2} - q_eq))
//   vbar_a += J_a^T jv_nh_bar_a at q^{n+1/2} (J^{n+1/2} v^n of substep 7)
//   qbar += qhbar; jv_n_bar = dt/2 qhbar; vbar_a += J_a^T jv_n_bar_a at q^n
// plus the gradients with respect to q^{n+1/2} and q^n.
template <typename real>
__global__ void __launch_bounds__(kAdjParticleThreads) k_adj_p_start(AdjParticles<real> P, State<real> Un, Geo G,
                                                                      PConsts<real> pc, Fields3<real> vb,
                                                                      double weight) {
  const int p = warp_particle(), lane = threadIdx.x & 31;
  if (p >= P.n) return;
  Sten<real> S;
  stencil_at<real>(P.q_half + 3 * p, pc, S);
  double qh[3];
  for (int c = 0; c < 3; ++c) {
    const double fbar = P.fbar[3 * p + c] + weight * P.dir[3 * p + c];
    qh[c] = P.qhbar[3 * p + c] - double(P.k_s[p]) * fbar;
  }
  // every gather (at q^{n+1/2} and at q^n) before any spread, so that the
  // loads are not held behind the atomics; the arithmetic is the same, in
  // the same order
  Sten<real> S0;
  stencil_at<real>(P.q_n + 3 * p, pc, S0);
  double J1[3], dJ1[3][3], J0[3], dJ0[3][3], jb1[3], jb0[3];
  for (int a = 0; a < 3; ++a) {
    jb1[a] = P.jvnh[3 * p + a];
    interp_grad<real>(S, 1 + a, G, lane, FaceV<real>{Un, G, pc.rho0, a}, J1[a], dJ1[a]);
    interp_grad<real>(S0, 1 + a, G, lane, FaceV<real>{Un, G, pc.rho0, a}, J0[a], dJ0[a]);
  }
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) qh[c] += jb1[a] * dJ1[a][c];
  double qb[3];
  for (int c = 0; c < 3; ++c) qb[c] = P.qbar[3 * p + c] + qh[c];
  for (int a = 0; a < 3; ++a) {
    jb0[a] = 0.5 * double(pc.dt) * qh[a];
    for (int c = 0; c < 3; ++c) qb[c] += jb0[a] * dJ0[a][c];
  }
  for (int a = 0; a < 3; ++a) spread_T<real>(S, 1 + a, G, lane, vb.f[a], jb1[a]);
  for (int a = 0; a < 3; ++a) spread_T<real>(S0, 1 + a, G, lane, vb.f[a], jb0[a]);
  if (lane == 0)
    for (int c = 0; c < 3; ++c) P.qbar[3 * p + c] = qb[c];
}

// ---------------------------------------------------------------- host
// d (drive amplitude of RK stage s of the given step) / d A
double stage_dpdA(const ic_ctx *ctx, int64_t step, int s) {
  const ic_grid_params &p = ctx->p;
  const double gamma = (4.0 * p.eta / 3.0 + p.zeta) / (2.0 * p.rho0);
  const int n_ax = p.wave_axis == 0 ? p.nx : (p.wave_axis == 1 ? p.ny : p.nz);
  const double per_A = p.forcing == IC_FORCE_MODE ? 2.0 * gamma * ctx->omega : double(n_ax) * gamma * ctx->omega;
  return per_A * std::sin(ctx->omega * (double(step) + kStageTimes[s]) * p.dt + p.wave_phase);
}

// The node a capturing stream added last (its single dependency), or null.
cudaGraphNode_t captured_node(cudaStream_t st) {
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive || nd != 1)
    return nullptr;
  return deps[0];
}

template <typename real>
cudaError_t adjoint_step_t(ic_ctx *ctx, const AdjStepTape &t, double weight, AdjGraph *cap) {
  AdjointStore &A = ctx->adj;
  const ic_grid_params &p = ctx->p;
  const Geo G{p.nx, p.ny, p.nz};
  const PConsts<real> pc = particle_consts<real>(ctx);
  const size_t cells = size_t(ctx->cells);
  const size_t fb = cells * sizeof(real);
  cudaStream_t st = ctx->stream;
  const int gblocks = int(std::min<size_t>((cells + kAdjThreads - 1) / kAdjThreads, size_t(ctx->sm_count) * 8));
  const int n = ctx->ps.n;
  constexpr int kParticlesPerBlock = kAdjParticleThreads / 32;
  const int pblocks = (n + kParticlesPerBlock - 1) / kParticlesPerBlock;
  const AdjParticles<real> P = adj_particles<real>(ctx, t);
  real *bar[4], *acc[4], *gp[3], *rf[3], *vel[3];
  Fields3<real> vb;
  for (int j = 0; j < 4; ++j) {
    bar[j] = static_cast<real *>(A.bar[j]);
    acc[j] = static_cast<real *>(A.acc[j]);
  }
  for (int a = 0; a < 3; ++a) {
    vb.f[a] = static_cast<real *>(A.vbar[a]);
    gp[a] = static_cast<real *>(A.gpart[a]);
    rf[a] = static_cast<real *>(A.rfbar[a]);
    vel[a] = static_cast<real *>(A.vel[a]);
  }
  real *pibar = static_cast<real *>(A.pibar), *rhox = static_cast<real *>(A.rhox);
  // the recorded step's states
  void *const *Un = t.Un;
  void *const *Unew = t.Unew;
  void *const U3v[4] = {Unew[0], t.G3[0], t.G3[1], t.G3[2]};
  void *const *Ustage[3] = {t.Un, t.U1, t.U2};
  const real rho0 = real(p.rho0);
  auto vt = [&](void *const *U) {
    cudaError_t e = timed_launch(ctx, kClassGrid, [&] {
      k_adj_velocity_T<real><<<gblocks, kAdjThreads, 0, st>>>(state_of<real>(U), G, rho0, vb.f[0], vb.f[1],
                                                               vb.f[2], bar[0], bar[1], bar[2], bar[3]);
      return cudaGetLastError();
    });
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = cudaMemsetAsync(vb.f[a], 0, fb, st);
    return e;
  };
  cudaError_t e = cudaSuccess;
#define IC_ADJ_TRY(x)                      \
  do {                                     \
    if ((e = (x)) != cudaSuccess) return e; \
  } while (0)
  for (int j = 0; j < 4; ++j) IC_ADJ_TRY(cudaMemsetAsync(acc[j], 0, fb, st));
  if (n > 0) {
    IC_ADJ_TRY(timed_launch(ctx, kClassParticles, [&] {
      k_adj_p_final<real><<<pblocks, kAdjParticleThreads, 0, st>>>(P, state_of<real>(Unew), G, pc, vb);
      return cudaGetLastError();
    }));
    IC_ADJ_TRY(vt(Unew));
    IC_ADJ_TRY(timed_launch(ctx, kClassParticles, [&] {
      k_adj_p_impulse<real><<<pblocks, kAdjParticleThreads, 0, st>>>(P, state_of<real>(U3v), G, pc, vb, bar[1],
                                                                     bar[2], bar[3], bar[0]);
      return cudaGetLastError();
    }));
    IC_ADJ_TRY(vt(U3v));
  }
  const real *cos_table = sizeof(real) == 4 ? (const real *)ctx->cos_table_f : (const real *)ctx->cos_table;
  for (int s = 2; s >= 0; --s) {
    StageAdjConsts k;
    k.coef = kB[s] * p.dt;
    k.inv_h = 1.0 / p.h;
    k.eta = p.eta;
    k.lam2 = p.zeta - 2.0 * p.eta / 3.0;
    k.rho0 = p.rho0;
    k.forcing = p.forcing;
    k.wave_axis = p.wave_axis;
    k.plane_index = p.plane_index;
    k.dpdA = stage_dpdA(ctx, t.step, s);
    const State<real> Us = state_of<real>(Ustage[s]);
    StageIn<real> In;
    for (int j = 0; j < 4; ++j) In.lam[j] = bar[j];
    for (int a = 0; a < 3; ++a) In.v[a] = vel[a];
    In.U = Us;
    IC_ADJ_TRY(timed_launch(ctx, kClassGrid, [&] {
      k_adj_face_velocity<real><<<gblocks, kAdjThreads, 0, st>>>(Us, G, rho0, vel[0], vel[1], vel[2]);
      return cudaGetLastError();
    }));
    constexpr size_t smem = size_t(kTileFields) * kHaloCells * sizeof(real);
    const dim3 tiles((p.nx + kTileX - 1) / kTileX, (p.ny + kTileY - 1) / kTileY, (p.nz + kTileZ - 1) / kTileZ);
    IC_ADJ_TRY(timed_launch(ctx, kClassStage, [&] {
      if (smem > 48 * 1024) cudaFuncSetAttribute(k_adj_stage_rates<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(smem));
      k_adj_stage_rates<real><<<tiles, kAdjThreads, smem, st>>>(In, G, k, cos_table, gp[0], gp[1], gp[2], rf[0],
                                                                rf[1], rf[2], pibar, A.gA);
      return cudaGetLastError();
    }));
    if (cap) {   // the drive derivative changes with the step: keep the node
      const cudaGraphNode_t nd = captured_node(st);
      if (!nd) return cudaErrorStreamCaptureUnsupported;
      cap->rates[s].keep(nd, reinterpret_cast<const void *>(k_adj_stage_rates<real>), tiles, dim3(kAdjThreads), smem, In,
                         G, k, cos_table, gp[0], gp[1], gp[2], rf[0], rf[1], rf[2], pibar, A.gA);
    }
    if (n > 0) {
      IC_ADJ_TRY(timed_launch(ctx, kClassParticles, [&] {
        k_adj_p_stage<real><<<pblocks, kAdjParticleThreads, 0, st>>>(P, Us, G, pc, pibar, bar[1], bar[2], bar[3],
                                                                     real(k.coef), rhox);
        return cudaGetLastError();
      }));
    }
    IC_ADJ_TRY(timed_launch(ctx, kClassGrid, [&] {
      k_adj_stage_combine<real><<<gblocks, kAdjThreads, 0, st>>>(G, real(kA[s]), real(kB[s]), real(p.c * p.c),
                                                                 s == 0, bar[0], bar[1], bar[2], bar[3], acc[0],
                                                                 acc[1], acc[2], acc[3], gp[0], gp[1], gp[2], rf[0],
                                                                 rf[1], rf[2], pibar, rhox);
      return cudaGetLastError();
    }));
  }
  if (n > 0) {
    IC_ADJ_TRY(timed_launch(ctx, kClassParticles, [&] {
      k_adj_p_start<real><<<pblocks, kAdjParticleThreads, 0, st>>>(P, state_of<real>(Un), G, pc, vb, weight);
      return cudaGetLastError();
    }));
    if (cap) {   // the weight changes with the step: keep the node
      const cudaGraphNode_t nd = captured_node(st);
      if (!nd) return cudaErrorStreamCaptureUnsupported;
      cap->start.keep(nd, reinterpret_cast<const void *>(k_adj_p_start<real>), dim3(pblocks), dim3(kAdjParticleThreads),
                      0, P, state_of<real>(Un), G, pc, vb, weight);
    }
    IC_ADJ_TRY(vt(Un));
  }
#undef IC_ADJ_TRY
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_adjoint_step(ic_ctx *ctx, const AdjStepTape &t, double weight, AdjGraph *cap) {
  if (ctx->p.precision == IC_FP32) return adjoint_step_t<float>(ctx, t, weight, cap);
  return adjoint_step_t<double>(ctx, t, weight, cap);
}

cudaError_t update_adjoint_graph(const ic_ctx *ctx, AdjGraph &g, const AdjStepTape &t, double weight) {
  for (int s = 0; s < 3; ++s) {
    KeptNode &n = g.rates[s];
    if (!n.node) continue;
    if (n.arg.size() != 12 || n.arg[2].size() != sizeof(StageAdjConsts)) return cudaErrorInvalidValue;
    StageAdjConsts k;
    std::memcpy(&k, n.arg[2].data(), sizeof(k));
    k.dpdA = stage_dpdA(ctx, t.step, s);
    std::memcpy(n.arg[2].data(), &k, sizeof(k));
    const cudaError_t e = cudaGraphExecKernelNodeSetParams(g.exec, n.node, &n.p);
    if (e != cudaSuccess) return e;
  }
  if (g.start.node) {
    if (g.start.arg.size() != 6 || g.start.arg[5].size() != sizeof(double)) return cudaErrorInvalidValue;
    std::memcpy(g.start.arg[5].data(), &weight, sizeof(weight));
    return cudaGraphExecKernelNodeSetParams(g.exec, g.start.node, &g.start.p);
  }
  return cudaSuccess;
}

IC_BOUNDS_READER(bounds_flag_adjoint)

}  // namespace ic
