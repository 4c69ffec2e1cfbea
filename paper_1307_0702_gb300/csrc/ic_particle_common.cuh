// Particle storage as the device kernels see it, shared by the particle
// kernels of the step (ic_particles.cu) and of its adjoint (ic_adjoint.cu):
// the position representation of each precision, the per-launch constants
// and typed views of the particle and grid arrays.
#pragma once
#include <cuda_runtime.h>

#include "ic_device.cuh"
#include "ic_internal.hpp"

namespace ic {

constexpr int kFixBits = 40;

template <typename real>
struct PConsts {
  int n[3];
  real h, inv_h, dt, rho0, vol, inv_h3;
  real L[3];
  long long span[3];   // n << kFixBits (FP32 positions)
  real cutoff;         // neighbour cutoff per axis (length)
  real rebuild_at;     // displacement since build that triggers a rebuild
  real skin_limit;     // displacement at which a list is no longer valid
  int nb[3], nbins;    // neighbour bins per axis and in all
};

template <typename real>
struct Pos;

// FP64 positions: length units, wrapped into [0, L).
template <>
struct Pos<double> {
  using T = double;
  __device__ static void axis(T q, const PConsts<double> &pc, int a, int &bc, double &rc, int &bf, double &rf) {
    const int n = a == 0 ? pc.n[0] : (a == 1 ? pc.n[1] : pc.n[2]);
    const double s = q / pc.h;
    const double fc = floor(s + 0.5);
    rc = s - fc;
    bc = wrap(int(fc), n);
    const double sf = s - 0.5;
    const double ff = floor(sf + 0.5);
    rf = sf - ff;
    bf = wrap(int(ff), n);
  }
  __device__ static int cell(T q, const PConsts<double> &pc, int a) {   // floor(q / h) in [0, n)
    const int n = a == 0 ? pc.n[0] : (a == 1 ? pc.n[1] : pc.n[2]);
    return min(max(int(floor(q / pc.h)), 0), n - 1);
  }
  __device__ static T advance(T q, double dq, const PConsts<double> &pc, int a) {
    const double L = a == 0 ? pc.L[0] : (a == 1 ? pc.L[1] : pc.L[2]);
    double r = fmod(q + dq, L);
    if (r < 0.0) r += L;
    if (r >= L) r -= L;
    return r;
  }
  __device__ static double diff(T x, T y, const PConsts<double> &pc, int a) {   // minimum image x - y
    const double L = a == 0 ? pc.L[0] : (a == 1 ? pc.L[1] : pc.L[2]);
    const double d = x - y;
    return d - L * rint(d / L);
  }
};

// FP32 positions: fixed point q / h in units of 2^-40, wrapped into [0, n 2^40).
template <>
struct Pos<float> {
  using T = long long;
  __device__ static void axis(T q, const PConsts<float> &pc, int a, int &bc, float &rc, int &bf, float &rf) {
    const int n = a == 0 ? pc.n[0] : (a == 1 ? pc.n[1] : pc.n[2]);
    const int cell = int(q >> kFixBits);
    const float frac = __uint2float_rn(uint32_t(q >> (kFixBits - 24)) & 0xFFFFFFu) * 0x1p-24f;   // [0, 1)
    // centre set: s = cell + frac, i0 = floor(s + 1/2); face set: i0 = floor(s) = cell
    const bool up = frac >= 0.5f;
    bc = up ? (cell + 1 == n ? 0 : cell + 1) : cell;
    rc = up ? frac - 1.0f : frac;
    bf = cell;
    rf = frac - 0.5f;
  }
  __device__ static int cell(T q, const PConsts<float> &, int) { return int(q >> kFixBits); }   // [0, n)
  __device__ static T advance(T q, float dq, const PConsts<float> &pc, int a) {
    const long long span = a == 0 ? pc.span[0] : (a == 1 ? pc.span[1] : pc.span[2]);
    // a non-finite displacement (a state that blew up, which the end-of-step
    // check reports) leaves the particle in place; any finite one wraps into
    // [0, span), so that no index derived from q leaves the grid
    const float d = dq * pc.inv_h * 0x1p40f;
    T r = q + (isfinite(d) ? __float2ll_rn(d) : 0ll);
    if (r < 0 || r >= span) {
      r %= span;
      if (r < 0) r += span;
    }
    return r;
  }
  __device__ static float diff(T x, T y, const PConsts<float> &pc, int a) {   // minimum image x - y (length)
    const long long span = a == 0 ? pc.span[0] : (a == 1 ? pc.span[1] : pc.span[2]);
    long long d = x - y;
    if (2 * d >= span) d -= span;
    if (2 * d < -span) d += span;
    // d = hi 2^32 + lo: two exact 32-bit conversions instead of an int64 one
    const float cells = __int2float_rn(int(d >> 32)) * 0x1p-8f + __uint2float_rn(uint32_t(d)) * 0x1p-40f;
    return cells * pc.h;
  }
};

template <typename real>
struct PV {
  using P = typename Pos<real>::T;
  int n;
  P *q, *q_eq, *q_build, *q_half;
  double *acc;
  real *u, *m_e, *eps, *k_s, *w, *jv_n, *force, *dg, *lam, *jrho;
  int *base, *nbr, *nnbr, *order, *bins;
};

template <typename real>
PV<real> view(const ParticleStore &s) {
  using P = typename Pos<real>::T;
  PV<real> v;
  v.n = s.n;
  v.q = (P *)s.q;
  v.q_eq = (P *)s.q_eq;
  v.q_build = (P *)s.q_build;
  v.q_half = (P *)s.q_half;
  v.acc = s.acc;
  v.u = (real *)s.u;
  v.m_e = (real *)s.m_e;
  v.eps = (real *)s.eps;
  v.k_s = (real *)s.k_s;
  v.w = (real *)s.w;
  v.jv_n = (real *)s.jv_n;
  v.force = (real *)s.force;
  v.dg = (real *)s.dg;
  v.lam = (real *)s.lam;
  v.jrho = (real *)s.jrho;
  v.base = s.base;
  v.nbr = s.nbr;
  v.nnbr = s.nnbr;
  v.order = s.order;
  v.bins = s.bins;
  return v;
}

template <typename real>
struct Grid4 {
  real *f[4];   // delta rho, g_x, g_y, g_z
};

template <typename real>
PConsts<real> particle_consts(const ic_ctx *ctx) {
  const ic_grid_params &p = ctx->p;
  PConsts<real> c{};
  const int n[3] = {p.nx, p.ny, p.nz};
  for (int a = 0; a < 3; ++a) {
    c.n[a] = n[a];
    c.L[a] = real(n[a] * p.h);
    c.span[a] = (long long)n[a] << kFixBits;
  }
  c.h = real(p.h);
  c.inv_h = real(1.0 / p.h);
  c.inv_h3 = real(1.0 / (p.h * p.h * p.h));
  c.dt = real(p.dt);
  c.rho0 = real(p.rho0);
  c.vol = real(8.0 * p.h * p.h * p.h);   // V = 1 / (J S) = 8 h^3 (Eq. (kvol))
  c.cutoff = real((4.0 + kSkin) * p.h);
  c.rebuild_at = real(0.25 * kSkin * p.h);
  c.skin_limit = real(0.5 * kSkin * p.h);
  c.nbins = neighbour_bins(p, c.nb);
  return c;
}

template <typename real>
Grid4<real> grid4(void *const U[4]) {
  Grid4<real> g;
  for (int j = 0; j < 4; ++j) g.f[j] = static_cast<real *>(U[j]);
  return g;
}

}  // namespace ic
