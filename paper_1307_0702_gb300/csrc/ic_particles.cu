// Particle kernels of libic: the particle substeps of App. A.2 coupled to the
// grid through the 3-point kernel (App. A.1).  One group of 16 lanes per
// particle (two per warp); each lane holds two of the 27 points of a location
// set.
//
// Per step (the fluid stages run in ic_fluid.cu between these launches):
//   kHalfStep   substeps 1-2: J^n v^n at q^n -> q^{n+1/2}; F^{n+1/2};
//               stencils at q^{n+1/2}; J^{n+1/2} v^n
//   kPressure   before each RK stage s: the particle pressure S Omega_s on the
//               centre cells (read by the stage kernel as part of pi)
//   kForce      after each RK stage s, only with tethers: b_s dt S F
//   kImpulse    substeps 4-5: dg, u^{n+1}, lambda from J v~^{n+1}
//   kSpread     substep 6: g^{n+1} = g~^{n+1} - S dg
//   kFinal      substep 7: q^{n+1}; weighted force sums; clears the pressure;
//               its last CTA sorts the neighbour bins (when due) and does the
//               end-of-step bookkeeping
//
// Spreading is deterministic and free of atomics: each grid point near
// particles is written by exactly one particle (its "owner": the lowest index
// among the particles whose stencil holds the point), which sums the
// contributions of itself and its neighbours in ascending index order.
// Neighbour lists (|dq_a| < 4h + skin on every axis) are rebuilt when a
// particle has moved more than a quarter skin: a counting sort of the
// particles into bins of whole cells at least the cutoff wide (kBin), then
// each particle tests the members of the 27 bins around its own and sorts its
// hits by index, so a rebuild is O(N_p) and gives the same ascending lists as
// a scan of all pairs would.
//
// Positions.  The FP64 path keeps positions in length units (double).  The
// FP32 path keeps them in 64-bit fixed point, q / h in units of 2^-40, so
// that no FP64 arithmetic runs in its kernels (GB300's FP64 rate is a small
// fraction of its FP32 rate) while a tethered particle's 1e-6 h displacement
// stays resolved; its weights and forces are FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ic_device.cuh"
#include "ic_end_step.cuh"
#include "ic_internal.hpp"
#include "ic_particle_common.cuh"

namespace ic {
namespace {

// Lanes of the group that serves one particle: kGroup consecutive lanes of a
// warp (two particles per warp), each lane holding up to kPointsPerLane of the
// 27 points of a location set.  With 1e4 particles a group of 16 keeps every
// particle of a launch resident at once on 152 SMs (a warp per particle would
// need more warps than the SMs hold and run the latency-bound work in waves).
constexpr int kGroup = 16;
constexpr int kPointsPerLane = (27 + kGroup - 1) / kGroup;
constexpr int kBlockThreads = 128;
constexpr int kGroupsPerBlock = kBlockThreads / kGroup;
// resident blocks per SM the register budget is sized for: in FP32 9 x 8 = 72
// particles per SM, 10944 on 152 SMs; FP64 keeps more registers per lane
template <typename real>
constexpr int min_blocks() { return sizeof(real) == 4 ? 9 : 5; }

struct Lanes {
  int sub;         // lane within the group
  unsigned mask;   // the group's lanes in the warp
};

__device__ __forceinline__ Lanes group_lanes() {
  const int lane = threadIdx.x & 31;
  return {lane & (kGroup - 1), kGroup == 32 ? 0xffffffffu : (((1u << kGroup) - 1u) << (lane & ~(kGroup - 1)))};
}

__device__ __forceinline__ int group_particle() { return int((blockIdx.x * kBlockThreads + threadIdx.x) / kGroup); }

template <typename T>
__device__ __forceinline__ T gshfl(const Lanes &L, T v, int src) { return __shfl_sync(L.mask, v, src, kGroup); }

template <typename real>
__device__ __forceinline__ real group_sum(const Lanes &L, real v) {
#pragma unroll
  for (int o = kGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(L.mask, v, o, kGroup);
  return v;
}

// ballot of the group's lanes, bit s = lane s of the group
__device__ __forceinline__ unsigned group_ballot(const Lanes &L, bool pred) {
  const int shift = int(threadIdx.x & 31) & ~(kGroup - 1);
  return (__ballot_sync(L.mask, pred) & L.mask) >> shift;
}

template <typename real>
__device__ __forceinline__ int n_of(const PConsts<real> &pc, int a) {
  return a == 0 ? pc.n[0] : (a == 1 ? pc.n[1] : pc.n[2]);
}

// Stencil of a particle (lane a < 3 of the group holds the position component
// q_a): centre base and weights, own-axis face base and weights, broadcast to
// the group.
template <typename real>
__device__ void stencil_group(typename Pos<real>::T qa, const Lanes &L, const PConsts<real> &pc, int base[6],
                              real w[18]) {
  int bc = 0, bf = 0;
  real wc[3] = {real(0), real(0), real(0)}, wf[3] = {real(0), real(0), real(0)};
  if (L.sub < 3) {
    real rc, rf;
    Pos<real>::axis(qa, pc, L.sub, bc, rc, bf, rf);
    peskin3(rc, wc);
    peskin3(rf, wf);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    base[a] = gshfl(L, bc, a);
    base[3 + a] = gshfl(L, bf, a);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      w[3 * a + j] = gshfl(L, wc[j], a);
      w[9 + 3 * a + j] = gshfl(L, wf[j], a);
    }
  }
}

template <typename real>
__device__ __forceinline__ size_t cell_index(int x, int y, int z, const PConsts<real> &pc) {
  return size_t(IC_CHK(x, pc.n[0])) + size_t(pc.n[0]) * (size_t(IC_CHK(y, pc.n[1])) + size_t(pc.n[1]) * size_t(IC_CHK(z, pc.n[2])));
}

__device__ __forceinline__ int step_coord(int b, int d, int n) {
  int v = b + d;
  if (v < 0) v += n;
  if (v >= n) v -= n;
  return v;
}

template <typename real>
__device__ __forceinline__ real sel3(const real *w3, int d) {   // w3[d + 1], d in {-1, 0, 1}
  return d < 0 ? w3[0] : (d == 0 ? w3[1] : w3[2]);
}

// Group gather at one stencil: J delta rho (out[0]) and J v^a (out[1+a]).
// Point t (0..26) is (t % 3, (t / 3) % 3, t / 9) - 1 of each location set;
// lane s of the group takes the points s, s + kGroup, ...
template <typename real>
__device__ void gather(const Grid4<real> &G, const int base[6], const real w[18], const PConsts<real> &pc,
                       const Lanes &L, bool want_rho, bool want_v, real out[4]) {
  real acc[4] = {real(0), real(0), real(0), real(0)};
#pragma unroll
  for (int k = 0; k < kPointsPerLane; ++k) {
    const int t = L.sub + kGroup * k;
    if (t >= 27) break;
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    const int cx = step_coord(base[0], dx, pc.n[0]), cy = step_coord(base[1], dy, pc.n[1]),
              cz = step_coord(base[2], dz, pc.n[2]);
    const real wcx = sel3(w + 0, dx), wcy = sel3(w + 3, dy), wcz = sel3(w + 6, dz);
    if (want_rho) acc[0] += wcx * wcy * wcz * G.f[0][cell_index(cx, cy, cz, pc)];
    if (want_v) {
      const real rho0 = pc.rho0, half = real(0.5);
      {  // x faces
        const int fx = step_coord(base[3], dx, pc.n[0]);
        const int fxp = (fx + 1 == pc.n[0]) ? 0 : fx + 1;
        const size_t i = cell_index(fx, cy, cz, pc), iu = cell_index(fxp, cy, cz, pc);
        acc[1] += sel3(w + 9, dx) * wcy * wcz * fdiv(G.f[1][i], rho0 + half * (G.f[0][i] + G.f[0][iu]));
      }
      {  // y faces
        const int fy = step_coord(base[4], dy, pc.n[1]);
        const int fyp = (fy + 1 == pc.n[1]) ? 0 : fy + 1;
        const size_t i = cell_index(cx, fy, cz, pc), iu = cell_index(cx, fyp, cz, pc);
        acc[2] += wcx * sel3(w + 12, dy) * wcz * fdiv(G.f[2][i], rho0 + half * (G.f[0][i] + G.f[0][iu]));
      }
      {  // z faces
        const int fz = step_coord(base[5], dz, pc.n[2]);
        const int fzp = (fz + 1 == pc.n[2]) ? 0 : fz + 1;
        const size_t i = cell_index(cx, cy, fz, pc), iu = cell_index(cx, cy, fzp, pc);
        acc[3] += wcx * wcy * sel3(w + 15, dz) * fdiv(G.f[3][i], rho0 + half * (G.f[0][i] + G.f[0][iu]));
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) out[j] = group_sum(L, acc[j]);
}

template <typename real>
__device__ __forceinline__ void load_stencil(const PV<real> &P, int p, int base[6], real w[18]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) base[j] = P.base[6 * p + j];
#pragma unroll
  for (int j = 0; j < 18; ++j) w[j] = P.w[18 * p + j];
}

// signed offset b - a on a ring of n points, for |b - a| < n (no division)
__device__ __forceinline__ int ring_d(int b, int a, int n) {
  int d = b - a;
  if (2 * d > n) d -= n;
  if (2 * d < -n) d += n;
  return d;
}

// Visits p and the neighbours of p whose centre bases lie within `reach`
// cells of p's on every axis, in ascending particle index.  The neighbour
// list is screened a group-width at a time (one parallel load of indices and
// bases) so that far neighbours cost no dependent round trip.
template <typename real, typename Visit>
__device__ __forceinline__ void for_near_members(const PV<real> &P, int p, const int pb[3], int reach,
                                                 const PConsts<real> &pc, const Lanes &L, Visit visit) {
  const int nn = P.nnbr[p];
  const int *nb = P.nbr + size_t(p) * kMaxNeighbours;
  bool self_done = false;
  for (int j0 = 0; j0 < nn; j0 += kGroup) {
    const int j = j0 + L.sub;
    int m_l = 0;
    bool near = false;
    if (j < nn) {
      m_l = IC_CHK(nb[j], P.n);
      near = true;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int d = ring_d(P.base[6 * m_l + b], pb[b], pc.n[b]);
        near = near && d <= reach && d >= -reach;
      }
    }
    unsigned bits = group_ballot(L, near);
    while (bits) {
      const int k = __ffs(bits) - 1;
      bits &= bits - 1;
      const int m = gshfl(L, m_l, k);
      if (!self_done && m > p) {
        visit(p);
        self_done = true;
      }
      visit(m);
    }
  }
  if (!self_done) visit(p);
}

template <typename real>
__device__ __forceinline__ real w1(const real *w3, int d) {
  return (unsigned(d + 1) < 3u) ? w3[d + 1] : real(0);
}

template <typename real>
__device__ __forceinline__ real pick3(const real v[4], int a) {
  return a == 0 ? v[1] : (a == 1 ? v[2] : v[3]);
}

// Per-group staging of one member particle for the face updates.
template <typename real>
struct Member {
  int base[6];
  real w[18];
  real vec[3];
};

// Owner-computes update of the faces of particle p's three face stencils (for
// each axis a, the 3 x 3 x 3 a-faces around its a-face base): every such face
// is updated by exactly one particle, the lowest-index one whose face stencils
// hold it, which adds  scale * sum_m W_a(m, f) vec_m[a] / h^3  over the
// particles m whose stencils reach the face, in ascending particle index.
// vec is the tether force (stage source S F) or the impulse (-S dg).
constexpr int kFacesPerLane = (81 + kGroup - 1) / kGroup;

template <typename real>
__device__ void update_owned_faces(const PV<real> &P, const Grid4<real> &G, int p, const Lanes &L,
                                   const real *vec, real scale, const PConsts<real> &pc, Member<real> *sm) {
  int pb[6];
#pragma unroll
  for (int b = 0; b < 6; ++b) pb[b] = P.base[6 * p + b];

  // this lane's faces: t = sub + kGroup j < 81; axis a = t / 27, point (t % 27)
  auto axis_of = [&](int j) { const int t = L.sub + kGroup * j; return t < 81 ? t / 27 : 0; };
  int fA[kFacesPerLane], fB1[kFacesPerLane], fB2[kFacesPerLane];
  unsigned owner = 0;   // bit j: this lane still owns face j
  real total[kFacesPerLane];
#pragma unroll
  for (int j = 0; j < kFacesPerLane; ++j) {
    const int t = L.sub + kGroup * j;
    const int a = axis_of(j), r = t % 27;
    const int b1 = a == 2 ? 0 : a + 1, b2 = a == 0 ? 2 : a - 1;
    const int pa = a == 0 ? pb[3] : (a == 1 ? pb[4] : pb[5]);     // face base along a
    const int p1 = b1 == 0 ? pb[0] : (b1 == 1 ? pb[1] : pb[2]);
    const int p2 = b2 == 0 ? pb[0] : (b2 == 1 ? pb[1] : pb[2]);
    fA[j] = step_coord(pa, r % 3 - 1, n_of(pc, a));
    fB1[j] = step_coord(p1, (r / 3) % 3 - 1, n_of(pc, b1));
    fB2[j] = step_coord(p2, r / 9 - 1, n_of(pc, b2));
    if (t < 81) owner |= 1u << j;
    total[j] = real(0);
  }

  // face stencils of two particles can share a face only if their centre
  // bases are within 3 cells on every axis
  // p's own term on each of its faces: the face sits at offsets (r % 3, r / 3 % 3,
  // r / 9) - 1 of p's stencils, so it needs no offset test
  real self_term[kFacesPerLane];
  __syncwarp(L.mask);
  for (int i = L.sub; i < 18; i += kGroup) sm->w[i] = P.w[18 * p + i];
  if (L.sub < 3) sm->vec[L.sub] = vec[3 * p + L.sub];
  __syncwarp(L.mask);
#pragma unroll
  for (int j = 0; j < kFacesPerLane; ++j) {
    const int r = (L.sub + kGroup * j) % 27;
    const int a = axis_of(j), b1 = a == 2 ? 0 : a + 1, b2 = a == 0 ? 2 : a - 1;
    const real wt = sm->w[9 + 3 * a + r % 3] * sm->w[3 * b1 + (r / 3) % 3] * sm->w[3 * b2 + r / 9];
    self_term[j] = wt * sm->vec[a];
  }

  for_near_members(P, p, pb, 3, pc, L, [&](int m) {
    if (m == p) {
#pragma unroll
      for (int j = 0; j < kFacesPerLane; ++j) total[j] += self_term[j] * pc.inv_h3;
      return;
    }
    __syncwarp(L.mask);
    if (L.sub < 6) sm->base[L.sub] = P.base[6 * m + L.sub];
    for (int i = L.sub; i < 18; i += kGroup) sm->w[i] = P.w[18 * m + i];
    if (L.sub < 3) sm->vec[L.sub] = vec[3 * m + L.sub];
    __syncwarp(L.mask);
    const bool lower = m < p;
#pragma unroll
    for (int j = 0; j < kFacesPerLane; ++j) {
      const int a = axis_of(j), b1 = a == 2 ? 0 : a + 1, b2 = a == 0 ? 2 : a - 1;
      const int df = ring_d(fA[j], sm->base[3 + a], n_of(pc, a));
      const int d1 = ring_d(fB1[j], sm->base[b1], n_of(pc, b1));
      const int d2 = ring_d(fB2[j], sm->base[b2], n_of(pc, b2));
      const bool inside = df >= -1 && df <= 1 && d1 >= -1 && d1 <= 1 && d2 >= -1 && d2 <= 1;
      if (lower && inside) owner &= ~(1u << j);
      const real wt = w1(sm->w + 9 + 3 * a, df) * w1(sm->w + 3 * b1, d1) * w1(sm->w + 3 * b2, d2);
      total[j] += wt * sm->vec[a] * pc.inv_h3;
    }
  });
#pragma unroll
  for (int j = 0; j < kFacesPerLane; ++j) {
    if (owner & (1u << j)) {
      const int a = axis_of(j);
      const int x = a == 0 ? fA[j] : (a == 1 ? fB2[j] : fB1[j]);
      const int y = a == 1 ? fA[j] : (a == 2 ? fB2[j] : fB1[j]);
      const int z = a == 2 ? fA[j] : (a == 0 ? fB2[j] : fB1[j]);
      real *ga = a == 0 ? G.f[1] : (a == 1 ? G.f[2] : G.f[3]);
      ga[cell_index(x, y, z, pc)] += scale * total[j];
    }
  }
}

// ------------------------------------------------------------------ kernels
// bin coordinate of particle p along axis a (slabs of whole cells)
template <typename real>
__device__ __forceinline__ int bin_axis(typename Pos<real>::T q, const PConsts<real> &pc, int a) {
  return Pos<real>::cell(q, pc, a) * pc.nb[a] / n_of(pc, a);
}

// bin of particle p; its position read from L2 (the last CTA of k_final bins
// positions that other CTAs of the same launch wrote)
template <typename real>
__device__ __forceinline__ int bin_of(const PV<real> &P, int p, const PConsts<real> &pc) {
  const int bx = bin_axis<real>(__ldcg(P.q + 3 * p), pc, 0), by = bin_axis<real>(__ldcg(P.q + 3 * p + 1), pc, 1),
            bz = bin_axis<real>(__ldcg(P.q + 3 * p + 2), pc, 2);
  return IC_CHK(bx + pc.nb[0] * (by + pc.nb[1] * bz), pc.nbins);
}

// Counting sort of the particles into the neighbour bins by the threads of
// one CTA (blockDim.x a multiple of 32): counts, exclusive prefix sums into
// bins[0..nbins], then each particle takes a slot of its bin through a
// cursor.  The order within a bin is that of the atomics; the lists built
// from it are sorted by index.  Counts and cursors live in L2 (atomics; read
// back with __ldcg).
template <typename real>
__device__ void bin_particles(const PV<real> &P, const PConsts<real> &pc, long long *rebuilds) {
  __shared__ int warp_off[32];
  const int t = threadIdx.x, nt = blockDim.x, nb = pc.nbins;
  int *start = P.bins, *cur = P.bins + nb + 1;
  for (int b = t; b < nb; b += nt) cur[b] = 0;
  __syncthreads();
  for (int p = t; p < P.n; p += nt) atomicAdd(cur + bin_of(P, p, pc), 1);
  __syncthreads();
  // thread t scans the contiguous chunk [b0, b1) of the bins
  const int chunk = (nb + nt - 1) / nt;
  const int b0 = min(nb, t * chunk), b1 = min(nb, b0 + chunk);
  int own = 0;
  for (int b = b0; b < b1; ++b) own += __ldcg(cur + b);
  int incl = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if ((t & 31) >= o) incl += v;
  }
  if ((t & 31) == 31) warp_off[t >> 5] = incl;
  __syncthreads();
  if (t < 32) {
    const int w = t < nt / 32 ? warp_off[t] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, wi, o);
      if (t >= o) wi += v;
    }
    if (t < nt / 32) warp_off[t] = wi - w;
  }
  __syncthreads();
  int run = warp_off[t >> 5] + incl - own;
  for (int b = b0; b < b1; ++b) {
    const int c = __ldcg(cur + b);
    start[b] = run;
    cur[b] = run;
    run += c;
  }
  if (t == 0) start[nb] = P.n;
  __syncthreads();
  for (int p = t; p < P.n; p += nt) P.order[IC_CHK(atomicAdd(cur + bin_of(P, p, pc), 1), P.n)] = p;
  if (t == 0) ++*rebuilds;
}

// The sort when the host has flagged a rebuild (particles added, a state
// restored); in a step the last CTA of k_final does it.
constexpr int kBinThreads = 1024;

template <typename real>
__global__ void __launch_bounds__(kBinThreads) k_bin(PV<real> P, PConsts<real> pc, const int *rebuild,
                                                     long long *rebuilds) {
  if (*rebuild == 0) return;
  bin_particles(P, pc, rebuilds);
}

template <typename real>
__global__ void __launch_bounds__(kBlockThreads, min_blocks<real>()) k_half_step(PV<real> P, Grid4<real> G, PConsts<real> pc,
                                                             int *rebuild, int *status) {
  pdl_enter();
  using PosT = Pos<real>;
  using T = typename PosT::T;
  const int p = group_particle();
  const Lanes L = group_lanes();
  if (p >= P.n) return;

  if (*rebuild) {
    // neighbour list from q^n: the hits among the members of the 27 bins
    // around p's (fewer where an axis has fewer than 3 bins), then sorted by
    // index (all distinct: a rank each)
    __shared__ int found[kGroupsPerBlock][kMaxNeighbours];
    __shared__ int nfound[kGroupsPerBlock];
    const int g = threadIdx.x / kGroup;
    const T q0 = P.q[3 * p], q1 = P.q[3 * p + 1], q2 = P.q[3 * p + 2];
    const int cb[3] = {bin_axis(q0, pc, 0), bin_axis(q1, pc, 1), bin_axis(q2, pc, 2)};
    if (L.sub == 0) nfound[g] = 0;
    __syncwarp(L.mask);
    for (int o = L.sub; o < 27; o += kGroup) {
      const int d[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
      bool repeat = false;
      int b = 0;
#pragma unroll
      for (int a = 2; a >= 0; --a) {
        repeat = repeat || (pc.nb[a] == 1 && d[a] != 0) || (pc.nb[a] == 2 && d[a] < 0);
        b = b * pc.nb[a] + wrap(cb[a] + d[a], pc.nb[a]);
      }
      if (repeat) continue;
      const int i1 = P.bins[IC_CHK(b, pc.nbins) + 1];
      for (int i = P.bins[b]; i < i1; ++i) {
        const int j = IC_CHK(P.order[IC_CHK(i, P.n)], P.n);
        if (j == p) continue;
        if (fabs(PosT::diff(P.q[3 * j], q0, pc, 0)) < pc.cutoff &&
            fabs(PosT::diff(P.q[3 * j + 1], q1, pc, 1)) < pc.cutoff &&
            fabs(PosT::diff(P.q[3 * j + 2], q2, pc, 2)) < pc.cutoff) {
          const int slot = atomicAdd(&nfound[g], 1);
          if (slot < kMaxNeighbours) found[g][slot] = j;
        }
      }
    }
    __syncwarp(L.mask);
    const int total = nfound[g], count = min(total, kMaxNeighbours);
    for (int e = L.sub; e < count; e += kGroup) {
      const int v = found[g][e];
      int rank = 0;
      for (int k = 0; k < count; ++k) rank += found[g][k] < v ? 1 : 0;
      P.nbr[size_t(p) * kMaxNeighbours + rank] = v;
    }
    if (L.sub == 0) {
      if (total > kMaxNeighbours) atomicOr(status, kStatusNbrOverflow);
      P.nnbr[p] = count;
    }
    if (L.sub < 3) P.q_build[3 * p + L.sub] = P.q[3 * p + L.sub];
  }

  // substep 1: q^{n+1/2} = q^n + dt/2 J^n v^n (lane a < 3 owns axis a)
  const T q_l = L.sub < 3 ? P.q[3 * p + L.sub] : T(0);
  int base[6];
  real w[18];
  stencil_group<real>(q_l, L, pc, base, w);
  real g4[4];
  gather(G, base, w, pc, L, false, true, g4);
  T qh_l = T(0);
  real F_l = real(0);
  if (L.sub < 3) {
    qh_l = PosT::advance(q_l, real(0.5) * pc.dt * pick3(g4, L.sub), pc, L.sub);
    // substep 2: tether force at q^{n+1/2}
    F_l = -P.k_s[p] * real(PosT::diff(qh_l, P.q_eq[3 * p + L.sub], pc, L.sub));
  }

  // stencil at q^{n+1/2}; J^{n+1/2} v^n
  stencil_group<real>(qh_l, L, pc, base, w);
  gather(G, base, w, pc, L, false, true, g4);
  if (L.sub < 3) {
    P.q_half[3 * p + L.sub] = qh_l;
    P.force[3 * p + L.sub] = F_l;
    P.jv_n[3 * p + L.sub] = pick3(g4, L.sub);
    if (fabs(PosT::diff(qh_l, P.q_build[3 * p + L.sub], pc, L.sub)) > pc.skin_limit) atomicOr(status, kStatusSkin);
  }
  if (L.sub == 0) {
#pragma unroll
    for (int j = 0; j < 6; ++j) P.base[6 * p + j] = base[j];
#pragma unroll
    for (int j = 0; j < 18; ++j) P.w[18 * p + j] = w[j];
  }
}

// Particle pressure of one RK stage (Eqs. (eq:pressure), (omega)): writes
// PP(c) = sum_m W_c(m, c) Omega_m / h^3, Omega_m = eps_m V J_m(rho_s - rho0),
// on the 27 centre cells of particle p, for the cells p owns (no lower-index
// particle's centre stencil holds them).  The Omega of the particles whose
// stencils reach p's cells are regathered here, so one launch suffices.
template <typename real>
__global__ void __launch_bounds__(kBlockThreads, min_blocks<real>()) k_pressure(PV<real> P, Grid4<real> G, PConsts<real> pc, real *pp,
                                                            int *rebuild) {
  pdl_enter();
  const int p = group_particle();
  const Lanes L = group_lanes();
  // the neighbour lists were rebuilt (if flagged) by the half step: clear the flag
  if (rebuild && blockIdx.x == 0 && threadIdx.x == 0) *rebuild = 0;
  if (p >= P.n) return;
  int pb[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) pb[b] = P.base[6 * p + b];
  // this lane's cells of p's centre stencil: t = sub + kGroup k < 27
  int cx[kPointsPerLane], cy[kPointsPerLane], cz[kPointsPerLane];
  bool owner[kPointsPerLane];
  real total[kPointsPerLane];
#pragma unroll
  for (int k = 0; k < kPointsPerLane; ++k) {
    const int t = L.sub + kGroup * k;
    cx[k] = step_coord(pb[0], t % 3 - 1, pc.n[0]);
    cy[k] = step_coord(pb[1], (t / 3) % 3 - 1, pc.n[1]);
    cz[k] = step_coord(pb[2], (t / 9) % 3 - 1, pc.n[2]);
    owner[k] = t < 27;
    total[k] = real(0);
  }
  // centre stencils of two particles share a cell only within 2 cells on every axis
  for_near_members(P, p, pb, 2, pc, L, [&](int m) {
    int mb[6];
    real mw[18];
    load_stencil(P, m, mb, mw);
    real g4[4];
    gather(G, mb, mw, pc, L, true, false, g4);
    const real omega = P.eps[m] * pc.vol * g4[0];
#pragma unroll
    for (int k = 0; k < kPointsPerLane; ++k) {
      const int ex = ring_d(cx[k], mb[0], pc.n[0]), ey = ring_d(cy[k], mb[1], pc.n[1]),
                ez = ring_d(cz[k], mb[2], pc.n[2]);
      const bool inside = ex >= -1 && ex <= 1 && ey >= -1 && ey <= 1 && ez >= -1 && ez <= 1;
      if (m < p && inside) owner[k] = false;
      if (inside) total[k] += sel3(mw + 0, ex) * sel3(mw + 3, ey) * sel3(mw + 6, ez) * omega;
    }
  });
#pragma unroll
  for (int k = 0; k < kPointsPerLane; ++k)
    if (owner[k]) pp[cell_index(cx[k], cy[k], cz[k], pc)] = total[k] * pc.inv_h3;
}

// Spring-force source of RK stage s (b_s dt S F) or the impulse (-S dg).
template <typename real, int KIND>
__global__ void __launch_bounds__(kBlockThreads, min_blocks<real>()) k_face_update(PV<real> P, Grid4<real> G, PConsts<real> pc,
                                                               real scale) {
  pdl_enter();
  __shared__ Member<real> sm[kGroupsPerBlock];
  const int p = group_particle();
  const Lanes L = group_lanes();
  if (p >= P.n) return;
  update_owned_faces<real>(P, G, p, L, KIND == 0 ? P.force : P.dg, scale, pc, &sm[threadIdx.x / kGroup]);
}

template <typename real>
__global__ void __launch_bounds__(kBlockThreads, min_blocks<real>()) k_impulse(PV<real> P, Grid4<real> G, PConsts<real> pc) {
  pdl_enter();
  const int p = group_particle();
  const Lanes L = group_lanes();
  if (p >= P.n) return;
  int base[6];
  real w[18];
  load_stencil(P, p, base, w);
  real g4[4];
  gather(G, base, w, pc, L, true, true, g4);
  if (L.sub < 3) {
    const real mf = pc.vol * (pc.rho0 + g4[0]);   // m_f = V J rho^{n+1}
    const real me = P.m_e[p];
    const real u = P.u[3 * p + L.sub];
    const real rel = pick3(g4, L.sub) - u;
    const real dg = me * mf / (me + mf) * rel;
    P.dg[3 * p + L.sub] = dg;
    P.u[3 * p + L.sub] = u + mf / (me + mf) * rel;
    P.lam[3 * p + L.sub] = dg / pc.dt - P.force[3 * p + L.sub];
    if (L.sub == 0) P.jrho[p] = pc.rho0 + g4[0];
  }
}

template <typename real>
__device__ void final_particle(const PV<real> &P, const Grid4<real> &G, const PConsts<real> &pc, const int64_t *step,
                               const double *weights, int *rebuild, real *pp, int p, const Lanes &L);

// Substep 7 for every particle; the CTA that finishes last then sorts the
// particles into the neighbour bins if any of them asked for a rebuild, and
// does the step's end-of-step bookkeeping (after every CTA has read the step
// counter it advances).
template <typename real>
__global__ void __launch_bounds__(kBlockThreads, min_blocks<real>()) k_final(PV<real> P, Grid4<real> G, PConsts<real> pc,
                                                         const double *weights, int *rebuild, real *pp, int *done,
                                                         long long *rebuilds, const EndArgs e) {
  pdl_enter();
  const int p = group_particle();
  const Lanes L = group_lanes();
  if (p < P.n) final_particle(P, G, pc, e.step, weights, rebuild, pp, p, L);
  __shared__ int last;
  __shared__ double red[kBlockThreads];
  __threadfence();   // this thread's q^{n+1} and rebuild flag, before the CTA counts itself done
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done, 1) == int(gridDim.x) - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (*reinterpret_cast<volatile int *>(rebuild)) bin_particles(P, pc, rebuilds);
  end_of_step_cta(e, red);
  if (threadIdx.x == 0) {
    // the step's status word beside lambda, so that one copy reads both back
    *reinterpret_cast<int *>(P.lam + 3 * size_t(P.n)) = *reinterpret_cast<volatile int *>(e.status);
    *done = 0;
  }
}

template <typename real>
__device__ void final_particle(const PV<real> &P, const Grid4<real> &G, const PConsts<real> &pc, const int64_t *step,
                               const double *weights, int *rebuild, real *pp, int p, const Lanes &L) {
  using PosT = Pos<real>;
  int base[6];
  real w[18];
  load_stencil(P, p, base, w);
  real g4[4];
  gather(G, base, w, pc, L, false, true, g4);
  // the particle pressure of this step is consumed: clear p's 27 cells
#pragma unroll
  for (int k = 0; k < kPointsPerLane; ++k) {
    const int t = L.sub + kGroup * k;
    if (t < 27)
      pp[cell_index(step_coord(base[0], t % 3 - 1, pc.n[0]), step_coord(base[1], (t / 3) % 3 - 1, pc.n[1]),
                    step_coord(base[2], t / 9 - 1, pc.n[2]), pc)] = real(0);
  }
  bool move = false;
  if (L.sub < 3) {
    const typename PosT::T qn = PosT::advance(
        P.q[3 * p + L.sub], real(0.5) * pc.dt * (pick3(g4, L.sub) + P.jv_n[3 * p + L.sub]), pc, L.sub);
    P.q[3 * p + L.sub] = qn;
    move = fabs(PosT::diff(qn, P.q_build[3 * p + L.sub], pc, L.sub)) > pc.rebuild_at;
  }
  if (__any_sync(L.mask, move) && L.sub == 0) *rebuild = 1;
  // weighted sums in FP64, one value per lane: lanes 0-2 the tether force, 3-5 lambda
  if (L.sub < 6) {
    const int64_t jw = step[0] - step[1];
    const double wt = (jw >= 0 && jw < step[2]) ? weights[jw] : 0.0;
    const real v = L.sub < 3 ? P.force[3 * p + L.sub] : P.lam[3 * p + L.sub - 3];
    P.acc[6 * p + L.sub] += wt * double(v);
  }
}

template <typename real>
__global__ void __launch_bounds__(kBlockThreads, min_blocks<real>()) k_init_velocity(PV<real> P, Grid4<real> G, PConsts<real> pc,
                                                                 int first, int n) {
  using T = typename Pos<real>::T;
  const int p = first + group_particle();
  const Lanes L = group_lanes();
  if (p >= first + n) return;
  const T q_l = L.sub < 3 ? P.q[3 * p + L.sub] : T(0);
  int base[6];
  real w[18];
  stencil_group<real>(q_l, L, pc, base, w);
  real g4[4];
  gather(G, base, w, pc, L, false, true, g4);
  if (L.sub < 3) P.u[3 * p + L.sub] = pick3(g4, L.sub);
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

template <typename real>
cudaError_t launch_particles_t(ic_ctx *ctx, ParticlePhase phase, int stage, void *const cur[4],
                               void *const tgt[4]) {
  const PV<real> P = view<real>(ctx->ps);
  if (P.n == 0) return cudaSuccess;
  const PConsts<real> pc = particle_consts<real>(ctx);
  const dim3 grid((P.n + kGroupsPerBlock - 1) / kGroupsPerBlock), block(kBlockThreads);
  static const double kCoef[3] = {1.0, 0.25, 2.0 / 3.0};
  real *pp = static_cast<real *>(ctx->pp);
  switch (phase) {
    case kHalfStep:
      return launch_k(k_half_step<real>, grid, block, 0, ctx->stream, P, grid4<real>(cur), pc, ctx->d.rebuild,
                      ctx->d.status);
    case kPressure:
      return launch_k(k_pressure<real>, grid, block, 0, ctx->stream, P, grid4<real>(tgt), pc, pp,
                      stage == 0 ? ctx->d.rebuild : nullptr);
    case kForce:
      return launch_k(k_face_update<real, 0>, grid, block, 0, ctx->stream, P, grid4<real>(tgt), pc,
                      real(kCoef[stage] * ctx->p.dt));
    case kImpulse:
      return launch_k(k_impulse<real>, grid, block, 0, ctx->stream, P, grid4<real>(tgt), pc);
    case kSpread:
      return launch_k(k_face_update<real, 1>, grid, block, 0, ctx->stream, P, grid4<real>(tgt), pc, real(-1));
    case kFinal:
      return launch_k(k_final<real>, grid, block, 0, ctx->stream, P, grid4<real>(tgt), pc, ctx->d.weights,
                      ctx->d.rebuild, pp, ctx->d.bin_done, ctx->d.rebuilds, end_args(ctx));
  }
  return cudaGetLastError();
}

}  // namespace

int neighbour_bins(const ic_grid_params &p, int nb[3]) {
  const int width = int(std::floor(4.0 + kSkin)) + 1;   // cells: the cutoff is (4 + skin) h
  const int n[3] = {p.nx, p.ny, p.nz};
  for (int a = 0; a < 3; ++a) nb[a] = std::max(1, n[a] / width);
  return nb[0] * nb[1] * nb[2];
}

cudaError_t launch_particles(ic_ctx *ctx, ParticlePhase phase, int stage, void *const cur[4],
                             void *const tgt[4]) {
  if (ctx->p.precision == IC_FP32) return launch_particles_t<float>(ctx, phase, stage, cur, tgt);
  return launch_particles_t<double>(ctx, phase, stage, cur, tgt);
}

cudaError_t launch_particle_bins(ic_ctx *ctx) {
  if (ctx->ps.n == 0) return cudaSuccess;
  if (ctx->p.precision == IC_FP32)
    k_bin<float><<<1, kBinThreads, 0, ctx->stream>>>(view<float>(ctx->ps), particle_consts<float>(ctx),
                                                     ctx->d.rebuild, ctx->d.rebuilds);
  else
    k_bin<double><<<1, kBinThreads, 0, ctx->stream>>>(view<double>(ctx->ps), particle_consts<double>(ctx),
                                                      ctx->d.rebuild, ctx->d.rebuilds);
  return cudaGetLastError();
}

cudaError_t launch_particle_velocity(ic_ctx *ctx, int first, int n, void *const state[4]) {
  const dim3 grid((n + kGroupsPerBlock - 1) / kGroupsPerBlock), block(kBlockThreads);
  if (ctx->p.precision == IC_FP32)
    k_init_velocity<float><<<grid, block, 0, ctx->stream>>>(view<float>(ctx->ps), grid4<float>(state),
                                                            particle_consts<float>(ctx), first, n);
  else
    k_init_velocity<double><<<grid, block, 0, ctx->stream>>>(view<double>(ctx->ps), grid4<double>(state),
                                                             particle_consts<double>(ctx), first, n);
  return cudaGetLastError();
}

cudaError_t launch_particle_momentum(ic_ctx *ctx, double *dev_out3) {
  if (ctx->p.precision == IC_FP32)
    k_particle_momentum<float><<<1, 256, 0, ctx->stream>>>(view<float>(ctx->ps), dev_out3);
  else
    k_particle_momentum<double><<<1, 256, 0, ctx->stream>>>(view<double>(ctx->ps), dev_out3);
  return cudaGetLastError();
}

// Host conversions of positions to and from the device representation.
void positions_to_device(const ic_ctx *ctx, const double *q, size_t n3, void *out) {
  const ic_grid_params &p = ctx->p;
  const int n[3] = {p.nx, p.ny, p.nz};
  if (p.precision == IC_FP32) {
    long long *o = static_cast<long long *>(out);
    for (size_t i = 0; i < n3; ++i) {
      const long long span = (long long)n[i % 3] << kFixBits;
      long long v = std::llround(q[i] / p.h * 0x1p40);
      v %= span;
      if (v < 0) v += span;
      o[i] = v;
    }
  } else {
    std::memcpy(out, q, n3 * sizeof(double));
  }
}

void positions_to_host(const ic_ctx *ctx, const void *in, size_t n3, double *q) {
  const ic_grid_params &p = ctx->p;
  if (p.precision == IC_FP32) {
    const long long *v = static_cast<const long long *>(in);
    for (size_t i = 0; i < n3; ++i) q[i] = double(v[i]) * 0x1p-40 * p.h;
  } else {
    std::memcpy(q, in, n3 * sizeof(double));
  }
}

IC_BOUNDS_READER(bounds_flag_particles)

}  // namespace ic
