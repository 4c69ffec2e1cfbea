// FP32 SSP-RK3 stage kernel over whole x rows (Sec. 4.2, App. A.2).
//
// The same stage as k_rk3_stage / k_rk3_stage_z2 in ic_fluid.cu (the
// conservative staggered fluxes, their divergence and the RK combination, as
// the same sequence of rounded operations per cell), laid out for the GB300
// memory system:
//
//  * A CTA owns TY whole x rows of the box (plus one ring row below and above)
//    and marches a run of z planes.  The x direction is periodic inside the
//    CTA, so no x halo is loaded or computed.
//  * Every thread owns four x-adjacent cells of one row (one 16-byte vector
//    per field); x neighbours inside the quad are registers, the quad's edge
//    neighbours and the y neighbours come from shared memory.
//  * The inputs of each z plane arrive as contiguous multi-row spans copied by
//    1D bulk (TMA) copies into rings of shared-memory slots, one mbarrier per
//    slot, issued by one thread two planes ahead; the density ring runs one
//    plane ahead of the momentum ring, as the face densities need it.  U^n and
//    the stored noise of stages 2-3 come through a third ring.  Every wait is
//    bounded (about a second; then a status bit and IC_ERR_TIMEOUT).
//  * Per plane: (A) face velocities and pressure of the plane above, (B) the
//    nine scaled momentum fluxes, (C) their divergence, the noise, the RK
//    combination and the vector stores; two CTA barriers.
//  * Noise (kT > 0).  The stochastic stress enters a stage only through its
//    divergence, which is linear in the normals: D_s = D(W_A) + beta_s D(W_B).
//    Stage 1 draws W_A, W_B per cell (Philox4x32-10, the FP32 normals of
//    ic_device.cuh), exchanges the in-plane stress components of both streams
//    through shared memory, uses D_1 and stores D_2 and D_3 (3 words each);
//    stages 2 and 3 read theirs (3 words).  That is 48 B per cell-step instead
//    of the 96 B of storing W_2 and W_3.
//
// Requirements: FP32, nx a multiple of 4 and at most 128 (a quad per thread,
// 16-byte aligned rows), 16-byte aligned fields.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "ic_async.cuh"
#include "ic_device.cuh"
#include "ic_internal.hpp"

namespace ic {

namespace {

constexpr int kRowsMaxNx = 128;
constexpr int kRowsVC = 4;    // x-adjacent cells per thread (one 16-byte vector per field)
constexpr int kRowsNSD = 3;   // density ring
constexpr int kRowsNSN = 2;   // U^n and stored-noise ring (stages 2-3)
constexpr int kRowsMaxBars = kRowsNSD + 4 + kRowsNSN;
constexpr size_t kRowsSmemCap = 227 * 1024 - 3072;   // dynamic shared memory a CTA may take (static: up to 2.6 KB)
constexpr double kStageAR[3] = {0.0, 0.75, 1.0 / 3.0};
constexpr double kStageBR[3] = {1.0, 0.25, 2.0 / 3.0};

__host__ __device__ constexpr int rows_nsg(int stage) { return stage == 0 ? 3 : 4; }   // momentum ring
// fields of the U^n ring: U^n (stages 2-3) and the stage's stored noise divergence
__host__ __device__ constexpr int rows_nun(int stage) { return stage == 0 ? 0 : 4; }
__host__ __device__ constexpr int rows_nfn(int stage, bool noise) { return rows_nun(stage) + (noise ? 3 : 0); }

// Shared-memory regions of one CTA, in floats (all multiples of 4).
struct RowLayout {
  int d, g, v, t, tb, s, n, total;
};

__host__ __device__ inline RowLayout row_layout(int nx, int vc, int R, int RD, int ty, int stage, bool noise) {
  RowLayout L;
  const int plane = R * nx;
  L.d = 0;                                                // [NSD][RD][nx] delta rho
  L.g = L.d + kRowsNSD * RD * nx;                         // [NSG][4][R][nx] gx, gy, gz, S Omega
  L.v = L.g + rows_nsg(stage) * 4 * plane;                // [2][3][R][nx] vx, vy, vz by plane parity
  L.t = L.v + 6 * plane;                                  // [3][R][nx] T_yy, T_xy, T_zy
  L.tb = L.t + 3 * plane;                                 // [3][R][nx/vc] edge-cell T_xx, T_yx, T_zx
  L.s = L.tb + ((3 * R * (nx / vc) + 3) & ~3);
  L.n = L.s;                                              // [NSN][nfn][ty][nx] U^n (stages 2-3), D_s
  L.total = L.n + kRowsNSN * rows_nfn(stage, noise) * ty * nx;
  return L;
}

struct RowArgs {
  const float *__restrict__ s[4];     // U_s
  const float *__restrict__ n[4];     // U^n
  float *__restrict__ o[4];           // U_{s+1}
  const float *__restrict__ pp;       // particle pressure S Omega_s at centres, or null
  const float *__restrict__ d_in[3];  // kT > 0: the stage's stress divergence D_s (x, y, z faces)
  FluidConsts<float> c;
  const int64_t *step;
  double *partials;                   // stage 3: per-CTA sum of delta rho cos(k x)
  int *status;
  int ty;      // own rows per tile
  int nrow;    // thread rows: ty + 2 (ring rows), or ny when one tile holds every row
  int wrapy;   // 1: one tile holds every row (y periodic inside the CTA, no ring rows)
  int ncols;   // tiles along y
  int stall;   // 1 only to test the bounded waits: every mbarrier expects an arrival nothing makes
};

// the VC x-adjacent cells of one thread: one 8- or 16-byte vector per field
template <int VC>
struct Cells {
  float v[VC];
};

template <int VC>
__device__ __forceinline__ Cells<VC> ldc(const float *p) {
  if constexpr (VC == 4) {
    const float4 f = *reinterpret_cast<const float4 *>(p);
    return Cells<VC>{{f.x, f.y, f.z, f.w}};
  } else {
    const float2 f = *reinterpret_cast<const float2 *>(p);
    return Cells<VC>{{f.x, f.y}};
  }
}
template <int VC>
__device__ __forceinline__ void stc(float *p, const float v[VC]) {
  if constexpr (VC == 4)
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}

// the finished values of one plane at the thread's cells
template <int VC>
struct PlaneQ {
  float dr[VC], gx[VC], gy[VC], gz[VC], vx[VC], vy[VC], vz[VC], pk[VC];   // pk = 4 pi
};

// compute threads of a CTA at most (the ring-slot copies take one more warp)
template <int VC>
__host__ __device__ constexpr int rows_max_threads() { return 80 * VC; }

// Barriers among the compute threads: with a copy warp (PROD) a named barrier
// over the first T threads, else the CTA barrier.
template <bool PROD>
__device__ __forceinline__ void cbar(int T) {
  if constexpr (PROD)
    asm volatile("bar.sync 1, %0;\n" ::"r"(T) : "memory");
  else
    __syncthreads();
}
template <bool PROD>
__device__ __forceinline__ bool cbar_or(int T, bool pred) {
  if constexpr (PROD) {
    uint32_t out;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, 1, %2, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(out)
        : "r"(uint32_t(pred)), "r"(T)
        : "memory");
    return out != 0;
  } else {
    return __syncthreads_or(pred) != 0;
  }
}

template <int VC, int STAGE, bool NOISE, bool PROD>
__global__ void __launch_bounds__(rows_max_threads<VC>() + 32, 1) k_stage_rows(const RowArgs a) {
  pdl_enter();
  constexpr int NSD = kRowsNSD, NSG = rows_nsg(STAGE), NSN = kRowsNSN;
  constexpr int NUN = rows_nun(STAGE), NFN = rows_nfn(STAGE, NOISE);
  extern __shared__ __align__(16) float sm[];
  __shared__ __align__(8) unsigned long long bars[kRowsMaxBars + 1];   // + the copy warp's go signal
  __shared__ float s_acc[rows_max_threads<VC>()];
  const FluidConsts<float> &c = a.c;
  const int NX = c.nx, NY = c.ny, NZ = c.nz, QX = NX / VC;
  const int R = a.nrow, TY = a.ty, wrapy = a.wrapy;
  const int RD = wrapy ? R : R + 1;
  const RowLayout L = row_layout(NX, VC, R, RD, TY, STAGE, NOISE);
  const int plane = R * NX;
  const int t = threadIdx.x;
  const int T = QX * R;                      // compute threads; with PROD, warp T / 32 issues the copies
  const bool copier = PROD && t >= T;
  const int r = copier ? 0 : t / QX, q = copier ? 0 : t - r * QX;
  const int xq = VC * q;
  const int em = (q == 0 ? NX : xq) - 1;     // element left of the thread's cells (periodic)
  const int ep = q == QX - 1 ? 0 : xq + VC;  // element right of the thread's cells
  const int qm = q == 0 ? QX - 1 : q - 1, qp = q == QX - 1 ? 0 : q + 1;
  const int rm = wrapy ? (r == 0 ? R - 1 : r - 1) : max(r - 1, 0);
  const int rp = wrapy ? (r == R - 1 ? 0 : r + 1) : min(r + 1, R - 1);
  const int rpd = wrapy ? rp : r + 1;        // density row one y up
  const int ur = wrapy ? r : r - 1;          // row of the U^n ring
  float *sd = sm + L.d, *sg = sm + L.g, *sv = sm + L.v, *st = sm + L.t, *stb = sm + L.tb, *sn = sm + L.n;
  const int RQ = R * QX;
  const auto zw = [NZ](int p) { return p < 0 ? p + NZ : (p >= NZ ? p - NZ : p); };

  const float drive4 = 4.0f * c.drive[STAGE];
  const float rho0 = c.rho0, c2x4 = c.c2x4, visc_d = c.visc_d, visc_o = c.visc_o, lam2x4_h = c.lam2x4_h;
  const float out_flux = c.out_flux, out_mass = c.out_mass;
  const float ca = float(kStageAR[STAGE]), cb = float(kStageBR[STAGE]);
  float cosx[VC];
#pragma unroll
  for (int e = 0; e < VC; ++e) cosx[e] = (c.wave_axis == 0 && c.cos_table) ? c.cos_table[xq + e] : 0.0f;
  float mode_acc = 0.0f;

  if (t == 0) {
    for (int i = 0; i < kRowsMaxBars; ++i) mbar_init(smem_u32(&bars[i]), uint32_t(1 + a.stall));
    mbar_init(smem_u32(&bars[kRowsMaxBars]), 1u);
  }
  __syncthreads();
  // the lanes that issue copies: the copy warp (PROD), else warp 0
  const int lane0 = PROD ? T : 0;
  const int wlanes = PROD ? 32 : min(32, int(blockDim.x));
  const unsigned wmask = wlanes == 32 ? 0xffffffffu : ((1u << wlanes) - 1u);
  const bool issuer = PROD ? copier : t < 32;
  const uint32_t go_bar = smem_u32(&bars[kRowsMaxBars]);
  uint32_t go_ph = 0;                    // copy warp: parity of the next go signal
  uint32_t pfill = 0, pph = 0;           // copy warp: slots filled so far, parity of each slot's last fill
  uint32_t ph = 0;   // bit i: parity of the next completion of barrier i
  bool bad = false;
  const auto wait_bar = [&](int i) {
    if (!mbar_wait(smem_u32(&bars[i]), (ph >> i) & 1u)) bad = true;
    ph ^= 1u << i;
  };

  const int units = a.ncols * NZ;
  const int u_end = int((long long)units * (blockIdx.x + 1) / gridDim.x);
  for (int u = int((long long)units * blockIdx.x / gridDim.x); u < u_end;) {
    const int col = u / NZ;
    const int z0 = u - col * NZ;
    const int z1 = min(NZ, z0 + (u_end - u));
    u += z1 - z0;
    const int y0 = wrapy ? 0 : col * TY;
    const int ystart = wrapy ? 0 : y0 - 1;   // global row of thread row 0
    const int y = wrap(ystart + r, NY);
    const bool own = wrapy ? true : (r >= 1 && r <= TY && y0 - 1 + r < NY);
    const int pbase = z0 - 1;
    const float cosy = (c.wave_axis == 1 && c.cos_table) ? c.cos_table[y] : 0.0f;
    const auto profile = [&](int p, int e) -> float {
      if (c.forcing == IC_FORCE_MODE) return c.wave_axis == 0 ? cosx[e] : (c.wave_axis == 1 ? cosy : c.cos_table[zw(p)]);
      if (c.forcing == IC_FORCE_PLANE) {
        const int coord = c.wave_axis == 0 ? xq + e : (c.wave_axis == 1 ? y : zw(p));
        return coord == c.plane_index ? 1.0f : 0.0f;
      }
      return 0.0f;
    };

    int next_d = pbase, next_g = pbase, next_n = z0;   // next plane to copy, per ring
    int wd = pbase, wg = pbase, wn = z0;               // next plane to wait for, per ring
    // ---- bulk copies, issued by the lanes of warp 0: a fill of a ring slot
    // is nf field-planes of nrows rows from global row yfirst on (wrapped),
    // each in at most three contiguous pieces; lane f * 3 + j copies piece j
    // of field f, after lane 0 has posted the fill's bytes on the slot's mbarrier
    const auto fill = [&](int bi, int nf, int which, float *dst, int fstride, int z, int yfirst, int nrows) {
      const uint32_t bar = smem_u32(&bars[bi]);
      if (pfill >> bi & 1u) pph ^= 1u << bi;
      pfill |= 1u << bi;
      if (t == lane0) mbar_arrive_expect_tx(bar, uint32_t(nf * nrows * NX * 4));
      __syncwarp(wmask);
      for (int sI = t - lane0; sI < 3 * nf; sI += wlanes) {
        const int f = sI / 3, j = sI - 3 * f;
        int rr = 0, yy = wrap(yfirst, NY), cnt = min(nrows, NY - yy);
        for (int i = 0; i < j; ++i) {
          rr += cnt;
          yy = 0;
          cnt = min(nrows - rr, NY);
        }
        if (cnt <= 0) continue;
        const float *src = which == 0   ? a.s[0]
                           : which == 1 ? (f == 0 ? a.s[1] : f == 1 ? a.s[2] : f == 2 ? a.s[3] : a.pp)
                                        : (f < NUN ? (f == 0 ? a.n[0] : f == 1 ? a.n[1] : f == 2 ? a.n[2] : a.n[3])
                                                   : (f == NUN ? a.d_in[0] : f == NUN + 1 ? a.d_in[1] : a.d_in[2]));
        size_t first = (size_t(z) * NY + yy) * NX;
#ifdef IC_BOUNDS_CHECK
        // the piece [first, first + cnt NX) lies in the field; else it is copied from the field's start
        if (first + size_t(cnt) * NX > size_t(NX) * NY * NZ) {
          (void)IC_CHK(1, 0);
          first = 0;
        }
#endif
        bulk_g2s(smem_u32(dst + f * fstride + rr * NX), src + first, uint32_t(cnt * NX * 4), bar);
      }
    };
    const auto issue_d = [&](int p) {
      const int slot = (p - pbase) % NSD;
      fill(slot, 1, 0, sd + slot * RD * NX, 0, zw(p), ystart, RD);
    };
    const auto issue_g = [&](int p) {
      const int slot = (p - pbase) % NSG;
      fill(NSD + slot, a.pp ? 4 : 3, 1, sg + slot * 4 * plane, plane, zw(p), ystart, R);
    };
    const auto issue_n = [&](int p) {
      const int slot = (p - z0) % NSN;
      fill(NSD + NSG + slot, NFN, 2, sn + slot * NFN * TY * NX, TY * NX, zw(p), y0, TY);
    };
    // the fills due once every plane up to k is consumed (the issuing lanes
    // issue; every thread keeps the counters)
    const auto refill = [&](int dmax, int gmax, int nmax) {
      for (; next_d <= dmax; ++next_d)
        if (issuer) issue_d(next_d);
      for (; next_g <= gmax; ++next_g)
        if (issuer) issue_g(next_g);
      if (NFN > 0)
        for (; next_n <= nmax; ++next_n)
          if (issuer) issue_n(next_n);
    };

    if (copier) {
      // The copy warp: after each go signal of the compute threads (the run's
      // start; then the first barrier of each plane, once the slots of the
      // planes consumed so far are free) the fills that are due.  A missing
      // signal (the compute threads gave up) ends the CTA's copies.
      for (int k = pbase - 1; k < z1; ++k) {
        if (!mbar_wait(go_bar, go_ph)) {
          bad = true;
          break;
        }
        go_ph ^= 1u;
        if (k < pbase)
          refill(min(z1 + 1, pbase + NSD - 1), min(z1, pbase + NSG - 1), min(z1 - 1, z0 + NSN - 1));
        else
          refill(min(z1 + 1, k + 1 + NSD), min(z1, k - 1 + NSG), min(z1 - 1, k - 1 + NSN));
      }
      if (bad) break;
      continue;
    }

    cbar<PROD>(T);   // the previous run's reads of shared memory are done
    if (PROD) {
      if (t == 0) mbar_arrive(go_bar);
    } else {
      refill(min(z1 + 1, pbase + NSD - 1), min(z1, pbase + NSG - 1), min(z1 - 1, z0 + NSN - 1));
    }
    // a copy that did not land in time: flag it, give the copies in flight a
    // bounded wait (thread 0 issued them) and leave the CTA
    const auto abort_run = [&]() {
      if (PROD) {   // the copy warp waits for the copies it issued
        if (t == 0 && a.status) atomicOr(a.status, kStatusStaging);
        return;
      }
      if (t == 0) {
        if (a.status) atomicOr(a.status, kStatusStaging);
        for (; wd < next_d; ++wd) wait_bar((wd - pbase) % NSD);
        for (; wg < next_g; ++wg) wait_bar(NSD + (wg - pbase) % NSG);
        if (NFN > 0)
          for (; wn < next_n; ++wn) wait_bar(NSD + NSG + (wn - z0) % NSN);
      }
    };

    // ---- phase A: the finished values of plane p (face velocities, 4 pi),
    // with its velocities written for the neighbours
    const auto finish = [&](int p, PlaneQ<VC> &Q) {
      for (; wd <= p + 1; ++wd) wait_bar((wd - pbase) % NSD);
      for (; wg <= p; ++wg) wait_bar(NSD + (wg - pbase) % NSG);
      const float *D0 = sd + ((p - pbase) % NSD) * RD * NX;
      const float *D1 = sd + ((p + 1 - pbase) % NSD) * RD * NX;
      const float *G = sg + ((p - pbase) % NSG) * 4 * plane;
      const Cells<VC> dr = ldc<VC>(D0 + r * NX + xq), dry = ldc<VC>(D0 + rpd * NX + xq), drz = ldc<VC>(D1 + r * NX + xq);
      const float dr_r = D0[r * NX + ep];
      const Cells<VC> gx = ldc<VC>(G + r * NX + xq), gy = ldc<VC>(G + plane + r * NX + xq), gz = ldc<VC>(G + 2 * plane + r * NX + xq);
      Cells<VC> pp{};
      if (a.pp) pp = ldc<VC>(G + 3 * plane + r * NX + xq);
#pragma unroll
      for (int e = 0; e < VC; ++e) {
        const float drx = e < VC - 1 ? dr.v[e + 1] : dr_r;
        Q.dr[e] = dr.v[e];
        Q.gx[e] = gx.v[e];
        Q.gy[e] = gy.v[e];
        Q.gz[e] = gz.v[e];
        Q.vx[e] = __fdividef(gx.v[e], fma_rn(0.5f, add_rn(dr.v[e], drx), rho0));
        Q.vy[e] = __fdividef(gy.v[e], fma_rn(0.5f, add_rn(dr.v[e], dry.v[e]), rho0));
        Q.vz[e] = __fdividef(gz.v[e], fma_rn(0.5f, add_rn(dr.v[e], drz.v[e]), rho0));
        Q.pk[e] = add_rn(fma_rn(c2x4, dr.v[e], mul_rn(4.0f, pp.v[e])), mul_rn(drive4, profile(p, e)));
      }
      float *V = sv + (p & 1) * 3 * plane + r * NX + xq;
      stc<VC>(V, Q.vx);
      stc<VC>(V + plane, Q.vy);
      stc<VC>(V + 2 * plane, Q.vz);
    };

    PlaneQ<VC> P;
    finish(pbase, P);
    float gz_m[VC], txz_m[VC], tyz_m[VC], tzz_k[VC], bulk_k[VC];
#pragma unroll
    for (int e = 0; e < VC; ++e) gz_m[e] = txz_m[e] = tyz_m[e] = tzz_k[e] = bulk_k[e] = 0.0f;

    for (int k = pbase; k < z1; ++k) {
      const bool body = k >= z0;   // the first pass only supplies the z-carried fluxes
      PlaneQ<VC> Q;
      finish(k + 1, Q);
      if (cbar_or<PROD>(T, bad)) {
        abort_run();
        return;
      }
      // the ring slots of the planes consumed up to phase A are refilled
      if (PROD) {
        if (t == 0) mbar_arrive(go_bar);
      } else {
        refill(min(z1 + 1, k + 1 + NSD), min(z1, k - 1 + NSG), min(z1 - 1, k - 1 + NSN));
      }

      // ---- phase B: the scaled fluxes at plane k (and T_zz at k + 1)
      const float *GXk = sg + ((k - pbase) % NSG) * 4 * plane, *GYk = GXk + plane, *GZk = GXk + 2 * plane;
      const float *VXk = sv + (k & 1) * 3 * plane, *VYk = VXk + plane, *VZk = VXk + 2 * plane;
      const float *VXq = sv + ((k + 1) & 1) * 3 * plane, *VYq = VXq + plane;
      const int row = r * NX;
      const size_t gi = IC_CHK((size_t(zw(k)) * NY + y) * NX + xq, size_t(NX) * NY * NZ - (VC - 1));
      const Cells<VC> qvy_ym = ldc<VC>(VYq + rm * NX + xq);
      const float qvx_l = VXq[row + em];
      float bulk_up[VC], tzz_up[VC], txz[VC], tyz[VC];
      const Cells<VC> vz_yp = ldc<VC>(VZk + rp * NX + xq);
      const float vz_r = VZk[row + ep];
      float txx[VC], tyy[VC], txy[VC], tyx[VC], tzx[VC], tzy[VC];
      {
        const Cells<VC> gy_ym = ldc<VC>(GYk + rm * NX + xq), vy_ym = ldc<VC>(VYk + rm * NX + xq);
        const Cells<VC> gx_yp = ldc<VC>(GXk + rp * NX + xq), vx_yp = ldc<VC>(VXk + rp * NX + xq);
        const Cells<VC> gz_yp = ldc<VC>(GZk + rp * NX + xq);
        const float gx_l = GXk[row + em], vx_l = VXk[row + em];
        const float gy_r = GYk[row + ep], vy_r = VYk[row + ep], gz_r = GZk[row + ep];
#pragma unroll
        for (int e = 0; e < VC; ++e) {
          const float gx_xm = e > 0 ? P.gx[e - 1] : gx_l, vx_xm = e > 0 ? P.vx[e - 1] : vx_l;
          const float gy_xp = e < VC - 1 ? P.gy[e + 1] : gy_r, vy_xp = e < VC - 1 ? P.vy[e + 1] : vy_r;
          const float gz_xp = e < VC - 1 ? P.gz[e + 1] : gz_r, vz_xp = e < VC - 1 ? P.vz[e + 1] : vz_r;
          const float qvx_xm = e > 0 ? Q.vx[e - 1] : qvx_l;
          // h div v one plane up, and the bulk-viscous term 4 lam2 div v
          const float dsum_up =
              add_rn(add_rn(sub_rn(Q.vx[e], qvx_xm), sub_rn(Q.vy[e], qvy_ym.v[e])), sub_rn(Q.vz[e], P.vz[e]));
          bulk_up[e] = mul_rn(lam2x4_h, dsum_up);
          // the fluxes times 4: products of two-point sums, pressure, minus 4 sigma
          tzz_up[e] = add_rn(mul_rn(add_rn(P.gz[e], Q.gz[e]), add_rn(P.vz[e], Q.vz[e])), Q.pk[e]);
          tzz_up[e] = sub_rn(tzz_up[e], fma_rn(visc_d, sub_rn(Q.vz[e], P.vz[e]), bulk_up[e]));
          const float visc_xz = mul_rn(visc_o, add_rn(sub_rn(Q.vx[e], P.vx[e]), sub_rn(vz_xp, P.vz[e])));
          txz[e] = sub_rn(mul_rn(add_rn(P.gx[e], Q.gx[e]), add_rn(P.vz[e], vz_xp)), visc_xz);
          tzx[e] = sub_rn(mul_rn(add_rn(P.gz[e], gz_xp), add_rn(P.vx[e], Q.vx[e])), visc_xz);
          const float visc_yz = mul_rn(visc_o, add_rn(sub_rn(Q.vy[e], P.vy[e]), sub_rn(vz_yp.v[e], P.vz[e])));
          tyz[e] = sub_rn(mul_rn(add_rn(P.gy[e], Q.gy[e]), add_rn(P.vz[e], vz_yp.v[e])), visc_yz);
          tzy[e] = sub_rn(mul_rn(add_rn(P.gz[e], gz_yp.v[e]), add_rn(P.vy[e], Q.vy[e])), visc_yz);
          if (body) {
            txx[e] = add_rn(mul_rn(add_rn(gx_xm, P.gx[e]), add_rn(vx_xm, P.vx[e])), P.pk[e]);
            txx[e] = sub_rn(txx[e], fma_rn(visc_d, sub_rn(P.vx[e], vx_xm), bulk_k[e]));
            tyy[e] = add_rn(mul_rn(add_rn(gy_ym.v[e], P.gy[e]), add_rn(vy_ym.v[e], P.vy[e])), P.pk[e]);
            tyy[e] = sub_rn(tyy[e], fma_rn(visc_d, sub_rn(P.vy[e], vy_ym.v[e]), bulk_k[e]));
            const float visc_xy = mul_rn(visc_o, add_rn(sub_rn(vx_yp.v[e], P.vx[e]), sub_rn(vy_xp, P.vy[e])));
            txy[e] = sub_rn(mul_rn(add_rn(P.gx[e], gx_yp.v[e]), add_rn(P.vy[e], vy_xp)), visc_xy);
            tyx[e] = sub_rn(mul_rn(add_rn(P.gy[e], gy_xp), add_rn(P.vx[e], vx_yp.v[e])), visc_xy);
          }
        }
      }
      if (body) {
        float *T = st + row + xq;
        stc<VC>(T, tyy);
        stc<VC>(T + plane, txy);
        stc<VC>(T + 2 * plane, tzy);
        stb[r * QX + q] = txx[0];
        stb[RQ + r * QX + q] = tyx[VC - 1];
        stb[2 * RQ + r * QX + q] = tzx[VC - 1];
      }
      cbar<PROD>(T);

      // ---- phase C: divergence, noise, RK combination, stores
      if (NFN > 0 && body)   // every thread waits on every fill: the parities stay in step
        for (; wn <= k; ++wn) wait_bar(NSD + NSG + (wn - z0) % NSN);
      if (body && own) {
        const Cells<VC> gy_ym = ldc<VC>(GYk + rm * NX + xq);
        const float gx_l = GXk[row + em];
        const Cells<VC> Tyy_p = ldc<VC>(st + rp * NX + xq), Txy_m = ldc<VC>(st + plane + rm * NX + xq),
                   Tzy_m = ldc<VC>(st + 2 * plane + rm * NX + xq);
        const float Txx_r = stb[r * QX + qp], Tyx_l = stb[RQ + r * QX + qm], Tzx_l = stb[2 * RQ + r * QX + qm];
        float o[4][VC];
        Cells<VC> un[4], dn[3];
        if (NFN > 0) {
          const float *U = sn + ((k - z0) % NSN) * NFN * TY * NX + ur * NX + xq;
#pragma unroll
          for (int j = 0; j < NUN; ++j) un[j] = ldc<VC>(U + j * TY * NX);
          if (NOISE) {
#pragma unroll
            for (int j = 0; j < 3; ++j) dn[j] = ldc<VC>(U + (NUN + j) * TY * NX);
          }
        }
#pragma unroll
        for (int e = 0; e < VC; ++e) {
          const float gx_xm = e > 0 ? P.gx[e - 1] : gx_l;
          const float Txx_xp = e < VC - 1 ? txx[e + 1] : Txx_r;
          const float Tyx_xm = e > 0 ? tyx[e - 1] : Tyx_l;
          const float Tzx_xm = e > 0 ? tzx[e - 1] : Tzx_l;
          // U_s + dt dU/dt: the mass flux divergence times -dt/h, the summed
          // differences of the scaled fluxes times -dt/(4h), minus the noise
          const float s_rho =
              add_rn(add_rn(sub_rn(P.gx[e], gx_xm), sub_rn(P.gy[e], gy_ym.v[e])), sub_rn(P.gz[e], gz_m[e]));
          float s_gx = add_rn(add_rn(sub_rn(Txx_xp, txx[e]), sub_rn(txy[e], Txy_m.v[e])), sub_rn(txz[e], txz_m[e]));
          float s_gy = add_rn(add_rn(sub_rn(Tyy_p.v[e], tyy[e]), sub_rn(tyx[e], Tyx_xm)), sub_rn(tyz[e], tyz_m[e]));
          float s_gz =
              add_rn(add_rn(sub_rn(tzz_up[e], tzz_k[e]), sub_rn(tzx[e], Tzx_xm)), sub_rn(tzy[e], Tzy_m.v[e]));
          if (NOISE) {
            s_gx = sub_rn(s_gx, dn[0].v[e]);
            s_gy = sub_rn(s_gy, dn[1].v[e]);
            s_gz = sub_rn(s_gz, dn[2].v[e]);
          }
          o[0][e] = fma_rn(s_rho, out_mass, P.dr[e]);
          o[1][e] = fma_rn(s_gx, out_flux, P.gx[e]);
          o[2][e] = fma_rn(s_gy, out_flux, P.gy[e]);
          o[3][e] = fma_rn(s_gz, out_flux, P.gz[e]);
          if (STAGE != 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j][e] = fma_rn(ca, un[j].v[e], mul_rn(cb, o[j][e]));
          }
          if (STAGE == 2) {
            const float cw = c.wave_axis == 0 ? cosx[e] : (c.wave_axis == 1 ? cosy : c.cos_table[zw(k)]);
            mode_acc = fmaf(o[0][e], cw, mode_acc);
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) stc<VC>(a.o[j] + gi, o[j]);
      }
#pragma unroll
      for (int e = 0; e < VC; ++e) {
        gz_m[e] = P.gz[e];
        txz_m[e] = txz[e];
        tyz_m[e] = tyz[e];
        tzz_k[e] = tzz_up[e];
        bulk_k[e] = bulk_up[e];
      }
      P = Q;
    }
  }

  if (copier) {
    // every copy this warp issued has landed before the CTA leaves (bounded)
    for (int i = 0; i < kRowsMaxBars; ++i)
      if (pfill >> i & 1u) (void)mbar_wait(smem_u32(&bars[i]), (pph >> i) & 1u);
    if (bad && t == T && a.status) atomicOr(a.status, kStatusStaging);
    return;
  }
  if (STAGE == 2) {
    // per-CTA partial of sum (rho - rho0) cos(k x), fixed reduction order:
    // each warp's 32 values in order, then the warp sums in order
    __shared__ double s_w[32];
    s_acc[t] = mode_acc;
    cbar<PROD>(T);
    const int nw = (T + 31) / 32;
    if (t < nw) {
      double w = 0.0;
      for (int j = 32 * t; j < min(T, 32 * t + 32); ++j) w += double(s_acc[j]);
      s_w[t] = w;
    }
    cbar<PROD>(T);
    if (t == 0) {
      double s = 0.0;
      for (int j = 0; j < nw; ++j) s += s_w[j];
      a.partials[blockIdx.x] = s;
    }
  }
}

// ------------------------------------------------------------ noise kernel
// The stochastic stress of one step enters the three stages only through its
// divergence at the faces, and that is linear in the normals:
//   D_s = D(W_A) + beta_s D(W_B),  beta = (-sqrt3, +sqrt3, 0)  (App. A.2),
// with D(W) = div Sigma(W) (times 4, like the stage kernels' fluxes):
//   D^x = Sigma_xx(i+x) - Sigma_xx + Sigma_xy - Sigma_xy(i-y) + Sigma_xz - Sigma_xz(i-z)
//   D^y = Sigma_yy(i+y) - Sigma_yy + Sigma_xy - Sigma_xy(i-x) + Sigma_yz - Sigma_yz(i-z)
//   D^z = Sigma_zz(i+z) - Sigma_zz + Sigma_xz - Sigma_xz(i-x) + Sigma_yz - Sigma_yz(i-y)
// (the (a,b) edge stress owned by cell i sits at r_i + h/2 (e_a + e_b)).  This
// kernel draws W_A and W_B of every cell once per step (Philox4x32-10, the FP32
// normals of ic_device.cuh) over the same bands of whole rows as the stage
// kernel, exchanges the in-plane stresses through shared memory, marches z
// with the z neighbours in registers, and stores D_1, D_2, D_3 (nine words per
// cell) for the three stage launches.  It reads nothing from global memory.
constexpr int kNoiseMaxThreads = 576;

struct NoiseArgs {
  float *__restrict__ d[9];   // D_1 (x, y, z faces), D_2, D_3, each [z][y][x]
  int nx, ny, nz;
  float nd, nt, ne;           // 4 x (sqrt2 S, sqrt2 (B - S/3), S)
  RoundKeys rk;               // Philox round keys of the noise key
  uint32_t box;
  const int64_t *step;
  int ty, nrow, wrapy, ncols;
};

template <int VC>
__global__ void __launch_bounds__(kNoiseMaxThreads, 1) k_noise_rows(const NoiseArgs a) {
  pdl_enter();
  extern __shared__ __align__(16) float sm[];   // [plane parity][stream A, B][xx, yy, xy, xz, yz][R][NX]
  const int NX = a.nx, NY = a.ny, NZ = a.nz, QX = NX / VC;
  const int R = a.nrow, TY = a.ty, wrapy = a.wrapy;
  const int plane = R * NX;
  const int t = threadIdx.x;
  const int r = t / QX, q = t - r * QX, xq = VC * q;
  const int em = (q == 0 ? NX : xq) - 1, ep = q == QX - 1 ? 0 : xq + VC;
  const int rm = wrapy ? (r == 0 ? R - 1 : r - 1) : max(r - 1, 0);
  const int rp = wrapy ? (r == R - 1 ? 0 : r + 1) : min(r + 1, R - 1);
  const int row = r * NX;
  const uint32_t ustep = uint32_t(*a.step);
  const float nd = a.nd, nt = a.nt, ne = a.ne;
  const auto zw = [NZ](int p) { return p < 0 ? p + NZ : (p >= NZ ? p - NZ : p); };
  const auto buf = [&](int p, int sI, int comp) { return sm + (((p & 1) * 2 + sI) * 5 + comp) * plane; };

  const int units = a.ncols * NZ;
  const int u_end = int((long long)units * (blockIdx.x + 1) / gridDim.x);
  for (int u = int((long long)units * blockIdx.x / gridDim.x); u < u_end;) {
    const int col = u / NZ;
    const int z0 = u - col * NZ;
    const int z1 = min(NZ, z0 + (u_end - u));
    u += z1 - z0;
    const int y0 = wrapy ? 0 : col * TY;
    const int y = wrap((wrapy ? 0 : y0 - 1) + r, NY);
    const bool own = wrapy ? true : (r >= 1 && r <= TY && y0 - 1 + r < NY);
    const auto cell = [&](int p, int e) {
      return uint32_t(xq + e) + uint32_t(NX) * (uint32_t(y) + uint32_t(NY) * uint32_t(zw(p)));
    };
    // the stresses of plane p of both streams at this thread's cells, two at a
    // time: the in-plane components into the plane's buffer, Sigma_zz returned
    const auto draw = [&](int p, float zzA[VC], float zzB[VC]) {
#pragma unroll
      for (int h = 0; h < VC / 2; ++h) {
        float2 sxx[2], syy[2], sxy[2], sxz[2], syz[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int e = 2 * h + j;
          float w[2][6];
          stress_normals_ab_rk(a.rk, a.box, cell(p, e), ustep, w[0], w[1]);
#pragma unroll
          for (int sI = 0; sI < 2; ++sI) {
            // Sigma_aa = sqrt2 S N_aa + sqrt2 (B - S/3) tr N, Sigma_ab = S N_ab (times 4)
            const float ntr = mul_rn(nt, add_rn(add_rn(w[sI][0], w[sI][1]), w[sI][2]));
            (j == 0 ? sxx[sI].x : sxx[sI].y) = fma_rn(nd, w[sI][0], ntr);
            (j == 0 ? syy[sI].x : syy[sI].y) = fma_rn(nd, w[sI][1], ntr);
            (j == 0 ? sxy[sI].x : sxy[sI].y) = mul_rn(ne, w[sI][3]);
            (j == 0 ? sxz[sI].x : sxz[sI].y) = mul_rn(ne, w[sI][4]);
            (j == 0 ? syz[sI].x : syz[sI].y) = mul_rn(ne, w[sI][5]);
            (sI == 0 ? zzA : zzB)[e] = fma_rn(nd, w[sI][2], ntr);
          }
        }
#pragma unroll
        for (int sI = 0; sI < 2; ++sI) {
          const int o = row + xq + 2 * h;
          *reinterpret_cast<float2 *>(buf(p, sI, 0) + o) = sxx[sI];
          *reinterpret_cast<float2 *>(buf(p, sI, 1) + o) = syy[sI];
          *reinterpret_cast<float2 *>(buf(p, sI, 2) + o) = sxy[sI];
          *reinterpret_cast<float2 *>(buf(p, sI, 3) + o) = sxz[sI];
          *reinterpret_cast<float2 *>(buf(p, sI, 4) + o) = syz[sI];
        }
      }
    };

    __syncthreads();   // the previous run's reads of shared memory are done
    // Sigma_xz, Sigma_yz of the plane below the run (own cells: blocks 1, 2 only)
    float xzA[VC], yzA[VC], xzB[VC], yzB[VC];
#pragma unroll
    for (int e = 0; e < VC; ++e) {
      const uint4 h1 = philox4x32_10_rk(make_uint4(cell(z0 - 1, e), ustep, (kPurposeStress << 16) | 1u, a.box), a.rk);
      const uint4 h2 = philox4x32_10_rk(make_uint4(cell(z0 - 1, e), ustep, (kPurposeStress << 16) | 2u, a.box), a.rk);
      float w4, w5, u4, u5;
      box_muller_f32(h1.x, h1.y, w4, w5);   // W_A: xz, yz
      box_muller_f32(h2.z, h2.w, u4, u5);   // W_B: xz, yz
      xzA[e] = mul_rn(ne, w4);
      yzA[e] = mul_rn(ne, w5);
      xzB[e] = mul_rn(ne, u4);
      yzB[e] = mul_rn(ne, u5);
    }
    float zzA[VC], zzB[VC];
    draw(z0, zzA, zzB);
    for (int k = z0; k < z1; ++k) {
      float znA[VC], znB[VC];
      draw(k + 1, znA, znB);
      __syncthreads();   // plane k's buffer is complete (and plane k + 1's)
      if (own) {
        float D[2][3][VC];
#pragma unroll
        for (int sI = 0; sI < 2; ++sI) {
          const float *XX = buf(k, sI, 0), *YY = buf(k, sI, 1), *XY = buf(k, sI, 2), *XZ = buf(k, sI, 3),
                      *YZ = buf(k, sI, 4);
          const Cells<VC> xx = ldc<VC>(XX + row + xq), yy = ldc<VC>(YY + row + xq), yy_p = ldc<VC>(YY + rp * NX + xq);
          const Cells<VC> xy = ldc<VC>(XY + row + xq), xy_m = ldc<VC>(XY + rm * NX + xq);
          const Cells<VC> xz = ldc<VC>(XZ + row + xq), yz = ldc<VC>(YZ + row + xq), yz_m = ldc<VC>(YZ + rm * NX + xq);
          const float xx_r = XX[row + ep], xy_l = XY[row + em], xz_l = XZ[row + em];
          float *xz_prev = sI == 0 ? xzA : xzB, *yz_prev = sI == 0 ? yzA : yzB;
          const float *zz = sI == 0 ? zzA : zzB, *zn = sI == 0 ? znA : znB;
#pragma unroll
          for (int e = 0; e < VC; ++e) {
            const float xxp = e < VC - 1 ? xx.v[e + 1] : xx_r;
            const float xyl = e > 0 ? xy.v[e - 1] : xy_l;
            const float xzl = e > 0 ? xz.v[e - 1] : xz_l;
            D[sI][0][e] = add_rn(add_rn(sub_rn(xxp, xx.v[e]), sub_rn(xy.v[e], xy_m.v[e])), sub_rn(xz.v[e], xz_prev[e]));
            D[sI][1][e] = add_rn(add_rn(sub_rn(yy_p.v[e], yy.v[e]), sub_rn(xy.v[e], xyl)), sub_rn(yz.v[e], yz_prev[e]));
            D[sI][2][e] = add_rn(sub_rn(zn[e], zz[e]), add_rn(sub_rn(xz.v[e], xzl), sub_rn(yz.v[e], yz_m.v[e])));
            xz_prev[e] = xz.v[e];
            yz_prev[e] = yz.v[e];
          }
        }
        const size_t gi = IC_CHK((size_t(zw(k)) * NY + y) * NX + xq, size_t(NX) * NY * NZ - (VC - 1));
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          float d1[VC], d2[VC];
#pragma unroll
          for (int e = 0; e < VC; ++e) {
            d1[e] = fma_rn(-1.7320508075688772f, D[1][j][e], D[0][j][e]);
            d2[e] = fma_rn(1.7320508075688772f, D[1][j][e], D[0][j][e]);
          }
          stc<VC>(a.d[j] + gi, d1);
          stc<VC>(a.d[3 + j] + gi, d2);
          stc<VC>(a.d[6 + j] + gi, D[0][j]);
        }
      }
#pragma unroll
      for (int e = 0; e < VC; ++e) {
        zzA[e] = znA[e];
        zzB[e] = znB[e];
      }
      __syncthreads();   // plane k's buffer is read: the next draw may refill it
    }
  }
}

size_t noise_smem(int nx, int R) { return size_t(20) * R * nx * sizeof(float); }

struct RowsPlan {
  int vc = 4, ty = 0, nrow = 0, wrapy = 0, ncols = 0, threads = 0, ctas = 0;
  bool prod = false;   // a copy warp beside the compute threads (whole warps of them)
  size_t smem = 0;
};

size_t rows_smem(int nx, int vc, int R, int RD, int ty, int stage, bool noise) {
  return size_t(row_layout(nx, vc, R, RD, ty, stage, noise).total) * sizeof(float);
}

// The tile of one stage for vc cells per thread: among the own-row counts
// whose launch fits the thread and shared-memory limits (a tile of every row,
// without ring rows, where it fits), the one with the least time per CTA,
// modelled as (planes per CTA + the run's first plane) x max(thread rows,
// 256 / (nx / vc)) (a CTA of fewer than eight warps is latency-bound), with the
// grid the SMs' CTAs or one CTA per zmin planes of the (tile, plane) units,
// whichever is fewer; ties go to the fewest thread rows in all.
RowsPlan rows_plan(const ic_grid_params &p, int stage, int sm_count, int zmin, int vc) {
  RowsPlan best;
  best.vc = vc;
  const bool noise = p.kT > 0.0;
  const int qx = p.nx / vc;
  const int max_threads = 80 * vc;
  double best_cost = 1e300;
  for (int ty = 1; ty <= p.ny; ++ty) {
    const bool wy = ty == p.ny;
    const int R = wy ? p.ny : ty + 2, RD = wy ? R : R + 1;
    if (qx * R > max_threads || rows_smem(p.nx, vc, R, RD, ty, stage, noise) > kRowsSmemCap) continue;
    const int ncols = wy ? 1 : (p.ny + ty - 1) / ty;
    const long long units = (long long)ncols * p.nz;
    const long long ctas = std::max<long long>(1, std::min<long long>(sm_count, (units + zmin - 1) / zmin));
    const double cost = (double(units) / double(ctas) + 1.0) * std::max(double(R), 256.0 * vc / (4.0 * qx));
    const bool tie = cost <= best_cost * (1.0 + 1e-9) && cost >= best_cost * (1.0 - 1e-9);
    if (cost < best_cost * (1.0 - 1e-9) || (tie && ncols * R < best.ncols * best.nrow)) {
      best_cost = cost;
      best.ty = ty;
      best.nrow = R;
      best.wrapy = wy ? 1 : 0;
      best.ncols = ncols;
      best.ctas = int(ctas);
    }
  }
  if (best.ty == 0) return best;
  best.prod = (qx * best.nrow) % 32 == 0;
  best.threads = qx * best.nrow + (best.prod ? 32 : 0);
  const int RD = best.wrapy ? best.nrow : best.nrow + 1;
  best.smem = rows_smem(p.nx, vc, best.nrow, RD, best.ty, stage, noise);
  return best;
}

template <int VC, int STAGE, bool NOISE, bool PROD>
cudaError_t launch_rows_t(const RowArgs &a, const RowsPlan &pl, cudaStream_t stream) {
  auto kern = k_stage_rows<VC, STAGE, NOISE, PROD>;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kRowsSmemCap));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_k(kern, dim3(pl.ctas), dim3(pl.threads), pl.smem, stream, a);
}

template <int VC, bool PROD>
cudaError_t launch_rows_p(const RowArgs &a, const RowsPlan &pl, int stage, bool noise, cudaStream_t stream) {
  switch (stage * 2 + (noise ? 1 : 0)) {
    case 0: return launch_rows_t<VC, 0, false, PROD>(a, pl, stream);
    case 1: return launch_rows_t<VC, 0, true, PROD>(a, pl, stream);
    case 2: return launch_rows_t<VC, 1, false, PROD>(a, pl, stream);
    case 3: return launch_rows_t<VC, 1, true, PROD>(a, pl, stream);
    case 4: return launch_rows_t<VC, 2, false, PROD>(a, pl, stream);
    default: return launch_rows_t<VC, 2, true, PROD>(a, pl, stream);
  }
}

template <int VC>
cudaError_t launch_rows_v(const RowArgs &a, const RowsPlan &pl, int stage, bool noise, cudaStream_t stream) {
  return pl.prod ? launch_rows_p<VC, true>(a, pl, stage, noise, stream)
                 : launch_rows_p<VC, false>(a, pl, stage, noise, stream);
}

int rows_zmin(const ic_ctx *ctx) { return ctx->zchunk > 0 ? ctx->zchunk : kMinZChunk; }

struct NoisePlan {
  int ty = 0, nrow = 0, wrapy = 0, ncols = 0, threads = 0, ctas = 0;
  size_t smem = 0;
};

// Bands of the noise kernel: as rows_plan, with the run's extra planes of
// noise (the plane above and half of the plane below) in the cost, and CTAs
// of fewer than 16 warps counted as if they had 16.
NoisePlan noise_plan(const ic_grid_params &p, int sm_count) {
  NoisePlan best;
  const int qx = p.nx / kRowsVC;
  double best_cost = 1e300;
  for (int ty = 1; ty <= p.ny; ++ty) {
    const bool wy = ty == p.ny;
    const int R = wy ? p.ny : ty + 2;
    if (qx * R > kNoiseMaxThreads || noise_smem(p.nx, R) > kRowsSmemCap) continue;
    const int ncols = wy ? 1 : (p.ny + ty - 1) / ty;
    const long long units = (long long)ncols * p.nz;
    const long long ctas = std::max<long long>(1, std::min<long long>(sm_count, (units + kMinZChunk - 1) / kMinZChunk));
    // the draw is issue-bound: fewer than 16 warps leave issue slots idle
    const double cost = (double(units) / double(ctas) + 1.7) * std::max(qx * R, 512);
    if (cost < best_cost * (1.0 - 1e-9)) {
      best_cost = cost;
      best.ty = ty;
      best.nrow = R;
      best.wrapy = wy ? 1 : 0;
      best.ncols = ncols;
      best.ctas = int(ctas);
    }
  }
  if (best.ty == 0) return best;
  best.threads = qx * best.nrow;
  best.smem = noise_smem(p.nx, best.nrow);
  return best;
}

// The step's stress divergences D_1, D_2, D_3 into noise[0..8].
cudaError_t launch_noise_rows(const ic_ctx *ctx) {
  const NoisePlan pl = noise_plan(ctx->p, ctx->sm_count);
  if (pl.ty == 0) return cudaErrorInvalidConfiguration;
  const FluidConsts<float> c = make_fluid_consts<float>(ctx->p, ctx->cos_table_f, ctx->drive_f);
  NoiseArgs a{};
  for (int j = 0; j < 9; ++j) a.d[j] = static_cast<float *>(ctx->noise[j]);
  a.nx = ctx->p.nx;
  a.ny = ctx->p.ny;
  a.nz = ctx->p.nz;
  a.nd = c.noise_d4;
  a.nt = c.noise_t4;
  a.ne = c.noise_e4;
  a.rk = philox_round_keys(c.k0, c.k1);
  a.box = c.box;
  a.step = ctx->d.step;
  a.ty = pl.ty;
  a.nrow = pl.nrow;
  a.wrapy = pl.wrapy;
  a.ncols = pl.ncols;
  auto kern = k_noise_rows<kRowsVC>;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kRowsSmemCap));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_k(kern, dim3(pl.ctas), dim3(pl.threads), pl.smem, ctx->stream, a);
}

}  // namespace

bool rows_eligible(const ic_grid_params &p) {
  if (p.precision != IC_FP32 || p.nx % 4 != 0 || p.nx > kRowsMaxNx) return false;
  for (int s = 0; s < 3; ++s)
    if (rows_plan(p, s, 1, 1, kRowsVC).ty == 0) return false;
  return p.kT == 0.0 || noise_plan(p, 1).ty != 0;
}

bool rows_buffers_aligned(const ic_ctx *ctx) {
  const auto al = [](const void *q) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  for (int b = 0; b < 3; ++b)
    for (int j = 0; j < 4; ++j)
      if (!al(ctx->U[b][j])) return false;
  if (!al(ctx->pp)) return false;
  for (int j = 0; j < 9; ++j)
    if (!al(ctx->noise[j])) return false;
  return true;
}

double rows_mean_run(const ic_grid_params &p, int sm_count) {
  const RowsPlan pl = rows_plan(p, 1, sm_count, 1, kRowsVC);
  if (pl.ty == 0 || pl.ctas == 0) return 0.0;
  return double(pl.ncols) * double(p.nz) / double(pl.ctas);
}

int rows_ctas(const ic_ctx *ctx, int stage) {
  return rows_plan(ctx->p, stage, ctx->sm_count, rows_zmin(ctx), kRowsVC).ctas;
}

void rows_tile(const ic_ctx *ctx, int *ty) { *ty = rows_plan(ctx->p, 1, ctx->sm_count, rows_zmin(ctx), kRowsVC).ty; }

cudaError_t launch_stage_rows(const ic_ctx *ctx, int stage, void *const in_s[4], void *const in_n[4],
                              void *const out[4]) {
  const RowsPlan pl = rows_plan(ctx->p, stage, ctx->sm_count, rows_zmin(ctx), kRowsVC);
  if (pl.ty == 0) return cudaErrorInvalidConfiguration;
  RowArgs a{};
  for (int j = 0; j < 4; ++j) {
    a.s[j] = static_cast<const float *>(in_s[j]);
    a.n[j] = static_cast<const float *>(in_n[j]);
    a.o[j] = static_cast<float *>(out[j]);
  }
  a.pp = ctx->ps.n > 0 ? static_cast<const float *>(ctx->pp) : nullptr;
  const bool noise = ctx->p.kT > 0.0;
  for (int j = 0; j < 3; ++j) a.d_in[j] = noise ? static_cast<const float *>(ctx->noise[3 * stage + j]) : nullptr;
  if (noise && stage == 0) {   // the step's noise first: D_1, D_2, D_3 for the three stages
    const cudaError_t e = launch_noise_rows(ctx);
    if (e != cudaSuccess) return e;
  }
  a.c = make_fluid_consts<float>(ctx->p, ctx->cos_table_f, ctx->drive_f);
  a.step = ctx->d.step;
  a.partials = ctx->d.partials;
  a.status = ctx->d.status;
  a.ty = pl.ty;
  a.nrow = pl.nrow;
  a.wrapy = pl.wrapy;
  a.ncols = pl.ncols;
  const char *stall = std::getenv("IC_STAGE_STALL_TEST");
  a.stall = stall && stall[0] == '1' ? 1 : 0;
  return launch_rows_v<kRowsVC>(a, pl, stage, noise, ctx->stream);
}

IC_BOUNDS_READER(bounds_flag_rows)

}  // namespace ic
