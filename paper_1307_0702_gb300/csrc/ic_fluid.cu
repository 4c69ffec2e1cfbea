// Fluid kernels of libic: one SSP-RK3 stage of compressible Landau-Lifshitz
// fluctuating hydrodynamics on the periodic staggered grid (Sec. 4.2 and
// App. A.2), the thermal initial state and the grid reductions.
//
// Discretisation (conservative flux form; the paper defers it to other work):
//   d rho/dt   = -(1/h) sum_a (g^a_i - g^a_{i-a})
//   d g^a/dt   = -(1/h) [T_aa(i+a) - T_aa(i) + sum_{b!=a} (T_ab(i) - T_ab(i-b))]
//   T = g v + pi I - sigma - Sigma, diagonal at centres, off-diagonal on the
//   (a,b) edge owned by cell i (at r_i + h/2 (e_a + e_b)), v^a = g^a / rho^a with
//   the face density rho^a = (rho_i + rho_{i+a}) / 2;
//   advective parts are products of two-point averages; sigma = eta (grad v +
//   grad v^T) + (zeta - 2 eta/3) div v I; pi = c^2 (rho - rho0) + S Omega + p_ext
//   with the particle pressure S Omega read from a field written by
//   ic_particles.cu before each stage;
//   Sigma_aa = sqrt2 S N_aa + sqrt2 (B - S/3) tr N, Sigma_ab = S N_ab with
//   N = W_A + beta_s W_B (beta = -sqrt3, +sqrt3, 0 for stages 1..3).
//   Stage s: U_{s+1} = a_s U^n + b_s (U_s + dt dU/dt(U_s, t_s)), (a, b) =
//   (0, 1), (3/4, 1/4), (1/3, 2/3); t_s = t^n, t^{n+1}, t^{n+1/2}.
//
// Kernel layout.  The grid is cut into TX x TY columns of cells; a CTA marches
// up runs of z planes of a column ("2.5D" blocking).  Its (TX+2) x (TY+2)
// threads also cover a one-cell ring so that each thread computes the fluxes
// of one cell; the in-plane neighbours come from shared memory and the z
// neighbours from registers carried between planes.  Per plane: one load of
// the next plane, one flux evaluation, and one fused combination with U^n.
// State stores delta rho = rho - rho0.  Stage 1 draws W_A and W_B of each
// cell (Philox), uses W_1 and stores W_2 and W_3 for stages 2 and 3 (storing
// them costs less than drawing them three times).
//
// Schedule.  The (column, plane) pairs are numbered column by column and split
// into gridDim.x equal contiguous ranges, one per CTA; a range that crosses a
// column boundary is marched as two runs.  With the grid sized to the CTAs the
// SMs hold at once, every CTA gets the same number of planes, so no partial
// last wave is left (a grid of fixed z chunks leaves one at most sizes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "ic_async.cuh"
#include "ic_end_step.cuh"
#include "ic_device.cuh"
#include "ic_internal.hpp"

namespace ic {
namespace {

template <typename real>
struct StageArgs {
  const real *__restrict__ s[4];   // U_s
  const real *__restrict__ n[4];   // U^n
  real *__restrict__ o[4];         // U_{s+1}
  const real *__restrict__ pp;     // particle pressure S Omega_s at centres, or null
  const real *__restrict__ noise_in[6];   // stages 2-3 (and a pre-drawn stage 1): stored W_s
                                          // (xx, yy, zz, xy, xz, yz)
  real *__restrict__ noise_out[12];       // stage 1: stores W_2 = W_A + sqrt3 W_B and W_3 = W_A
  FluidConsts<real> c;
  const int64_t *step;
  double *partials;                // stage 3: per-CTA sum of delta rho cos(k x)
  int *status;                     // error bits (bulk staging timeout), or null
  int stall;                       // row staging: arrivals expected beyond the row threads' (0;
                                   // 1 only to test the bounded wait: nothing makes it)
  int ncols_x, ncols_y;            // tile columns along x and y
};


template <typename real>
struct NoiseOut {
  real *__restrict__ p[18];   // W_2 (0..5), W_3 (6..11), W_1 (12..17)
};

// ------------------------------------------------------------ FP64 noise
// The step's stochastic stresses drawn once per cell (App. A.2's W_A, W_B):
// W_1 = W_A - sqrt3 W_B, W_2 = W_A + sqrt3 W_B and W_3 = W_A, the same
// rounded operations as the stage-1 kernel's inline draw, so the step's bits
// do not depend on which of the two drew them.  The FP64 transcendentals of
// the 6 Box-Muller pairs dominate an FP64 step; drawn inline they are redone
// for the ring cells of every tile (1.6x the cells at 32 x 4, 1.4x at 32 x 6).
template <typename real>
__global__ void __launch_bounds__(256) k_draw_noise(RngKey key, const int64_t *step, uint32_t cells,
                                                    NoiseOut<real> w) {
  pdl_enter();
  const uint32_t ustep = uint32_t(*step);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += gridDim.x * blockDim.x) {
    real wa[6], wb[6];
    stress_normals_ab(key, i, ustep, wa, wb);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      w.p[12 + j][i] = fma_rn(real(-1.7320508075688772), wb[j], wa[j]);
      w.p[j][i] = fma_rn(real(1.7320508075688772), wb[j], wa[j]);
      w.p[6 + j][i] = wa[j];
    }
  }
}

template <typename real>
struct PlaneVals {
  real gx, gy, gz, vx, vy, vz, dr, pp;
  real nz[6];
};

// the global loads of one plane, issued one iteration before they are used
template <typename real>
struct PlaneRaw {
  real dr, drx, dry, drz, gx, gy, gz, pp;
};

constexpr double kStageTime[3] = {0.0, 1.0, 0.5};
constexpr double kStageA[3] = {0.0, 0.75, 1.0 / 3.0};
constexpr double kStageB[3] = {1.0, 0.25, 2.0 / 3.0};

// Tile height of the FP32 (pair) stage kernel and register budget of the
// scalar one, tuned on GB300.
#ifndef IC_FP32_TILE_Y
#define IC_FP32_TILE_Y 13
#endif
#ifndef IC_FP32_MIN_CTAS
#define IC_FP32_MIN_CTAS 2
#endif

// CTAs per SM the register budget of the scalar kernel is sized for: in FP32
// the budget of IC_FP32_MIN_CTAS CTAs of 340 threads, whatever the tile
template <typename real, int EXY>
constexpr int min_ctas() {
  return sizeof(real) == 4 ? (IC_FP32_MIN_CTAS * 340 + EXY - 1) / EXY : 1;
}

template <typename real, int TX, int TY, int STAGE, bool NOISE, bool PRE>
__global__ void __launch_bounds__((TX + 2) * (TY + 2), min_ctas<real, (TX + 2) * (TY + 2)>())
    k_rk3_stage(const StageArgs<real> a) {
  pdl_enter();
  constexpr int EX = TX + 2, EY = TY + 2, EXY = EX * EY;
  enum { GX = 0, GY, GZ, VX, VY, VZ };
  enum { TXX = 0, TYY, TXY, TYX, TZX, TZY };
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *sm = reinterpret_cast<real *>(smem_raw);
  real *T = sm + 12 * EXY;
  const FluidConsts<real> &c = a.c;
  const int NX = c.nx, NY = c.ny, NZ = c.nz;
  const int t = threadIdx.x;
  const int ex = t % EX, ey = t / EX;
  const int eXm = ey * EX + max(ex - 1, 0), eXp = ey * EX + min(ex + 1, EX - 1);
  const int eYm = max(ey - 1, 0) * EX + ex, eYp = min(ey + 1, EY - 1) * EX + ex;
  const auto zwrap = [NZ](int kk) { return kk < 0 ? kk + NZ : (kk >= NZ ? kk - NZ : kk); };

  const int64_t step = *a.step;
  const real four = real(4);
  const real drive4 = four * c.drive[STAGE];
  const real rho0 = c.rho0, half = real(0.5);
  const real c2x4 = c.c2x4, visc_d = c.visc_d, visc_o = c.visc_o, lam2x4_h = c.lam2x4_h;
  const real out_flux = c.out_flux, out_mass = c.out_mass;
  const real nd = c.noise_d4, nt = c.noise_t4, ne = c.noise_e4;
  const real beta = STAGE == 0 ? real(-1.7320508075688772) : (STAGE == 1 ? real(1.7320508075688772) : real(0));
  const RngKey key{c.k0, c.k1, c.box};
  const uint32_t ustep = uint32_t(step);
  const real ca = real(kStageA[STAGE]), cb = real(kStageB[STAGE]);
  const uint32_t plane_n = uint32_t(NX) * uint32_t(NY);
  [[maybe_unused]] const size_t cells = size_t(plane_n) * size_t(NZ);
  real mode_acc = real(0);

  // this CTA's share of the (column, plane) pairs
  const int units = a.ncols_x * a.ncols_y * NZ;
  const int u_end = int((long long)units * (blockIdx.x + 1) / gridDim.x);
  for (int u = int((long long)units * blockIdx.x / gridDim.x); u < u_end;) {
  const int col = u / NZ;
  const int z0 = u - col * NZ;
  const int z1 = min(NZ, z0 + (u_end - u));
  u += z1 - z0;
  const int gx_raw = (col % a.ncols_x) * TX + ex - 1;
  const int gy_raw = (col / a.ncols_x) * TY + ey - 1;
  const int x = wrap(gx_raw, NX), y = wrap(gy_raw, NY);
  const int xp = (x + 1 == NX) ? 0 : x + 1;
  const int yp = (y + 1 == NY) ? 0 : y + 1;
  const bool interior = ex >= 1 && ex <= TX && ey >= 1 && ey <= TY && gx_raw < NX && gy_raw < NY;
  __syncthreads();   // the previous run's last reads of shared memory are done

  // cos(k x) along the wave axis (mode amplitude and MODE drive), and the
  // drive profile: cos(k x) (MODE) or the indicator of the driven plane (PLANE)
  const real cos_xy = c.wave_axis < 2 ? c.cos_table[c.wave_axis == 0 ? x : y] : real(0);
  auto cosw = [&](int kk) -> real { return c.wave_axis < 2 ? cos_xy : c.cos_table[zwrap(kk)]; };
  auto profile = [&](int kk) -> real {
    if (c.forcing == IC_FORCE_MODE) return cosw(kk);
    if (c.forcing == IC_FORCE_PLANE) {
      const int coord = c.wave_axis == 0 ? x : (c.wave_axis == 1 ? y : zwrap(kk));
      return real(coord == c.plane_index ? 1 : 0);
    }
    return real(0);
  };

  // 32-bit cell offsets: in-plane offsets fixed per thread, plus k * plane
  const uint32_t o_c = uint32_t(x) + uint32_t(NX) * uint32_t(y);
  const uint32_t o_xp = uint32_t(xp) + uint32_t(NX) * uint32_t(y);
  const uint32_t o_yp = uint32_t(x) + uint32_t(NX) * uint32_t(yp);
  auto cell_of = [&](int kk) { return IC_CHK(o_c + uint32_t(zwrap(kk)) * plane_n, cells); };
  auto fetch = [&](int kk) {
    PlaneRaw<real> r;
    const int k = zwrap(kk);
    const uint32_t kb = uint32_t(k) * plane_n;
    const uint32_t kpb = (k + 1 == NZ) ? 0u : kb + plane_n;
    const uint32_t i = IC_CHK(o_c + kb, cells);
    r.dr = a.s[0][i];
    r.drx = a.s[0][IC_CHK(o_xp + kb, cells)];
    r.dry = a.s[0][IC_CHK(o_yp + kb, cells)];
    r.drz = a.s[0][IC_CHK(o_c + kpb, cells)];
    r.gx = a.s[1][i];
    r.gy = a.s[2][i];
    r.gz = a.s[3][i];
    r.pp = a.pp ? a.pp[i] : real(0);
    return r;
  };
  auto finish = [&](int kk, const PlaneRaw<real> &r) {
    PlaneVals<real> v;
    v.dr = r.dr;
    v.gx = r.gx;
    v.gy = r.gy;
    v.gz = r.gz;
    v.pp = r.pp;
    v.vx = fdiv(v.gx, fma_rn(half, v.dr + r.drx, rho0));
    v.vy = fdiv(v.gy, fma_rn(half, v.dr + r.dry, rho0));
    v.vz = fdiv(v.gz, fma_rn(half, v.dr + r.drz, rho0));
    if (NOISE && STAGE == 0 && !PRE) {
      // W_1 = W_A - sqrt3 W_B for this stage; the cell's own CTA stores W_2, W_3
      const uint32_t i = cell_of(kk);
      real wa[6], wb[6];
      stress_normals_ab(key, uint32_t(i), ustep, wa, wb);
#pragma unroll
      for (int j = 0; j < 6; ++j) v.nz[j] = fma_rn(beta, wb[j], wa[j]);
      if (interior && kk >= z0 && kk < z1) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          a.noise_out[j][i] = fma_rn(real(1.7320508075688772), wb[j], wa[j]);
          a.noise_out[6 + j][i] = wa[j];
        }
      }
    } else if (NOISE) {
      const uint32_t i = cell_of(kk);
#pragma unroll
      for (int j = 0; j < 6; ++j) v.nz[j] = a.noise_in[j][i];
    } else {
#pragma unroll
      for (int j = 0; j < 6; ++j) v.nz[j] = real(0);
    }
    return v;
  };
  auto store_plane = [&](int buf, const PlaneVals<real> &v) {
    real *B = sm + buf * 6 * EXY;
    B[GX * EXY + t] = v.gx;
    B[GY * EXY + t] = v.gy;
    B[GZ * EXY + t] = v.gz;
    B[VX * EXY + t] = v.vx;
    B[VY * EXY + t] = v.vy;
    B[VZ * EXY + t] = v.vz;
  };

  PlaneVals<real> P = finish(z0 - 1, fetch(z0 - 1));
  store_plane((z0 - 1) & 1, P);
  PlaneRaw<real> R = fetch(z0);
  real vz_m = real(0), gz_m = real(0), txz_m = real(0), tyz_m = real(0), tzz_k = real(0);

  for (int k = z0 - 1; k < z1; ++k) {
    // prefetch plane k + 2 (the last plane any flux of this chunk needs is z1)
    PlaneRaw<real> Rn;
    if (k + 2 <= z1) Rn = fetch(k + 2);
    // and U^n of the output plane k
    const bool out_here = interior && k >= z0;
    const uint32_t i_out = cell_of(k);
    real un[4] = {real(0), real(0), real(0), real(0)};
    if (STAGE != 0 && out_here) {
#pragma unroll
      for (int j = 0; j < 4; ++j) un[j] = a.n[j][i_out];
    }
    const PlaneVals<real> Q = finish(k + 1, R);
    store_plane((k + 1) & 1, Q);
    __syncthreads();
    const real *Pk = sm + (k & 1) * 6 * EXY;
    const real *Pq = sm + ((k + 1) & 1) * 6 * EXY;

    const real gx_xm = Pk[GX * EXY + eXm], vx_xm = Pk[VX * EXY + eXm];
    const real gy_ym = Pk[GY * EXY + eYm], vy_ym = Pk[VY * EXY + eYm];
    const real gx_yp = Pk[GX * EXY + eYp], vx_yp = Pk[VX * EXY + eYp];
    const real gy_xp = Pk[GY * EXY + eXp], vy_xp = Pk[VY * EXY + eXp];
    const real gz_xp = Pk[GZ * EXY + eXp], vz_xp = Pk[VZ * EXY + eXp];
    const real gz_yp = Pk[GZ * EXY + eYp], vz_yp = Pk[VZ * EXY + eYp];
    const real vx1_xm = Pq[VX * EXY + eXm], vy1_ym = Pq[VY * EXY + eYm];

    // h div v of the planes k and k + 1
    const real dsum_k = add_rn(add_rn(sub_rn(P.vx, vx_xm), sub_rn(P.vy, vy_ym)), sub_rn(P.vz, vz_m));
    const real dsum_k1 = add_rn(add_rn(sub_rn(Q.vx, vx1_xm), sub_rn(Q.vy, vy1_ym)), sub_rn(Q.vz, P.vz));
    // 4 pi = 4 (c^2 delta rho + S Omega + p_ext)
    const real pk = add_rn(fma_rn(c2x4, P.dr, mul_rn(four, P.pp)), mul_rn(drive4, profile(k)));
    const real pk1 = add_rn(fma_rn(c2x4, Q.dr, mul_rn(four, Q.pp)), mul_rn(drive4, profile(k + 1)));
    const real bulk_k = mul_rn(lam2x4_h, dsum_k), bulk_k1 = mul_rn(lam2x4_h, dsum_k1);

    // the fluxes times 4: products of two-point sums, pressure, minus 4 sigma
    real txx = add_rn(mul_rn(add_rn(gx_xm, P.gx), add_rn(vx_xm, P.vx)), pk);
    txx = sub_rn(txx, fma_rn(visc_d, sub_rn(P.vx, vx_xm), bulk_k));
    real tyy = add_rn(mul_rn(add_rn(gy_ym, P.gy), add_rn(vy_ym, P.vy)), pk);
    tyy = sub_rn(tyy, fma_rn(visc_d, sub_rn(P.vy, vy_ym), bulk_k));
    real tzz1 = add_rn(mul_rn(add_rn(P.gz, Q.gz), add_rn(P.vz, Q.vz)), pk1);
    tzz1 = sub_rn(tzz1, fma_rn(visc_d, sub_rn(Q.vz, P.vz), bulk_k1));
    const real visc_xy = mul_rn(visc_o, add_rn(sub_rn(vx_yp, P.vx), sub_rn(vy_xp, P.vy)));
    real txy = sub_rn(mul_rn(add_rn(P.gx, gx_yp), add_rn(P.vy, vy_xp)), visc_xy);
    real tyx = sub_rn(mul_rn(add_rn(P.gy, gy_xp), add_rn(P.vx, vx_yp)), visc_xy);
    const real visc_xz = mul_rn(visc_o, add_rn(sub_rn(Q.vx, P.vx), sub_rn(vz_xp, P.vz)));
    real txz = sub_rn(mul_rn(add_rn(P.gx, Q.gx), add_rn(P.vz, vz_xp)), visc_xz);
    real tzx = sub_rn(mul_rn(add_rn(P.gz, gz_xp), add_rn(P.vx, Q.vx)), visc_xz);
    const real visc_yz = mul_rn(visc_o, add_rn(sub_rn(Q.vy, P.vy), sub_rn(vz_yp, P.vz)));
    real tyz = sub_rn(mul_rn(add_rn(P.gy, Q.gy), add_rn(P.vz, vz_yp)), visc_yz);
    real tzy = sub_rn(mul_rn(add_rn(P.gz, gz_yp), add_rn(P.vy, Q.vy)), visc_yz);
    if (NOISE) {
      // Sigma_aa = sqrt2 S N_aa + sqrt2 (B - S/3) tr N, Sigma_ab = S N_ab
      const real ntr = mul_rn(nt, add_rn(add_rn(P.nz[0], P.nz[1]), P.nz[2]));
      const real ntr1 = mul_rn(nt, add_rn(add_rn(Q.nz[0], Q.nz[1]), Q.nz[2]));
      txx = sub_rn(txx, fma_rn(nd, P.nz[0], ntr));
      tyy = sub_rn(tyy, fma_rn(nd, P.nz[1], ntr));
      tzz1 = sub_rn(tzz1, fma_rn(nd, Q.nz[2], ntr1));
      const real sxy = mul_rn(ne, P.nz[3]), sxz = mul_rn(ne, P.nz[4]), syz = mul_rn(ne, P.nz[5]);
      txy = sub_rn(txy, sxy);
      tyx = sub_rn(tyx, sxy);
      txz = sub_rn(txz, sxz);
      tzx = sub_rn(tzx, sxz);
      tyz = sub_rn(tyz, syz);
      tzy = sub_rn(tzy, syz);
    }

    T[TXX * EXY + t] = txx;
    T[TYY * EXY + t] = tyy;
    T[TXY * EXY + t] = txy;
    T[TYX * EXY + t] = tyx;
    T[TZX * EXY + t] = tzx;
    T[TZY * EXY + t] = tzy;
    __syncthreads();

    if (out_here) {
      // U_s + dt dU/dt: the mass flux divergence times -dt/h, the summed
      // differences of the scaled fluxes times -dt/(4h)
      const real s_rho = add_rn(add_rn(sub_rn(P.gx, gx_xm), sub_rn(P.gy, gy_ym)), sub_rn(P.gz, gz_m));
      const real s_gx =
          add_rn(add_rn(sub_rn(T[TXX * EXY + eXp], txx), sub_rn(txy, T[TXY * EXY + eYm])), sub_rn(txz, txz_m));
      const real s_gy =
          add_rn(add_rn(sub_rn(T[TYY * EXY + eYp], tyy), sub_rn(tyx, T[TYX * EXY + eXm])), sub_rn(tyz, tyz_m));
      const real s_gz =
          add_rn(add_rn(sub_rn(tzz1, tzz_k), sub_rn(tzx, T[TZX * EXY + eXm])), sub_rn(tzy, T[TZY * EXY + eYm]));
      const uint32_t i = i_out;
      real o0 = fma_rn(s_rho, out_mass, P.dr), o1 = fma_rn(s_gx, out_flux, P.gx),
           o2 = fma_rn(s_gy, out_flux, P.gy), o3 = fma_rn(s_gz, out_flux, P.gz);
      if (STAGE != 0) {
        o0 = fma_rn(ca, un[0], mul_rn(cb, o0));
        o1 = fma_rn(ca, un[1], mul_rn(cb, o1));
        o2 = fma_rn(ca, un[2], mul_rn(cb, o2));
        o3 = fma_rn(ca, un[3], mul_rn(cb, o3));
      }
      a.o[0][i] = o0;
      a.o[1][i] = o1;
      a.o[2][i] = o2;
      a.o[3][i] = o3;
      if (STAGE == 2) mode_acc += o0 * cosw(k);
    }
    vz_m = P.vz;
    gz_m = P.gz;
    txz_m = txz;
    tyz_m = tyz;
    tzz_k = tzz1;
    P = Q;
    R = Rn;
  }
  }   // runs

  if (STAGE == 2) {
    // per-CTA partial of sum (rho - rho0) cos(k x), fixed reduction order
    const real v = warp_sum(mode_acc);
    __shared__ real s_red[32];
    const int lane = t & 31, wid = t >> 5;
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      const int nw = (EXY + 31) / 32;
      for (int j = 0; j < nw; ++j) s += double(s_red[j]);
      a.partials[blockIdx.x] = s;
    }
  }
}

// ------------------------------------------------------- FP32 pair kernel
// The FP32 form of the stage kernel for the wide tile: each thread marches two
// z planes at a time and holds every per-cell quantity as a pair {plane k,
// plane k+1}, so that shared memory moves 8-byte pairs and the barriers, the
// address arithmetic and the loop overhead are paid once per two planes; the
// next pair's loads are staged into shared memory with asynchronous copies
// while the current pair's fluxes are computed.  Quantities one plane up or
// down ("U" and "D" below) are pairs shifted by one element, assembled from
// the neighbouring pair or from values carried between iterations.  Each
// plane's values are the same sequence of rounded operations as in the scalar
// kernel, whichever element of a pair, CTA, run or kernel computes them, so
// every tiling gives the same bits.

__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }
// Pair arithmetic element by element with the scalar rounded intrinsics.
// (The packed FP32x2 intrinsics were measured no faster here, and the
// compiler fuses a packed multiply and add into one packed FMA even in their
// round-to-nearest forms, so their results would depend on the tiling.)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, -b.x), __fadd_rn(a.y, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 up2(float2 p, float q_x) { return make_float2(p.y, q_x); }     // {X(k+1), X(k+2)}
__device__ __forceinline__ float2 dn2(float carried, float2 p) { return make_float2(carried, p.x); }   // {X(k-1), X(k)}

// 4-byte asynchronous global -> shared copies (one per value, issued by the
// thread that later reads it back, so no barrier guards the staging slot)
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// staging slot of one plane pair: the thread's own values, [field][EXY]
enum StageField {
  SF_DR0, SF_DR1, SF_DR2, SF_DRX0, SF_DRX1, SF_DRY0, SF_DRY1, SF_GX0, SF_GX1, SF_GY0, SF_GY1, SF_GZ0, SF_GZ1,
  SF_PP0, SF_PP1, SF_NZ, kStageFields = SF_NZ + 12
};

// Row staging: per plane pair, each staged field-plane is copied as tile
// rows of TX + 8 floats (x from x0 - 4 to x0 + TX + 4, 16-byte aligned; a row
// that crosses the periodic seam is copied in two pieces), one thread per
// row, either by one or two TMA bulk copies (kStageBulk) or by 16-byte
// asynchronous copies (kStageRows16); an mbarrier tracks the pair.  Field-planes:
// delta rho at k, k+1, k+2 (TY + 3 rows: the thread rows and one above, for
// the y neighbour), then g_x, g_y, g_z, S Omega and the six stored normals at
// k, k+1 (TY + 2 rows each).
enum BulkField { BF_DR0, BF_DR1, BF_DR2, BF_GX0, BF_PP0 = BF_GX0 + 6, BF_NZ = BF_PP0 + 2, kBulkFields = BF_NZ + 12 };

template <int EY>
__host__ __device__ constexpr int bulk_row0(int fp) { return fp < 3 ? fp * (EY + 1) : 3 * (EY + 1) + (fp - 3) * EY; }
template <int TX, int TY>
__host__ __device__ constexpr int bulk_rows_max() { return bulk_row0<TY + 2>(kBulkFields); }

// Offset, from this thread's own element of the first row block, of the
// staged value that the per-thread staging slot keeps as field f.
template <int EY, int RP>
__device__ __forceinline__ constexpr int bulk_offset(int f) {
  return f == SF_DR0    ? 0
         : f == SF_DR1  ? bulk_row0<EY>(BF_DR1) * RP
         : f == SF_DR2  ? bulk_row0<EY>(BF_DR2) * RP
         : f == SF_DRX0 ? 1
         : f == SF_DRX1 ? bulk_row0<EY>(BF_DR1) * RP + 1
         : f == SF_DRY0 ? RP
         : f == SF_DRY1 ? (bulk_row0<EY>(BF_DR1) + 1) * RP
         : f <= SF_GZ1  ? bulk_row0<EY>(BF_GX0 + (f - SF_GX0)) * RP
         : f <= SF_PP1  ? bulk_row0<EY>(BF_PP0 + (f - SF_PP0)) * RP
                        : bulk_row0<EY>(BF_NZ + (f - SF_NZ)) * RP;
}

template <int TX, int TY, bool BULK>
constexpr size_t z2_smem_bytes() {
  constexpr int EXY = (TX + 2) * (TY + 2);
  return 18 * EXY * sizeof(float2) +
         (BULK ? size_t(bulk_rows_max<TX, TY>()) * (TX + 8) * sizeof(float) : kStageFields * EXY * sizeof(float));
}

// the finished values of a plane pair
struct Pair2 {
  float2 dr, gx, gy, gz, vx, vy, vz, pk;   // pk = c^2 delta rho + S Omega + p_ext
  float2 s[6];                              // Sigma: xx, yy, zz, xy, xz, yz
};

// resident CTAs per SM the register budget is sized for (a 34 x 10 tile: 1)
template <int EXY>
constexpr int z2_min_ctas() {
#ifdef IC_Z2_MIN_CTAS
  return IC_Z2_MIN_CTAS;
#else
  return (34 * (IC_FP32_TILE_Y + 2) + EXY - 1) / EXY;
#endif
}

// staging of the pair kernel's loads
enum { kStageThread = 0, kStageBulk = 1, kStageRows16 = 2 };

template <int TX, int TY, int STAGE, bool NOISE, int STG>
__global__ void __launch_bounds__((TX + 2) * (TY + 2), z2_min_ctas<(TX + 2) * (TY + 2)>())
    k_rk3_stage_z2(const StageArgs<float> a) {
  pdl_enter();
  constexpr int EX = TX + 2, EY = TY + 2, EXY = EX * EY, RP = TX + 8;
  constexpr bool BULK = STG != kStageThread;   // row layout, mbarrier
  static_assert(bulk_rows_max<TX, TY>() <= EXY, "one staged row per thread");
  enum { GX = 0, GY, GZ, VX, VY, VZ };
  enum { TXX = 0, TYY, TXY, TYX, TZX, TZY };
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);   // [2 slots][6 fields][EXY]
  float2 *T = sm + 12 * EXY;                            // [6 fluxes][EXY]
  float *stg = reinterpret_cast<float *>(T + 6 * EXY);  // [kStageFields][EXY], or the bulk rows
  const FluidConsts<float> &c = a.c;
  const int NX = c.nx, NY = c.ny, NZ = c.nz;
  const int t = threadIdx.x;
  const int ex = t % EX, ey = t / EX;
  const int eXm = ey * EX + max(ex - 1, 0), eXp = ey * EX + min(ex + 1, EX - 1);
  const int eYm = max(ey - 1, 0) * EX + ex, eYp = min(ey + 1, EY - 1) * EX + ex;
  // planes touched lie in [-2, NZ + 3): one compare-and-add wraps them (NZ >= 6)
  const auto zwrap = [NZ](int kk) { return kk < 0 ? kk + NZ : (kk >= NZ ? kk - NZ : kk); };

  const int64_t step = *a.step;
  const float drive4 = 4.0f * c.drive[STAGE];
  const float2 rho0 = splat2(c.rho0), half = splat2(0.5f), four = splat2(4.0f);
  const float2 c2x4 = splat2(c.c2x4), visc_d = splat2(c.visc_d), visc_o = splat2(c.visc_o);
  const float2 lam2x4_h = splat2(c.lam2x4_h), out_flux = splat2(c.out_flux), out_mass = splat2(c.out_mass);
  const float2 nd = splat2(c.noise_d4), nt = splat2(c.noise_t4), ne = splat2(c.noise_e4);
  const float beta = STAGE == 0 ? -1.7320508075688772f : (STAGE == 1 ? 1.7320508075688772f : 0.0f);
  const RngKey key{c.k0, c.k1, c.box};
  const uint32_t ustep = uint32_t(step);
  const float2 ca = splat2(float(kStageA[STAGE])), cb = splat2(float(kStageB[STAGE]));
  const uint32_t plane_n = uint32_t(NX) * uint32_t(NY);
  [[maybe_unused]] const size_t cells = size_t(plane_n) * size_t(NZ);
  float mode_acc = 0.0f;

  // Bulk staging: thread t < nrows copies one row of one field-plane per pair
  __shared__ __align__(8) unsigned long long s_bar;
  const uint32_t bar = smem_u32(&s_bar);
  uint32_t phase = 0;
  bool bad = false;
  int my_fp = -1, my_ry = 0;
  if (BULK) {
    const bool has_pp = a.pp != nullptr, has_nz = NOISE && STAGE != 0;
    const int nrows = 3 * (EY + 1) + EY * (6 + (has_pp ? 2 : 0) + (has_nz ? 12 : 0));
    if (t < 3 * (EY + 1)) {
      my_fp = t / (EY + 1);
      my_ry = t - my_fp * (EY + 1);
    } else if (t < nrows) {
      const int r = t - 3 * (EY + 1);
      my_fp = r / EY;
      my_ry = r - my_fp * EY;
      my_fp += BF_GX0;
      if (!has_pp && my_fp >= BF_PP0) my_fp += 2;
    }
    if (t == 0) mbar_init(bar, uint32_t(nrows + a.stall));
    __syncthreads();
  }
  const float *my_field = nullptr;
  int my_dz = 0;
  uint32_t my_dst = 0;
  if (BULK && my_fp >= 0) {
    my_field = my_fp < BF_GX0   ? a.s[0]
               : my_fp < BF_PP0 ? a.s[1 + (my_fp - BF_GX0) / 2]
               : my_fp < BF_NZ  ? a.pp
                                : a.noise_in[(my_fp - BF_NZ) / 2];
    my_dz = my_fp < BF_GX0 ? my_fp : ((my_fp - BF_GX0) & 1);
    my_dst = smem_u32(stg + (bulk_row0<EY>(my_fp) + my_ry) * RP);
  }
  // a bulk copy that did not land in time: flag it, give the copies in
  // flight another bounded wait, and leave the CTA (the decision is uniform)
  const auto staging_abort = [&]() {
    if (bad && a.status) atomicOr(a.status, kStatusStaging);
    if (STG == kStageRows16) cp_async_wait_all();
    (void)mbar_wait(bar, phase ^ 1);
  };

  const int units = a.ncols_x * a.ncols_y * NZ;
  const int u_end = int((long long)units * (blockIdx.x + 1) / gridDim.x);
  for (int u = int((long long)units * blockIdx.x / gridDim.x); u < u_end;) {
    const int col = u / NZ;
    const int z0 = u - col * NZ;
    const int z1 = min(NZ, z0 + (u_end - u));
    u += z1 - z0;
    const int gx_raw = (col % a.ncols_x) * TX + ex - 1;
    const int gy_raw = (col / a.ncols_x) * TY + ey - 1;
    const int x = wrap(gx_raw, NX), y = wrap(gy_raw, NY);
    const int xp = (x + 1 == NX) ? 0 : x + 1;
    const int yp = (y + 1 == NY) ? 0 : y + 1;
    const bool interior = ex >= 1 && ex <= TX && ey >= 1 && ey <= TY && gx_raw < NX && gy_raw < NY;
    const uint32_t o_c = uint32_t(x) + uint32_t(NX) * uint32_t(y);
    const uint32_t o_xp = uint32_t(xp) + uint32_t(NX) * uint32_t(y);
    const uint32_t o_yp = uint32_t(x) + uint32_t(NX) * uint32_t(yp);
    const float cos_xy = c.wave_axis < 2 ? c.cos_table[c.wave_axis == 0 ? x : y] : 0.0f;
    auto cosw = [&](int kk) -> float { return c.wave_axis < 2 ? cos_xy : c.cos_table[zwrap(kk)]; };
    auto profile = [&](int kk) -> float {
      if (c.forcing == IC_FORCE_MODE) return cosw(kk);
      if (c.forcing == IC_FORCE_PLANE) {
        const int coord = c.wave_axis == 0 ? x : (c.wave_axis == 1 ? y : zwrap(kk));
        return coord == c.plane_index ? 1.0f : 0.0f;
      }
      return 0.0f;
    };
    const auto stored = [&](int kk) { return interior && kk >= z0 && kk < z1; };

    // this thread's staged row in the run: its global row and the x pieces
    // (x0 - 4 .. x0 + TX + 4 wrapped; the second piece, if any, starts at x = 0)
    const float *row_src = nullptr;
    int seg_a_x = 0, seg_a_len = 0;
    if (BULK && my_fp >= 0) {
      row_src = my_field + size_t(wrap((col / a.ncols_x) * TY - 1 + my_ry, NY)) * size_t(NX);
      const int xs = (col % a.ncols_x) * TX - 4;
      seg_a_x = xs < 0 ? NX - 4 : xs;
      seg_a_len = xs < 0 ? 4 : min(RP, NX - xs);
    }

    // asynchronous loads of the planes kk, kk + 1 into this thread's staging slot
    auto issue2 = [&](int kk) {
      if constexpr (BULK) {
        if (row_src) {
          const float *src = row_src + size_t(zwrap(kk + my_dz)) * plane_n;
#ifdef IC_BOUNDS_CHECK
          {  // the row's pieces [x, x + len) and [0, RP - len) lie in the field; else copy from its start
            const size_t row0 = size_t(src - my_field);
            if (row0 + size_t(seg_a_x) + size_t(seg_a_len) > cells || row0 + size_t(RP - seg_a_len) > cells) {
              (void)IC_CHK(cells, cells);
              src = my_field;
              seg_a_x = 0;
            }
          }
#endif
          if constexpr (STG == kStageBulk) {
            mbar_arrive_expect_tx(bar, RP * sizeof(float));
            bulk_g2s(my_dst, src + seg_a_x, uint32_t(seg_a_len) * sizeof(float), bar);
            if (seg_a_len < RP)
              bulk_g2s(my_dst + uint32_t(seg_a_len) * sizeof(float), src, uint32_t(RP - seg_a_len) * sizeof(float),
                       bar);
          } else {
#pragma unroll
            for (int j = 0; j < RP / 4; ++j) {
              const int xo = 4 * j;
              cp_async16(my_dst + 16u * j, xo < seg_a_len ? src + seg_a_x + xo : src + (xo - seg_a_len));
            }
            cp_async_commit();
            cp_async_mbar_arrive(bar);
          }
        }
        return;
      }
      const uint32_t b0 = uint32_t(zwrap(kk)) * plane_n, b1 = uint32_t(zwrap(kk + 1)) * plane_n,
                     b2 = uint32_t(zwrap(kk + 2)) * plane_n;
      const float *S0 = a.s[0];
      cp_async4(stg + SF_DR0 * EXY + t, IC_AT(S0, o_c, b0, cells));
      cp_async4(stg + SF_DR1 * EXY + t, IC_AT(S0, o_c, b1, cells));
      cp_async4(stg + SF_DR2 * EXY + t, IC_AT(S0, o_c, b2, cells));
      cp_async4(stg + SF_DRX0 * EXY + t, IC_AT(S0, o_xp, b0, cells));
      cp_async4(stg + SF_DRX1 * EXY + t, IC_AT(S0, o_xp, b1, cells));
      cp_async4(stg + SF_DRY0 * EXY + t, IC_AT(S0, o_yp, b0, cells));
      cp_async4(stg + SF_DRY1 * EXY + t, IC_AT(S0, o_yp, b1, cells));
      cp_async4(stg + SF_GX0 * EXY + t, IC_AT(a.s[1], o_c, b0, cells));
      cp_async4(stg + SF_GX1 * EXY + t, IC_AT(a.s[1], o_c, b1, cells));
      cp_async4(stg + SF_GY0 * EXY + t, IC_AT(a.s[2], o_c, b0, cells));
      cp_async4(stg + SF_GY1 * EXY + t, IC_AT(a.s[2], o_c, b1, cells));
      cp_async4(stg + SF_GZ0 * EXY + t, IC_AT(a.s[3], o_c, b0, cells));
      cp_async4(stg + SF_GZ1 * EXY + t, IC_AT(a.s[3], o_c, b1, cells));
      if (a.pp) {
        cp_async4(stg + SF_PP0 * EXY + t, IC_AT(a.pp, o_c, b0, cells));
        cp_async4(stg + SF_PP1 * EXY + t, IC_AT(a.pp, o_c, b1, cells));
      }
      if (NOISE && STAGE != 0) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          cp_async4(stg + (SF_NZ + 2 * j) * EXY + t, IC_AT(a.noise_in[j], o_c, b0, cells));
          cp_async4(stg + (SF_NZ + 2 * j + 1) * EXY + t, IC_AT(a.noise_in[j], o_c, b1, cells));
        }
      }
      cp_async_commit();
    };
    // finished values of the planes kk, kk + 1 from the staged loads
    auto finish2 = [&](int kk) -> Pair2 {
      const uint32_t b0 = uint32_t(zwrap(kk)) * plane_n, b1 = uint32_t(zwrap(kk + 1)) * plane_n;
      const float *R = stg + ey * RP + ex + 3;   // bulk: own element of the first row block
      if constexpr (BULK) {
        if (!mbar_wait(bar, phase)) bad = true;
        phase ^= 1;
      } else {
        cp_async_wait_all();
      }
      auto ld = [&](int f) { return BULK ? R[bulk_offset<EY, RP>(f)] : stg[f * EXY + t]; };
      const float2 dr = make_float2(ld(SF_DR0), ld(SF_DR1));
      const float2 drx = make_float2(ld(SF_DRX0), ld(SF_DRX1));
      const float2 dry = make_float2(ld(SF_DRY0), ld(SF_DRY1));
      const float2 drz = make_float2(dr.y, ld(SF_DR2));
      Pair2 P;
      P.dr = dr;
      P.gx = make_float2(ld(SF_GX0), ld(SF_GX1));
      P.gy = make_float2(ld(SF_GY0), ld(SF_GY1));
      P.gz = make_float2(ld(SF_GZ0), ld(SF_GZ1));
      const float2 pp = a.pp ? make_float2(ld(SF_PP0), ld(SF_PP1)) : splat2(0.0f);
      const float2 rfx = fma2(half, add2(dr, drx), rho0);
      const float2 rfy = fma2(half, add2(dr, dry), rho0);
      const float2 rfz = fma2(half, add2(dr, drz), rho0);
      P.vx = make_float2(__fdividef(P.gx.x, rfx.x), __fdividef(P.gx.y, rfx.y));
      P.vy = make_float2(__fdividef(P.gy.x, rfy.x), __fdividef(P.gy.y, rfy.y));
      P.vz = make_float2(__fdividef(P.gz.x, rfz.x), __fdividef(P.gz.y, rfz.y));
      // 4 pi = 4 (c^2 delta rho + S Omega + p_ext)
      P.pk = add2(fma2(c2x4, dr, mul2(four, pp)), mul2(splat2(drive4), make_float2(profile(kk), profile(kk + 1))));
      if (NOISE) {
        float2 w[6];
        if (STAGE == 0) {
          // W_1 = W_A - sqrt3 W_B for this stage; the cell's own CTA stores W_2, W_3
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const uint32_t i = IC_CHK(o_c + (e == 0 ? b0 : b1), cells);
            float wa[6], wb[6];
            stress_normals_ab(key, i, ustep, wa, wb);
            const bool st = stored(kk + e);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
              const float v = fma_rn(beta, wb[j], wa[j]);
              if (e == 0) w[j].x = v; else w[j].y = v;
              if (st) {
                a.noise_out[j][i] = fma_rn(1.7320508075688772f, wb[j], wa[j]);
                a.noise_out[6 + j][i] = wa[j];
              }
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 6; ++j) w[j] = make_float2(ld(SF_NZ + 2 * j), ld(SF_NZ + 2 * j + 1));
        }
        const float2 tr = add2(add2(w[0], w[1]), w[2]);
        const float2 ntr = mul2(nt, tr);
        P.s[0] = fma2(nd, w[0], ntr);
        P.s[1] = fma2(nd, w[1], ntr);
        P.s[2] = fma2(nd, w[2], ntr);
        P.s[3] = mul2(ne, w[3]);
        P.s[4] = mul2(ne, w[4]);
        P.s[5] = mul2(ne, w[5]);
      }
      return P;
    };
    auto store_pair = [&](int slot, const Pair2 &v) {
      float2 *B = sm + slot * 6 * EXY;
      B[GX * EXY + t] = v.gx;
      B[GY * EXY + t] = v.gy;
      B[GZ * EXY + t] = v.gz;
      B[VX * EXY + t] = v.vx;
      B[VY * EXY + t] = v.vy;
      B[VZ * EXY + t] = v.vz;
    };

    __syncthreads();   // the previous run's last reads of shared memory are done
    // one pair below the run supplies the values carried into its first plane
    issue2(z0 - 2);
    Pair2 P = finish2(z0 - 2);
    // bulk rows are read by neighbours: all reads done before the slot is refilled
    if (BULK && __syncthreads_or(bad)) return staging_abort();
    issue2(z0);
    store_pair(0, P);
    float gz_m = 0.0f, txz_m = 0.0f, tyz_m = 0.0f, tzz_k = 0.0f, bulk_k = 0.0f;
    int slot = 0;
    for (int k = z0 - 2; k < z1; k += 2, slot ^= 1) {
      // U^n of the output planes
      const bool out0 = stored(k), out1 = stored(k + 1);
      const uint32_t i0 = IC_CHK(o_c + uint32_t(zwrap(k)) * plane_n, cells),
                     i1 = IC_CHK(o_c + uint32_t(zwrap(k + 1)) * plane_n, cells);
      float2 un[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        un[j] = splat2(0.0f);
        if (STAGE != 0) {
          if (out0) un[j].x = a.n[j][i0];
          if (out1) un[j].y = a.n[j][i1];
        }
      }
      const Pair2 Q = finish2(k + 2);
      if (!BULK && k + 2 < z1) issue2(k + 4);   // the next iteration's pair; overlaps this flux work
      store_pair(slot ^ 1, Q);
      if (BULK) {
        if (__syncthreads_or(bad)) return staging_abort();
        if (k + 2 < z1) issue2(k + 4);
      } else {
        __syncthreads();
      }
      const float2 *Ps = sm + slot * 6 * EXY;
      const float2 *Qs = sm + (slot ^ 1) * 6 * EXY;
      const float2 gx_xm = Ps[GX * EXY + eXm], vx_xm = Ps[VX * EXY + eXm];
      const float2 gy_ym = Ps[GY * EXY + eYm], vy_ym = Ps[VY * EXY + eYm];
      const float2 gx_yp = Ps[GX * EXY + eYp], vx_yp = Ps[VX * EXY + eYp];
      const float2 gy_xp = Ps[GY * EXY + eXp], vy_xp = Ps[VY * EXY + eXp];
      const float2 gz_xp = Ps[GZ * EXY + eXp], vz_xp = Ps[VZ * EXY + eXp];
      const float2 gz_yp = Ps[GZ * EXY + eYp], vz_yp = Ps[VZ * EXY + eYp];
      const float qvx_xm = Qs[VX * EXY + eXm].x, qvy_ym = Qs[VY * EXY + eYm].x;

      // pairs one plane up: {k+1, k+2}
      const float2 Uvx = up2(P.vx, Q.vx.x), Uvy = up2(P.vy, Q.vy.x), Uvz = up2(P.vz, Q.vz.x);
      const float2 Ugx = up2(P.gx, Q.gx.x), Ugy = up2(P.gy, Q.gy.x), Ugz = up2(P.gz, Q.gz.x);
      // h div v one plane up, and the bulk-viscous term 4 lam2 div v of both planes
      const float2 dsum_up = add2(add2(sub2(Uvx, up2(vx_xm, qvx_xm)), sub2(Uvy, up2(vy_ym, qvy_ym))),
                                  sub2(Uvz, P.vz));
      const float2 bulk_up = mul2(lam2x4_h, dsum_up);
      const float2 bulk = dn2(bulk_k, bulk_up);   // {plane k, plane k+1}

      // the fluxes times 4: products of two-point sums, pressure, minus 4 sigma
      float2 txx = add2(mul2(add2(gx_xm, P.gx), add2(vx_xm, P.vx)), P.pk);
      txx = sub2(txx, fma2(visc_d, sub2(P.vx, vx_xm), bulk));
      float2 tyy = add2(mul2(add2(gy_ym, P.gy), add2(vy_ym, P.vy)), P.pk);
      tyy = sub2(tyy, fma2(visc_d, sub2(P.vy, vy_ym), bulk));
      float2 tzz_up = add2(mul2(add2(P.gz, Ugz), add2(P.vz, Uvz)), up2(P.pk, Q.pk.x));
      tzz_up = sub2(tzz_up, fma2(visc_d, sub2(Uvz, P.vz), bulk_up));
      const float2 visc_xy = mul2(visc_o, add2(sub2(vx_yp, P.vx), sub2(vy_xp, P.vy)));
      float2 txy = sub2(mul2(add2(P.gx, gx_yp), add2(P.vy, vy_xp)), visc_xy);
      float2 tyx = sub2(mul2(add2(P.gy, gy_xp), add2(P.vx, vx_yp)), visc_xy);
      const float2 visc_xz = mul2(visc_o, add2(sub2(Uvx, P.vx), sub2(vz_xp, P.vz)));
      float2 txz = sub2(mul2(add2(P.gx, Ugx), add2(P.vz, vz_xp)), visc_xz);
      float2 tzx = sub2(mul2(add2(P.gz, gz_xp), add2(P.vx, Uvx)), visc_xz);
      const float2 visc_yz = mul2(visc_o, add2(sub2(Uvy, P.vy), sub2(vz_yp, P.vz)));
      float2 tyz = sub2(mul2(add2(P.gy, Ugy), add2(P.vz, vz_yp)), visc_yz);
      float2 tzy = sub2(mul2(add2(P.gz, gz_yp), add2(P.vy, Uvy)), visc_yz);
      if (NOISE) {
        txx = sub2(txx, P.s[0]);
        tyy = sub2(tyy, P.s[1]);
        tzz_up = sub2(tzz_up, up2(P.s[2], Q.s[2].x));
        txy = sub2(txy, P.s[3]);
        tyx = sub2(tyx, P.s[3]);
        txz = sub2(txz, P.s[4]);
        tzx = sub2(tzx, P.s[4]);
        tyz = sub2(tyz, P.s[5]);
        tzy = sub2(tzy, P.s[5]);
      }
      T[TXX * EXY + t] = txx;
      T[TYY * EXY + t] = tyy;
      T[TXY * EXY + t] = txy;
      T[TYX * EXY + t] = tyx;
      T[TZX * EXY + t] = tzx;
      T[TZY * EXY + t] = tzy;
      __syncthreads();

      if (out0 || out1) {
        // U_s + dt dU/dt: the mass flux divergence times -dt/h, the summed
        // differences of the scaled fluxes times -dt/(4h)
        const float2 s_rho = add2(add2(sub2(P.gx, gx_xm), sub2(P.gy, gy_ym)), sub2(P.gz, dn2(gz_m, P.gz)));
        const float2 s_gx = add2(add2(sub2(T[TXX * EXY + eXp], txx), sub2(txy, T[TXY * EXY + eYm])),
                                 sub2(txz, dn2(txz_m, txz)));
        const float2 s_gy = add2(add2(sub2(T[TYY * EXY + eYp], tyy), sub2(tyx, T[TYX * EXY + eXm])),
                                 sub2(tyz, dn2(tyz_m, tyz)));
        const float2 s_gz = add2(add2(sub2(tzz_up, dn2(tzz_k, tzz_up)), sub2(tzx, T[TZX * EXY + eXm])),
                                 sub2(tzy, T[TZY * EXY + eYm]));
        float2 o[4] = {fma2(s_rho, out_mass, P.dr), fma2(s_gx, out_flux, P.gx), fma2(s_gy, out_flux, P.gy),
                       fma2(s_gz, out_flux, P.gz)};
        if (STAGE != 0) {
#pragma unroll
          for (int j = 0; j < 4; ++j) o[j] = fma2(ca, un[j], mul2(cb, o[j]));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (out0) a.o[j][i0] = o[j].x;
          if (out1) a.o[j][i1] = o[j].y;
        }
        if (STAGE == 2) {
          if (out0) mode_acc = fmaf(o[0].x, cosw(k), mode_acc);
          if (out1) mode_acc = fmaf(o[0].y, cosw(k + 1), mode_acc);
        }
      }
      gz_m = P.gz.y;
      txz_m = txz.y;
      tyz_m = tyz.y;
      tzz_k = tzz_up.y;
      bulk_k = bulk_up.y;
      P = Q;
    }
  }

  if (STAGE == 2) {
    // per-CTA partial of sum (rho - rho0) cos(k x), fixed reduction order
    const float v = warp_sum(mode_acc);
    __shared__ float s_red[32];
    const int lane = t & 31, wid = t >> 5;
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      const int nw = (EXY + 31) / 32;
      for (int j = 0; j < nw; ++j) s += double(s_red[j]);
      a.partials[blockIdx.x] = s;
    }
  }
}

template <typename real>
FluidConsts<real> fluid_consts(const ic_ctx *ctx) {
  if constexpr (sizeof(real) == 4)
    return make_fluid_consts<float>(ctx->p, ctx->cos_table_f, ctx->drive_f);
  else
    return make_fluid_consts<double>(ctx->p, ctx->cos_table, ctx->drive);
}

// Tile shapes of the stage kernel: variant 0 is the wide tile tuned for large
// boxes; variant 1 is a 16 x 8 (FP32) or 16 x 4 (FP64) tile that boxes with
// edges of 16, 24, 32 or 48 cells fill exactly (the autotuner picks between
// them and the z chunk).
template <typename real, int V>
struct TileShape;
template <>
struct TileShape<float, 0> {
  static constexpr int TX = 32, TY = IC_FP32_TILE_Y;
};
template <>
struct TileShape<float, 1> {
  static constexpr int TX = 16, TY = 8;
};
template <>
struct TileShape<double, 0> {
  // 34 x 8 = 272 threads: nine warps a CTA at <= 227 registers (the stages
  // use 162-165), against six at 32 x 4, and a smaller ring share
  static constexpr int TX = 32, TY = 6;
};
template <>
struct TileShape<double, 1> {
  static constexpr int TX = 16, TY = 4;
};

// Fewest z planes a CTA marches: the grid is the CTAs the SMs hold at once
// (the register budget of the launch bounds) unless the box has fewer than
// IC_ZCHUNK planes per such CTA, so that a small box does not pay the 2.5D
// prologue (one extra plane per run) on runs of a few planes.
#ifndef IC_ZCHUNK
#define IC_ZCHUNK 32
#endif
int zchunk_for(const ic_ctx *ctx) { return std::min<int>(ctx->p.nz, ctx->zchunk > 0 ? ctx->zchunk : IC_ZCHUNK); }

struct StageLayout {
  int ncols_x, ncols_y, ctas;
};

// The pair kernel runs the wide FP32 tile; the scalar kernel the narrow FP32
// tile (small boxes, short runs) and FP64.  Both evaluate the same rounded
// operations per plane.
template <typename real, int TX>
constexpr bool use_pair_kernel() { return sizeof(real) == 4 && TX == 32; }

// CTAs per SM the launched stage kernel is budgeted for
template <typename real, int TX, int TY>
constexpr int stage_min_ctas() {
  if constexpr (use_pair_kernel<real, TX>()) return z2_min_ctas<(TX + 2) * (TY + 2)>();
  return min_ctas<real, (TX + 2) * (TY + 2)>();
}

// The bounded wait of the row staging under test: IC_STAGE_STALL_TEST=1 makes
// each CTA's mbarrier expect one arrival that no thread makes, so every wait
// runs out (about a second) and the launch reports IC_ERR_TIMEOUT.
int stage_stall_test() {
  const char *v = std::getenv("IC_STAGE_STALL_TEST");
  return v && v[0] == '1' ? 1 : 0;
}

// Bulk row staging needs 16-byte aligned rows: x extents a multiple of 4 of
// at least TX + 8 cells (so a row crosses the periodic seam at most once) and
// 16-byte aligned fields.
template <int TX, int STAGE, bool NOISE>
bool bulk_staging_ok(const StageArgs<float> &a) {
  const auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (a.c.nx % 4 != 0 || a.c.nx < TX + 8) return false;
  for (int j = 0; j < 4; ++j)
    if (!al(a.s[j])) return false;
  if (a.pp && !al(a.pp)) return false;
  if (NOISE && STAGE != 0)
    for (int j = 0; j < 6; ++j)
      if (!al(a.noise_in[j])) return false;
  return true;
}

template <int TX, int TY, int STAGE, bool NOISE, bool PRE = false, typename real>
void launch_stage_kernel(const StageArgs<real> &a, int ctas, cudaStream_t stream, int stage_copy) {
  constexpr int EXY = (TX + 2) * (TY + 2);
  if constexpr (use_pair_kernel<real, TX>()) {
    const int stg = stage_copy != kStageThread && bulk_staging_ok<TX, STAGE, NOISE>(a) ? stage_copy : kStageThread;
    const size_t smem = stg != kStageThread ? z2_smem_bytes<TX, TY, true>() : z2_smem_bytes<TX, TY, false>();
    auto kern = stg == kStageBulk     ? k_rk3_stage_z2<TX, TY, STAGE, NOISE, kStageBulk>
                : stg == kStageRows16 ? k_rk3_stage_z2<TX, TY, STAGE, NOISE, kStageRows16>
                                      : k_rk3_stage_z2<TX, TY, STAGE, NOISE, kStageThread>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    launch_k(kern, dim3(ctas), dim3(EXY), smem, stream, a);
  } else {
    const size_t smem = 18 * EXY * sizeof(real);
    auto kern = k_rk3_stage<real, TX, TY, STAGE, NOISE, PRE>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    launch_k(kern, dim3(ctas), dim3(EXY), smem, stream, a);
  }
}

template <typename real, int V>
StageLayout stage_layout_v(const ic_grid_params &p, int zchunk, int sm_count) {
  constexpr int TX = TileShape<real, V>::TX, TY = TileShape<real, V>::TY;
  StageLayout l;
  l.ncols_x = (p.nx + TX - 1) / TX;
  l.ncols_y = (p.ny + TY - 1) / TY;
  const long long units = (long long)l.ncols_x * l.ncols_y * p.nz;
  const long long resident = (long long)stage_min_ctas<real, TX, TY>() * sm_count;
  l.ctas = int(std::max<long long>(1, std::min<long long>(resident, (units + zchunk - 1) / zchunk)));
  return l;
}

template <typename real>
StageLayout stage_layout(const ic_ctx *ctx) {
  return ctx->tile_variant == 1 ? stage_layout_v<real, 1>(ctx->p, zchunk_for(ctx), ctx->sm_count)
                                : stage_layout_v<real, 0>(ctx->p, zchunk_for(ctx), ctx->sm_count);
}

template <typename real, int V, int STAGE, bool NOISE>
cudaError_t launch_stage_t(const ic_ctx *ctx, void *const in_s[4], void *const in_n[4],
                           void *const out[4]) {
  constexpr int TX = TileShape<real, V>::TX, TY = TileShape<real, V>::TY;
  StageArgs<real> a{};
  for (int j = 0; j < 4; ++j) {
    a.s[j] = static_cast<const real *>(in_s[j]);
    a.n[j] = static_cast<const real *>(in_n[j]);
    a.o[j] = static_cast<real *>(out[j]);
  }
  a.pp = ctx->ps.n > 0 ? static_cast<const real *>(ctx->pp) : nullptr;
  // FP64: the step's noise drawn once per cell by k_draw_noise, stage 1 reads W_1
  constexpr bool predraw = NOISE && sizeof(real) == 8;
  for (int j = 0; j < 12; ++j)
    a.noise_out[j] = STAGE == 0 && !predraw ? static_cast<real *>(ctx->noise[j]) : nullptr;
  for (int j = 0; j < 6; ++j)
    a.noise_in[j] = STAGE == 0 ? (predraw ? static_cast<const real *>(ctx->noise[12 + j]) : nullptr)
                               : static_cast<const real *>(ctx->noise[(STAGE == 1 ? 0 : 6) + j]);
  a.c = fluid_consts<real>(ctx);
  if (predraw && STAGE == 0) {
    NoiseOut<real> w;
    for (int j = 0; j < 18; ++j) w.p[j] = static_cast<real *>(ctx->noise[j]);
    const int blocks = std::max(1, std::min<int>(int((ctx->cells + 255) / 256), 8 * ctx->sm_count));
    const cudaError_t e = launch_k(k_draw_noise<real>, dim3(blocks), dim3(256), 0, ctx->stream,
                                   RngKey{a.c.k0, a.c.k1, a.c.box}, ctx->d.step, uint32_t(ctx->cells), w);
    if (e != cudaSuccess) return e;
  }
  a.step = ctx->d.step;
  a.partials = ctx->d.partials;
  a.status = ctx->d.status;
  a.stall = stage_stall_test();
  const StageLayout l = stage_layout_v<real, V>(ctx->p, zchunk_for(ctx), ctx->sm_count);
  a.ncols_x = l.ncols_x;
  a.ncols_y = l.ncols_y;
  launch_stage_kernel<TX, TY, STAGE, NOISE, predraw>(a, l.ctas, ctx->stream, ctx->stage_copy);
  return cudaGetLastError();
}

template <typename real, int V>
cudaError_t launch_stage_v(const ic_ctx *ctx, int stage, void *const in_s[4], void *const in_n[4],
                           void *const out[4]) {
  const bool noise = ctx->p.kT > 0.0;
  switch (stage * 2 + (noise ? 1 : 0)) {
    case 0: return launch_stage_t<real, V, 0, false>(ctx, in_s, in_n, out);
    case 1: return launch_stage_t<real, V, 0, true>(ctx, in_s, in_n, out);
    case 2: return launch_stage_t<real, V, 1, false>(ctx, in_s, in_n, out);
    case 3: return launch_stage_t<real, V, 1, true>(ctx, in_s, in_n, out);
    case 4: return launch_stage_t<real, V, 2, false>(ctx, in_s, in_n, out);
    default: return launch_stage_t<real, V, 2, true>(ctx, in_s, in_n, out);
  }
}

template <typename real>
cudaError_t launch_stage_r(const ic_ctx *ctx, int stage, void *const in_s[4], void *const in_n[4],
                           void *const out[4]) {
  if (ctx->tile_variant == 1) return launch_stage_v<real, 1>(ctx, stage, in_s, in_n, out);
  return launch_stage_v<real, 0>(ctx, stage, in_s, in_n, out);
}

// ------------------------------------------------------------ thermal state
// Two passes over the cells: partial sums of the fluctuations, then the
// update with the means removed (the normals are regenerated, not stored).
constexpr int kRedBlocks = 304;   // 2 x 152 SMs
constexpr int kRedThreads = 256;

__device__ void thermal_values(const RngKey &key, uint32_t cell, double sd_rho, double sd_g,
                               double out[4]) {
  const uint4 h = philox_block(key, cell, 0, kPurposeThermal, 0);
  const uint4 l = philox_block(key, cell, 0, kPurposeThermal, 1);
  double z[4];
  box_muller(uniform52(h.x, l.x), uniform52(h.y, l.y), z[0], z[1]);
  box_muller(uniform52(h.z, l.z), uniform52(h.w, l.w), z[2], z[3]);
  out[0] = sd_rho * z[0];
  out[1] = sd_g * z[1];
  out[2] = sd_g * z[2];
  out[3] = sd_g * z[3];
}

template <int NV>
__device__ void block_reduce_store(double v[NV], double *dst) {
  __shared__ double s[NV][kRedThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const double r = warp_sum(v[j]);
    if (lane == 0) s[j][wid] = r;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double acc = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) acc += s[threadIdx.x][w];
    dst[size_t(blockIdx.x) * NV + threadIdx.x] = acc;
  }
}

__global__ void k_thermal_sums(RngKey key, int64_t cells, double sd_rho, double sd_g, double *partials) {
  double acc[4] = {0, 0, 0, 0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < cells;
       i += int64_t(gridDim.x) * blockDim.x) {
    double v[4];
    thermal_values(key, uint32_t(i), sd_rho, sd_g, v);
    for (int j = 0; j < 4; ++j) acc[j] += v[j];
  }
  block_reduce_store<4>(acc, partials);
}

// final fixed-order reduction of nb blocks x nv values into out[nv] (one block)
__global__ void k_reduce_partials(const double *partials, int nb, int nv, double *out, double scale) {
  __shared__ double s[kRedThreads];
  for (int j = 0; j < nv; ++j) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partials[size_t(b) * nv + j];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = s[0] * scale;
    __syncthreads();
  }
}

template <typename real>
__global__ void k_thermal_apply(RngKey key, int64_t cells, double sd_rho, double sd_g,
                                const double *mean, int add, real *dr, real *gx, real *gy, real *gz) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < cells;
       i += int64_t(gridDim.x) * blockDim.x) {
    double v[4];
    thermal_values(key, uint32_t(i), sd_rho, sd_g, v);
    real *f[4] = {dr, gx, gy, gz};
    for (int j = 0; j < 4; ++j) {
      const double fl = v[j] - mean[j];
      f[j][i] = add ? real(double(f[j][i]) + fl) : real(fl);
    }
  }
}

// sums of g (3 components) and of delta rho cos(k x) over the grid
template <typename real>
__global__ void k_field_sums(int nx, int ny, int nz, int axis, const double *cos_table,
                             const real *dr, const real *gx, const real *gy, const real *gz,
                             double *partials) {
  const int64_t cells = int64_t(nx) * ny * nz;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < cells;
       i += int64_t(gridDim.x) * blockDim.x) {
    acc[0] += double(gx[i]);
    acc[1] += double(gy[i]);
    acc[2] += double(gz[i]);
    if (cos_table) {
      const int64_t x = i % nx, y = (i / nx) % ny, z = i / (int64_t(nx) * ny);
      acc[3] += double(dr[i]) * cos_table[axis == 0 ? x : (axis == 1 ? y : z)];
    }
  }
  block_reduce_store<4>(acc, partials);
}

// End of step: A(t) from the stage-3 partials, weighted accumulation, the
// non-finite check, the step counter and the drive amplitudes of the next
// step (one block).
__global__ void k_end_of_step(const EndArgs e) {
  pdl_enter();
  __shared__ double s[kRedThreads];
  end_of_step_cta(e, s);
}

}  // namespace

void drive_amplitudes(const ic_ctx *ctx, int64_t step, double out[3]) {
  const ic_grid_params &p = ctx->p;
  for (int s = 0; s < 3; ++s) {
    const double t = (double(step) + kStageTime[s]) * p.dt;
    out[s] = (p.wave_amp == 0.0 || p.forcing == IC_FORCE_NONE) ? 0.0
                                                                : ctx->force_amp * std::sin(ctx->omega * t + p.wave_phase);
  }
}

size_t fluid_num_partials(const ic_ctx *ctx) {
  // the most CTAs any tile variant and z chunk the tuner may choose can launch
  const int ty = std::min<int>(TileShape<float, 1>::TY, TileShape<double, 1>::TY);
  const size_t n = size_t((ctx->p.nx + 15) / 16) * ((ctx->p.ny + ty - 1) / ty) * ((ctx->p.nz + kMinZChunk - 1) / kMinZChunk);
  return std::max<size_t>(n, size_t(kRedBlocks) * 4);
}

bool set_stage_tile(ic_ctx *ctx, int variant, int zchunk) {
  if (variant < 0 || variant > 2 || (zchunk < kMinZChunk && zchunk < ctx->p.nz)) return false;
  if (variant >= kTileRows && !rows_eligible(ctx->p)) return false;
  ctx->tile_variant = variant;
  ctx->zchunk = std::min(zchunk, ctx->p.nz);
  return true;
}

int stage_copy_active(const ic_ctx *ctx) {
  if (ctx->p.precision != IC_FP32 || ctx->tile_variant != 0 || !ctx->stage_copy) return 0;
  if (ctx->p.nx % 4 != 0 || ctx->p.nx < TileShape<float, 0>::TX + 8) return 0;
  const auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  for (int b = 0; b < 3; ++b)
    for (int j = 0; j < 4; ++j)
      if (!al(ctx->U[b][j])) return 0;
  if (!al(ctx->pp)) return 0;
  for (int j = 0; j < 12; ++j)
    if (ctx->noise[j] && !al(ctx->noise[j])) return 0;
  return ctx->stage_copy;
}

bool rows_active(const ic_ctx *ctx) {
  return ctx->tile_variant == kTileRows && rows_eligible(ctx->p) && rows_buffers_aligned(ctx);
}

void stage_tile(const ic_ctx *ctx, int *tx, int *ty, int *zchunk) {
  if (rows_active(ctx)) {
    *tx = ctx->p.nx;
    rows_tile(ctx, ty);
    *zchunk = ctx->zchunk > 0 ? ctx->zchunk : kMinZChunk;
    return;
  }
  const bool f = ctx->p.precision == IC_FP32, v1 = ctx->tile_variant == 1;
  *tx = v1 ? 16 : 32;
  *ty = f ? (v1 ? TileShape<float, 1>::TY : TileShape<float, 0>::TY)
          : (v1 ? TileShape<double, 1>::TY : TileShape<double, 0>::TY);
  *zchunk = zchunk_for(ctx);
}

cudaError_t launch_stage(const ic_ctx *ctx, int stage, void *const in_s[4], void *const in_n[4],
                         void *const out[4]) {
  if (rows_active(ctx)) return launch_stage_rows(ctx, stage, in_s, in_n, out);
  if (ctx->p.precision == IC_FP32) return launch_stage_r<float>(ctx, stage, in_s, in_n, out);
  return launch_stage_r<double>(ctx, stage, in_s, in_n, out);
}

template <typename real>
cudaError_t launch_stage_raw_t(const ic_grid_params &p, const FluidConsts<real> &c, int stage,
                               const void *const in_s[4], const void *const in_n[4], void *const out[4],
                               void *const noise[12], const int64_t *step, double *partials,
                               cudaStream_t stream) {
  constexpr int TX = TileShape<real, 0>::TX, TY = TileShape<real, 0>::TY;
  StageArgs<real> a{};
  for (int j = 0; j < 4; ++j) {
    a.s[j] = static_cast<const real *>(in_s[j]);
    a.n[j] = static_cast<const real *>(in_n[j]);
    a.o[j] = static_cast<real *>(out[j]);
  }
  a.pp = nullptr;   // the allocation-free step draws stage 1's noise inline
  for (int j = 0; j < 12; ++j) a.noise_out[j] = stage == 0 ? static_cast<real *>(noise[j]) : nullptr;
  for (int j = 0; j < 6; ++j)
    a.noise_in[j] = stage == 0 ? nullptr : static_cast<const real *>(noise[(stage == 1 ? 0 : 6) + j]);
  a.c = c;
  a.step = step;
  a.partials = partials;
  a.status = nullptr;
  a.stall = 0;
  const StageLayout l = stage_layout_v<real, 0>(p, std::min<int>(p.nz, IC_ZCHUNK), 1 << 20);
  a.ncols_x = l.ncols_x;
  a.ncols_y = l.ncols_y;
  const bool noise_on = p.kT > 0.0;
  switch (stage * 2 + (noise_on ? 1 : 0)) {
    case 0: launch_stage_kernel<TX, TY, 0, false>(a, l.ctas, stream, kDefaultStageCopy); break;
    case 1: launch_stage_kernel<TX, TY, 0, true>(a, l.ctas, stream, kDefaultStageCopy); break;
    case 2: launch_stage_kernel<TX, TY, 1, false>(a, l.ctas, stream, kDefaultStageCopy); break;
    case 3: launch_stage_kernel<TX, TY, 1, true>(a, l.ctas, stream, kDefaultStageCopy); break;
    case 4: launch_stage_kernel<TX, TY, 2, false>(a, l.ctas, stream, kDefaultStageCopy); break;
    default: launch_stage_kernel<TX, TY, 2, true>(a, l.ctas, stream, kDefaultStageCopy); break;
  }
  return cudaGetLastError();
}

size_t stage_ctas_raw(const ic_grid_params &p) {
  const int zc = std::min<int>(p.nz, IC_ZCHUNK);
  return size_t(p.precision == IC_FP32 ? stage_layout_v<float, 0>(p, zc, 1 << 20).ctas
                                       : stage_layout_v<double, 0>(p, zc, 1 << 20).ctas);
}

cudaError_t launch_stage_raw(const ic_grid_params &p, const void *consts, int stage, const void *const in_s[4],
                             const void *const in_n[4], void *const out[4], void *const noise[12],
                             const int64_t *step, double *partials, cudaStream_t stream) {
  if (p.precision == IC_FP32)
    return launch_stage_raw_t<float>(p, *static_cast<const FluidConsts<float> *>(consts), stage, in_s, in_n, out,
                                     noise, step, partials, stream);
  return launch_stage_raw_t<double>(p, *static_cast<const FluidConsts<double> *>(consts), stage, in_s, in_n, out,
                                    noise, step, partials, stream);
}

cudaError_t launch_thermal(ic_ctx *ctx, uint64_t seed, int add) {
  const ic_grid_params &p = ctx->p;
  const RngKey key{uint32_t(seed & 0xffffffffull), uint32_t(seed >> 32), p.box};
  const double vol = p.h * p.h * p.h;
  const double sd_rho = std::sqrt(p.rho0 * p.kT / (p.c * p.c * vol));
  const double sd_g = std::sqrt(p.rho0 * p.kT / vol);
  double *mean = ctx->d.scalars + 4;   // scratch slots 4..7
  k_thermal_sums<<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(key, ctx->cells, sd_rho, sd_g, ctx->d.partials);
  k_reduce_partials<<<1, kRedThreads, 0, ctx->stream>>>(ctx->d.partials, kRedBlocks, 4, mean,
                                                        1.0 / double(ctx->cells));
  void *const *U = ctx->U[ctx->cur];
  if (p.precision == IC_FP32)
    k_thermal_apply<float><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(
        key, ctx->cells, sd_rho, sd_g, mean, add, (float *)U[0], (float *)U[1], (float *)U[2], (float *)U[3]);
  else
    k_thermal_apply<double><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(
        key, ctx->cells, sd_rho, sd_g, mean, add, (double *)U[0], (double *)U[1], (double *)U[2], (double *)U[3]);
  return cudaGetLastError();
}

cudaError_t launch_field_sums(ic_ctx *ctx, void *const U[4], double *dev_out4) {
  const ic_grid_params &p = ctx->p;
  const double *tab = ctx->cos_table;
  if (p.precision == IC_FP32)
    k_field_sums<float><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(
        p.nx, p.ny, p.nz, p.wave_axis, tab, (const float *)U[0], (const float *)U[1], (const float *)U[2],
        (const float *)U[3], ctx->d.partials);
  else
    k_field_sums<double><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(
        p.nx, p.ny, p.nz, p.wave_axis, tab, (const double *)U[0], (const double *)U[1],
        (const double *)U[2], (const double *)U[3], ctx->d.partials);
  k_reduce_partials<<<1, kRedThreads, 0, ctx->stream>>>(ctx->d.partials, kRedBlocks, 4, dev_out4, 1.0);
  return cudaGetLastError();
}

EndArgs end_args(const ic_ctx *ctx) {
  const int nb = rows_active(ctx)                ? rows_ctas(ctx, 2)
                 : ctx->p.precision == IC_FP32 ? stage_layout<float>(ctx).ctas
                                               : stage_layout<double>(ctx).ctas;
  const ic_grid_params &p = ctx->p;
  EndArgs e{};
  e.partials = ctx->d.partials;
  e.nb = nb;
  e.inv_cells = 1.0 / double(ctx->cells);
  e.has_mode = 1;
  e.step = ctx->d.step;
  e.weights = ctx->d.weights;
  e.scalars = ctx->d.scalars;
  e.status = ctx->d.status;
  e.amp = (p.wave_amp == 0.0 || p.forcing == IC_FORCE_NONE) ? 0.0 : ctx->force_amp;
  e.omega = ctx->omega;
  e.dt = p.dt;
  e.phase = p.wave_phase;
  e.drive = ctx->drive;
  e.drive_f = ctx->drive_f;
  return e;
}

cudaError_t launch_end_of_step(ic_ctx *ctx) {
  return launch_k(k_end_of_step, dim3(1), dim3(kRedThreads), 0, ctx->stream, end_args(ctx));
}

// An index equal to its extent passed to the check, no memory touched: the
// debug build's flag must rise.
__global__ void k_bounds_probe(int n) { (void)IC_CHK(n, n); }

cudaError_t launch_bounds_probe(cudaStream_t stream) {
  k_bounds_probe<<<1, 1, 0, stream>>>(7);
  return cudaGetLastError();
}

IC_BOUNDS_READER(bounds_flag_fluid)

}  // namespace ic
