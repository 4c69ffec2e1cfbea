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
// State stores delta rho = rho - rho0.
//
// Schedule.  The (column, plane) pairs are numbered column by column and split
// into gridDim.x equal contiguous ranges, one per CTA; a range that crosses a
// column boundary is marched as two runs.  With the grid sized to the CTAs the
// SMs hold at once, every CTA gets the same number of planes, so no partial
// last wave is left (a grid of fixed z chunks leaves one at most sizes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

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
  const real *__restrict__ noise_in[6];   // stages 2-3: stored W_s (xx, yy, zz, xy, xz, yz)
  real *__restrict__ noise_out[12];       // stage 1: stores W_2 = W_A + sqrt3 W_B and W_3 = W_A
  FluidConsts<real> c;
  const int64_t *step;
  double *partials;                // stage 3: per-CTA sum of delta rho cos(k x)
  int ncols_x, ncols_y;            // tile columns along x and y
};

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

// Tile shape and register budget of the FP32 stage kernel (tuned on GB300).
#ifndef IC_FP32_TILE_Y
#define IC_FP32_TILE_Y 8
#endif
#ifndef IC_FP32_MIN_CTAS
#define IC_FP32_MIN_CTAS 2
#endif

// CTAs per SM the register budget is sized for: in FP32 the budget of
// IC_FP32_MIN_CTAS wide (34 x (TY + 2)-thread) CTAs, whatever the tile
template <typename real, int EXY>
constexpr int min_ctas() {
  return sizeof(real) == 4 ? (IC_FP32_MIN_CTAS * 34 * (IC_FP32_TILE_Y + 2) + EXY - 1) / EXY : 1;
}

template <typename real, int TX, int TY, int STAGE, bool NOISE>
__global__ void __launch_bounds__((TX + 2) * (TY + 2), min_ctas<real, (TX + 2) * (TY + 2)>())
    k_rk3_stage(const StageArgs<real> a) {
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
  const real drive = c.drive[STAGE];
  const real rho0 = c.rho0, half = real(0.5), quarter = real(0.25);
  const real inv_h = c.inv_h, c2 = c.c2, eta = c.eta, lam2 = c.lam2;
  const real two_eta = real(2) * eta;
  const real nd = c.noise_diag, nt = c.noise_trace, ne = c.noise_edge;
  const real beta = STAGE == 0 ? real(-1.7320508075688772) : (STAGE == 1 ? real(1.7320508075688772) : real(0));
  const RngKey key{c.k0, c.k1, c.box};
  const uint32_t ustep = uint32_t(step);
  const real ca = real(kStageA[STAGE]), cb = real(kStageB[STAGE]);
  const real dt = c.dt;
  const uint32_t plane_n = uint32_t(NX) * uint32_t(NY);
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
  auto cell_of = [&](int kk) { return o_c + uint32_t(zwrap(kk)) * plane_n; };
  auto fetch = [&](int kk) {
    PlaneRaw<real> r;
    const int k = zwrap(kk);
    const uint32_t kb = uint32_t(k) * plane_n;
    const uint32_t kpb = (k + 1 == NZ) ? 0u : kb + plane_n;
    const uint32_t i = o_c + kb;
    r.dr = a.s[0][i];
    r.drx = a.s[0][o_xp + kb];
    r.dry = a.s[0][o_yp + kb];
    r.drz = a.s[0][o_c + kpb];
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
    if (NOISE && STAGE == 0) {
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

    const real div_k = ((P.vx - vx_xm) + (P.vy - vy_ym) + (P.vz - vz_m)) * inv_h;
    const real div_k1 = ((Q.vx - vx1_xm) + (Q.vy - vy1_ym) + (Q.vz - P.vz)) * inv_h;
    const real pk = c2 * P.dr + P.pp + drive * profile(k);
    const real pk1 = c2 * Q.dr + Q.pp + drive * profile(k + 1);

    const real tr_k = P.nz[0] + P.nz[1] + P.nz[2];
    const real tr_k1 = Q.nz[0] + Q.nz[1] + Q.nz[2];
    const real sxx = nd * P.nz[0] + nt * tr_k;
    const real syy = nd * P.nz[1] + nt * tr_k;
    const real szz1 = nd * Q.nz[2] + nt * tr_k1;
    const real sxy = ne * P.nz[3], sxz = ne * P.nz[4], syz = ne * P.nz[5];

    const real txx = quarter * (gx_xm + P.gx) * (vx_xm + P.vx) + pk -
                     (two_eta * (P.vx - vx_xm) * inv_h + lam2 * div_k) - sxx;
    const real tyy = quarter * (gy_ym + P.gy) * (vy_ym + P.vy) + pk -
                     (two_eta * (P.vy - vy_ym) * inv_h + lam2 * div_k) - syy;
    const real tzz1 = quarter * (P.gz + Q.gz) * (P.vz + Q.vz) + pk1 -
                      (two_eta * (Q.vz - P.vz) * inv_h + lam2 * div_k1) - szz1;
    const real visc_xy = eta * ((vx_yp - P.vx) + (vy_xp - P.vy)) * inv_h;
    const real txy = quarter * (P.gx + gx_yp) * (P.vy + vy_xp) - visc_xy - sxy;
    const real tyx = quarter * (P.gy + gy_xp) * (P.vx + vx_yp) - visc_xy - sxy;
    const real visc_xz = eta * ((Q.vx - P.vx) + (vz_xp - P.vz)) * inv_h;
    const real txz = quarter * (P.gx + Q.gx) * (P.vz + vz_xp) - visc_xz - sxz;
    const real tzx = quarter * (P.gz + gz_xp) * (P.vx + Q.vx) - visc_xz - sxz;
    const real visc_yz = eta * ((Q.vy - P.vy) + (vz_yp - P.vz)) * inv_h;
    const real tyz = quarter * (P.gy + Q.gy) * (P.vz + vz_yp) - visc_yz - syz;
    const real tzy = quarter * (P.gz + gz_yp) * (P.vy + Q.vy) - visc_yz - syz;

    T[TXX * EXY + t] = txx;
    T[TYY * EXY + t] = tyy;
    T[TXY * EXY + t] = txy;
    T[TYX * EXY + t] = tyx;
    T[TZX * EXY + t] = tzx;
    T[TZY * EXY + t] = tzy;
    __syncthreads();

    if (out_here) {
      const real r_rho = -((P.gx - gx_xm) + (P.gy - gy_ym) + (P.gz - gz_m)) * inv_h;
      const real r_gx = -((T[TXX * EXY + eXp] - txx) + (txy - T[TXY * EXY + eYm]) + (txz - txz_m)) * inv_h;
      const real r_gy = -((T[TYY * EXY + eYp] - tyy) + (tyx - T[TYX * EXY + eXm]) + (tyz - tyz_m)) * inv_h;
      const real r_gz = -((tzz1 - tzz_k) + (tzx - T[TZX * EXY + eXm]) + (tzy - T[TZY * EXY + eYm])) * inv_h;
      const uint32_t i = i_out;
      real o0 = P.dr + dt * r_rho, o1 = P.gx + dt * r_gx, o2 = P.gy + dt * r_gy, o3 = P.gz + dt * r_gz;
      if (STAGE != 0) {
        o0 = ca * un[0] + cb * o0;
        o1 = ca * un[1] + cb * o1;
        o2 = ca * un[2] + cb * o2;
        o3 = ca * un[3] + cb * o3;
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

template <typename real>
FluidConsts<real> fluid_consts(const ic_ctx *ctx) {
  const ic_grid_params &p = ctx->p;
  FluidConsts<real> c{};
  c.nx = p.nx;
  c.ny = p.ny;
  c.nz = p.nz;
  c.rho0 = real(p.rho0);
  c.c2 = real(p.c * p.c);
  c.inv_h = real(1.0 / p.h);
  c.dt = real(p.dt);
  c.eta = real(p.eta);
  c.lam2 = real(p.zeta - 2.0 * p.eta / 3.0);
  const double vol_dt = p.h * p.h * p.h * p.dt;
  const double S = std::sqrt(2.0 * p.eta * p.kT / vol_dt);
  const double B = std::sqrt(p.zeta * p.kT / (3.0 * vol_dt));
  c.noise_diag = real(std::sqrt(2.0) * S);
  c.noise_trace = real(std::sqrt(2.0) * (B - S / 3.0));
  c.noise_edge = real(S);
  c.forcing = (p.wave_amp == 0.0) ? IC_FORCE_NONE : p.forcing;
  c.wave_axis = p.wave_axis;
  c.plane_index = p.plane_index;
  if constexpr (sizeof(real) == 4) {
    c.cos_table = ctx->cos_table_f;
    c.drive = ctx->drive_f;
  } else {
    c.cos_table = ctx->cos_table;
    c.drive = ctx->drive;
  }
  c.k0 = uint32_t(p.seed & 0xffffffffull);
  c.k1 = uint32_t(p.seed >> 32);
  c.box = p.box;
  c.noise = p.kT > 0.0;
  return c;
}

// Tile shapes of the stage kernel: variant 0 is the wide tile tuned for large
// boxes; variant 1 halves the x extent so that 16- and 48-cell boxes fill
// their tiles (the autotuner picks between them and the z chunk).
template <typename real, int V>
struct TileShape;
template <>
struct TileShape<float, 0> {
  static constexpr int TX = 32, TY = IC_FP32_TILE_Y;
};
template <>
struct TileShape<float, 1> {
  static constexpr int TX = 16, TY = IC_FP32_TILE_Y;
};
template <>
struct TileShape<double, 0> {
  static constexpr int TX = 32, TY = 4;
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

template <typename real, int V>
StageLayout stage_layout_v(const ic_grid_params &p, int zchunk, int sm_count) {
  constexpr int TX = TileShape<real, V>::TX, TY = TileShape<real, V>::TY;
  constexpr int EXY = (TX + 2) * (TY + 2);
  StageLayout l;
  l.ncols_x = (p.nx + TX - 1) / TX;
  l.ncols_y = (p.ny + TY - 1) / TY;
  const long long units = (long long)l.ncols_x * l.ncols_y * p.nz;
  const long long resident = (long long)min_ctas<real, EXY>() * sm_count;
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
  constexpr int EXY = (TX + 2) * (TY + 2);
  StageArgs<real> a;
  for (int j = 0; j < 4; ++j) {
    a.s[j] = static_cast<const real *>(in_s[j]);
    a.n[j] = static_cast<const real *>(in_n[j]);
    a.o[j] = static_cast<real *>(out[j]);
  }
  a.pp = ctx->ps.n > 0 ? static_cast<const real *>(ctx->pp) : nullptr;
  for (int j = 0; j < 12; ++j) a.noise_out[j] = STAGE == 0 ? static_cast<real *>(ctx->noise[j]) : nullptr;
  for (int j = 0; j < 6; ++j)
    a.noise_in[j] = STAGE == 0 ? nullptr : static_cast<const real *>(ctx->noise[(STAGE == 1 ? 0 : 6) + j]);
  a.c = fluid_consts<real>(ctx);
  a.step = ctx->d.step;
  a.partials = ctx->d.partials;
  const StageLayout l = stage_layout_v<real, V>(ctx->p, zchunk_for(ctx), ctx->sm_count);
  a.ncols_x = l.ncols_x;
  a.ncols_y = l.ncols_y;
  const size_t smem = 18 * EXY * sizeof(real);
  auto kern = k_rk3_stage<real, TX, TY, STAGE, NOISE>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  kern<<<l.ctas, EXY, smem, ctx->stream>>>(a);
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
__global__ void k_end_of_step(const double *partials, int nb, double inv_cells, int has_mode,
                              int64_t *step, const double *weights, double *scalars, int *status,
                              double amp, double omega, double dt, double phase, double *drive, float *drive_f) {
  __shared__ double s[kRedThreads];
  const int64_t n0 = step[0];   // read by every thread before thread 0 advances it
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partials[b];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double A = has_mode ? 2.0 * s[0] * inv_cells : 0.0;
    const int64_t j = n0 - step[1];
    const double w = (j >= 0 && j < step[2]) ? weights[j] : 0.0;
    if (!isfinite(s[0])) atomicOr(status, kStatusNonfinite);
    scalars[0] += w;
    scalars[1] += w * A * A;
    scalars[2] = A;
    step[0] = n0 + 1;
  }
  if (threadIdx.x < 3) {
    // drive amplitudes of the RK stages of the next step (t^n, t^{n+1}, t^{n+1/2})
    const double frac = threadIdx.x == 0 ? 0.0 : (threadIdx.x == 1 ? 1.0 : 0.5);
    const double t = (double(n0 + 1) + frac) * dt;
    const double d = amp * sin(omega * t + phase);
    drive[threadIdx.x] = d;
    drive_f[threadIdx.x] = float(d);
  }
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
  if (variant < 0 || variant > 1 || (zchunk < kMinZChunk && zchunk < ctx->p.nz)) return false;
  ctx->tile_variant = variant;
  ctx->zchunk = std::min(zchunk, ctx->p.nz);
  return true;
}

void stage_tile(const ic_ctx *ctx, int *tx, int *ty, int *zchunk) {
  const bool f = ctx->p.precision == IC_FP32, v1 = ctx->tile_variant == 1;
  *tx = v1 ? 16 : 32;
  *ty = f ? TileShape<float, 0>::TY : TileShape<double, 0>::TY;
  *zchunk = zchunk_for(ctx);
}

cudaError_t launch_stage(const ic_ctx *ctx, int stage, void *const in_s[4], void *const in_n[4],
                         void *const out[4]) {
  if (ctx->p.precision == IC_FP32) return launch_stage_r<float>(ctx, stage, in_s, in_n, out);
  return launch_stage_r<double>(ctx, stage, in_s, in_n, out);
}

template <typename real>
cudaError_t launch_stage_raw_t(const ic_grid_params &p, const FluidConsts<real> &c, int stage,
                               const void *const in_s[4], const void *const in_n[4], void *const out[4],
                               void *const noise[12], const int64_t *step, double *partials,
                               cudaStream_t stream) {
  constexpr int TX = TileShape<real, 0>::TX, TY = TileShape<real, 0>::TY;
  constexpr int EXY = (TX + 2) * (TY + 2);
  StageArgs<real> a;
  for (int j = 0; j < 4; ++j) {
    a.s[j] = static_cast<const real *>(in_s[j]);
    a.n[j] = static_cast<const real *>(in_n[j]);
    a.o[j] = static_cast<real *>(out[j]);
  }
  a.pp = nullptr;
  for (int j = 0; j < 12; ++j) a.noise_out[j] = stage == 0 ? static_cast<real *>(noise[j]) : nullptr;
  for (int j = 0; j < 6; ++j)
    a.noise_in[j] = stage == 0 ? nullptr : static_cast<const real *>(noise[(stage == 1 ? 0 : 6) + j]);
  a.c = c;
  a.step = step;
  a.partials = partials;
  const StageLayout l = stage_layout_v<real, 0>(p, std::min<int>(p.nz, IC_ZCHUNK), 1 << 20);
  a.ncols_x = l.ncols_x;
  a.ncols_y = l.ncols_y;
  const dim3 grid(l.ctas);
  const size_t smem = 18 * EXY * sizeof(real);
  const bool noise_on = p.kT > 0.0;
  switch (stage * 2 + (noise_on ? 1 : 0)) {
#define IC_RAW(S, N)                                                                       \
  {                                                                                        \
    auto kern = k_rk3_stage<real, TX, TY, S, N>;                                            \
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)); \
    kern<<<grid, EXY, smem, stream>>>(a);                                                   \
  } break;
    case 0: IC_RAW(0, false)
    case 1: IC_RAW(0, true)
    case 2: IC_RAW(1, false)
    case 3: IC_RAW(1, true)
    case 4: IC_RAW(2, false)
    default: IC_RAW(2, true)
#undef IC_RAW
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

cudaError_t launch_end_of_step(ic_ctx *ctx) {
  const int nb = ctx->p.precision == IC_FP32 ? stage_layout<float>(ctx).ctas : stage_layout<double>(ctx).ctas;
  const int has_mode = 1;
  const ic_grid_params &p = ctx->p;
  const double amp = (p.wave_amp == 0.0 || p.forcing == IC_FORCE_NONE) ? 0.0 : ctx->force_amp;
  k_end_of_step<<<1, kRedThreads, 0, ctx->stream>>>(ctx->d.partials, nb, 1.0 / double(ctx->cells), has_mode,
                                                    ctx->d.step, ctx->d.weights, ctx->d.scalars, ctx->d.status,
                                                    amp, ctx->omega, p.dt, p.wave_phase, ctx->drive, ctx->drive_f);
  return cudaGetLastError();
}

}  // namespace ic
