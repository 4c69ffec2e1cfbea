// Device-side building blocks of libic: the counter-based generator, the
// normal transform, the 3-point kernel weights and periodic index helpers.
//
// Random numbers.  The stochastic stress (Sec. 4.2) is drawn per cell and per
// step from Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11) with
//   key     = (seed & 0xffffffff, seed >> 32)
//   counter = (cell, step, (purpose << 16) | block, box).
// For purpose 0 the 6 blocks give 24 words per cell and step; normal j
// (j = 0..5: W_A components xx, yy, zz, xy, xz, yz; j = 6..11: W_B) takes its
// high word from word j and its low word from word 12 + j.  Normals come in
// Box-Muller pairs: (n_2i, n_2i+1) = r (cos 2 pi u_2i+1, sin 2 pi u_2i+1),
// r = sqrt(-2 ln u_2i).  The FP64 path builds 52-bit uniforms
// u = (2 m + 1) 2^-53, m = (hi << 20) | (lo >> 12); the FP32 path uses the
// high words alone (radius uniform (hi + 1/2) 2^-32, angle uniform from the
// top 23 bits), so its normals follow the FP64 ones to about 1e-6 and need
// only blocks 0-2.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ic {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kPurposeStress = 0u;
constexpr uint32_t kPurposeThermal = 1u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one widening multiply gives both halves of each 64-bit product
    const uint64_t p0 = uint64_t(kPhiloxM0) * c.x;
    const uint64_t p1 = uint64_t(kPhiloxM1) * c.z;
    c = make_uint4(uint32_t(p1 >> 32) ^ c.y ^ k0, uint32_t(p1), uint32_t(p0 >> 32) ^ c.w ^ k1, uint32_t(p0));
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

struct RngKey {
  uint32_t k0, k1, box;
};

// The ten round keys of a Philox4x32-10 key (k0 + r W0, k1 + r W1), computed
// once on the host: a kernel that draws many blocks with one key reads them
// as constants instead of stepping the key schedule per block.
struct RoundKeys {
  uint32_t k[20];
};

inline RoundKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  RoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0 + uint32_t(r) * kPhiloxW0;
    rk.k[2 * r + 1] = k1 + uint32_t(r) * kPhiloxW1;
  }
  return rk;
}

// Philox4x32-10 with precomputed round keys (the same function as philox4x32_10)
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = uint64_t(kPhiloxM0) * c.x;
    const uint64_t p1 = uint64_t(kPhiloxM1) * c.z;
    c = make_uint4(uint32_t(p1 >> 32) ^ c.y ^ rk.k[2 * r], uint32_t(p1), uint32_t(p0 >> 32) ^ c.w ^ rk.k[2 * r + 1],
                   uint32_t(p0));
  }
  return c;
}

// W_A and W_B of one cell and step in FP32 (the normals of stress_normals_ab)
// from precomputed round keys
__device__ __forceinline__ void stress_normals_ab_rk(const RoundKeys &rk, uint32_t box, uint32_t cell, uint32_t step,
                                                     float a[6], float b[6]);

__device__ __forceinline__ uint4 philox_block(const RngKey &key, uint32_t cell, uint32_t step,
                                              uint32_t purpose, uint32_t block) {
  return philox4x32_10(make_uint4(cell, step, (purpose << 16) | block, key.box), key.k0, key.k1);
}

__device__ __forceinline__ double uniform52(uint32_t hi, uint32_t lo) {
  const uint64_t m = (uint64_t(hi) << 20) | uint64_t(lo >> 12);
  return double(2ull * m + 1ull) * 0x1p-53;
}

__device__ __forceinline__ void box_muller(double u1, double u2, double &z0, double &z1) {
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincos(2.0 * 3.141592653589793 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

__device__ __forceinline__ void box_muller_f32(uint32_t h1, uint32_t h2, float &z0, float &z1) {
  // radius uniform u1 = (h1 + 1/2) 2^-32 resolved down to 2^-33 (tails to 6.8 sigma)
  const float u1 = __fmaf_rn(__uint2float_rn(h1), 0x1p-32f, 0x1p-33f);
  // angle uniform from the top 23 bits: t = u2 - 1/2 in [-1/2, 1/2)
  const float t = __uint_as_float(0x3f800000u | (h2 >> 9)) - 1.5f;
  const float x = fmaxf(-2.0f * __logf(u1), 1e-30f);
  const float r = x * rsqrtf(x);
  float s, c;
  __sincosf(6.2831853071795865f * t, &s, &c);   // 2 pi u2 = 2 pi t + pi
  z0 = -r * c;
  z1 = -r * s;
}

// The six combined normals W_A + beta W_B of one cell and step, ordered
// xx, yy, zz, xy, xz, yz.  with_b = false skips stream B (beta = 0).
__device__ __forceinline__ void stress_normals(const RngKey &key, uint32_t cell, uint32_t step,
                                               bool with_b, double beta, double out[6]) {
  const uint4 h0 = philox_block(key, cell, step, kPurposeStress, 0);
  const uint4 h1 = philox_block(key, cell, step, kPurposeStress, 1);
  const uint4 l0 = philox_block(key, cell, step, kPurposeStress, 3);
  const uint4 l1 = philox_block(key, cell, step, kPurposeStress, 4);
  double a[6];
  box_muller(uniform52(h0.x, l0.x), uniform52(h0.y, l0.y), a[0], a[1]);
  box_muller(uniform52(h0.z, l0.z), uniform52(h0.w, l0.w), a[2], a[3]);
  box_muller(uniform52(h1.x, l1.x), uniform52(h1.y, l1.y), a[4], a[5]);
  if (with_b) {
    const uint4 h2 = philox_block(key, cell, step, kPurposeStress, 2);
    const uint4 l2 = philox_block(key, cell, step, kPurposeStress, 5);
    double b[6];
    box_muller(uniform52(h1.z, l1.z), uniform52(h1.w, l1.w), b[0], b[1]);
    box_muller(uniform52(h2.x, l2.x), uniform52(h2.y, l2.y), b[2], b[3]);
    box_muller(uniform52(h2.z, l2.z), uniform52(h2.w, l2.w), b[4], b[5]);
#pragma unroll
    for (int j = 0; j < 6; ++j) out[j] = a[j] + beta * b[j];
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) out[j] = a[j];
  }
}

__device__ __forceinline__ void stress_normals(const RngKey &key, uint32_t cell, uint32_t step,
                                               bool with_b, float beta, float out[6]) {
  const uint4 h0 = philox_block(key, cell, step, kPurposeStress, 0);
  const uint4 h1 = philox_block(key, cell, step, kPurposeStress, 1);
  float a[6];
  box_muller_f32(h0.x, h0.y, a[0], a[1]);
  box_muller_f32(h0.z, h0.w, a[2], a[3]);
  box_muller_f32(h1.x, h1.y, a[4], a[5]);
  if (with_b) {
    const uint4 h2 = philox_block(key, cell, step, kPurposeStress, 2);
    float b[6];
    box_muller_f32(h1.z, h1.w, b[0], b[1]);
    box_muller_f32(h2.x, h2.y, b[2], b[3]);
    box_muller_f32(h2.z, h2.w, b[4], b[5]);
#pragma unroll
    for (int j = 0; j < 6; ++j) out[j] = __fmaf_rn(beta, b[j], a[j]);
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) out[j] = a[j];
  }
}

// Both streams of one cell and step, uncombined: W_A and W_B, each ordered
// xx, yy, zz, xy, xz, yz.
__device__ __forceinline__ void stress_normals_ab(const RngKey &key, uint32_t cell, uint32_t step, double a[6],
                                                  double b[6]) {
  const uint4 h0 = philox_block(key, cell, step, kPurposeStress, 0);
  const uint4 h1 = philox_block(key, cell, step, kPurposeStress, 1);
  const uint4 h2 = philox_block(key, cell, step, kPurposeStress, 2);
  const uint4 l0 = philox_block(key, cell, step, kPurposeStress, 3);
  const uint4 l1 = philox_block(key, cell, step, kPurposeStress, 4);
  const uint4 l2 = philox_block(key, cell, step, kPurposeStress, 5);
  box_muller(uniform52(h0.x, l0.x), uniform52(h0.y, l0.y), a[0], a[1]);
  box_muller(uniform52(h0.z, l0.z), uniform52(h0.w, l0.w), a[2], a[3]);
  box_muller(uniform52(h1.x, l1.x), uniform52(h1.y, l1.y), a[4], a[5]);
  box_muller(uniform52(h1.z, l1.z), uniform52(h1.w, l1.w), b[0], b[1]);
  box_muller(uniform52(h2.x, l2.x), uniform52(h2.y, l2.y), b[2], b[3]);
  box_muller(uniform52(h2.z, l2.z), uniform52(h2.w, l2.w), b[4], b[5]);
}

__device__ __forceinline__ void stress_normals_ab(const RngKey &key, uint32_t cell, uint32_t step, float a[6],
                                                  float b[6]) {
  const uint4 h0 = philox_block(key, cell, step, kPurposeStress, 0);
  const uint4 h1 = philox_block(key, cell, step, kPurposeStress, 1);
  const uint4 h2 = philox_block(key, cell, step, kPurposeStress, 2);
  box_muller_f32(h0.x, h0.y, a[0], a[1]);
  box_muller_f32(h0.z, h0.w, a[2], a[3]);
  box_muller_f32(h1.x, h1.y, a[4], a[5]);
  box_muller_f32(h1.z, h1.w, b[0], b[1]);
  box_muller_f32(h2.x, h2.y, b[2], b[3]);
  box_muller_f32(h2.z, h2.w, b[4], b[5]);
}

__device__ __forceinline__ void stress_normals_ab_rk(const RoundKeys &rk, uint32_t box, uint32_t cell, uint32_t step,
                                                     float a[6], float b[6]) {
  const uint4 h0 = philox4x32_10_rk(make_uint4(cell, step, (kPurposeStress << 16) | 0u, box), rk);
  const uint4 h1 = philox4x32_10_rk(make_uint4(cell, step, (kPurposeStress << 16) | 1u, box), rk);
  const uint4 h2 = philox4x32_10_rk(make_uint4(cell, step, (kPurposeStress << 16) | 2u, box), rk);
  box_muller_f32(h0.x, h0.y, a[0], a[1]);
  box_muller_f32(h0.z, h0.w, a[2], a[3]);
  box_muller_f32(h1.x, h1.y, a[4], a[5]);
  box_muller_f32(h1.z, h1.w, b[0], b[1]);
  box_muller_f32(h2.x, h2.y, b[2], b[3]);
  box_muller_f32(h2.z, h2.w, b[4], b[5]);
}

// ---------------------------------------------------------------- kernel
// 1D weights of the 3 points nearest to s (in grid units, already shifted by
// the location-set offset): i0 = floor(s + 1/2), r = s - i0 in [-1/2, 1/2),
// phi(i0-1 - s), phi(i0 - s), phi(i0+1 - s) of the Roma-Peskin function.
// With S = sqrt(1 - 3 r^2): (2 - 3r - S)/6, (1 + S)/3, (2 + 3r - S)/6.
template <typename real>
__device__ __forceinline__ void peskin3(real r, real w[3]) {
  const real s = sqrt(real(1) - real(3) * r * r);
  w[0] = (real(2) - real(3) * r - s) / real(6);
  w[1] = (real(1) + s) / real(3);
  w[2] = (real(2) + real(3) * r - s) / real(6);
}

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// minimum-image integer offset b - a on a ring of n points
__device__ __forceinline__ int ring_delta(int b, int a, int n) {
  int d = (b - a) % n;
  if (d < 0) d += n;
  if (2 * d > n) d -= n;
  return d;
}

// a / b for a face density b near rho0.  FP32: the fast reciprocal-multiply
// (2 ulp).  FP64: the FP32 reciprocal of b refined by two Newton-Raphson
// steps r <- r + r (1 - b r) (each squares the relative error: ~2^-23, then
// ~2^-46, then below the FP64 rounding), times a: within 2 ulp of the
// correctly rounded quotient for any normal b, in 4 FP64 FMAs and a multiply
// (the FP64 form is bound by its FP64 pipe, which an IEEE division occupies
// longer).
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) {
  double r = double(__frcp_rn(float(b)));
  r = __fma_rn(r, __fma_rn(-b, r, 1.0), r);
  r = __fma_rn(r, __fma_rn(-b, r, 1.0), r);
  return __dmul_rn(a, r);
}

// a * b + c with one rounding, never split by the compiler: values that more
// than one CTA computes for the same cell (halo planes) must round the same
// way in every inlined copy of the code that produces them
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename real>
__device__ __forceinline__ real warp_sum(real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Entry of a kernel launched with programmatic dependent launch (launch_k):
// wait until the preceding grid in the stream has completed and its writes
// are visible, then let the next grid launch (its CTAs become resident as
// this grid's leave, and wait in turn).  Without the launch attribute both
// return at once.  Nothing before this call may touch global memory.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Index checks of the debug build (compiled with -DIC_BOUNDS_CHECK into
// libic_bounds.so).  IC_CHK(i, n) passes an element index i of an array of n
// elements; outside [0, n) it sets this translation unit's flag and yields 0,
// so the access stays inside the array and the host reports IC_ERR_ARG.  The
// checks sit on every grid, noise and particle index the kernels form and
// stand in for a memory checker.  IC_AT(p, i, j, n) is the address of
// element i + j of the n-element array at p, checked alike.  Without the
// macro IC_CHK(i, n) is i and IC_AT(p, i, j, n) is p + i + j, summed in the
// order of the unchecked code.
#ifdef IC_BOUNDS_CHECK
static __device__ unsigned int ic_bounds_flag;
template <typename I>
__device__ __forceinline__ I ic_checked(I i, unsigned long long n) {
  if (static_cast<unsigned long long>(static_cast<long long>(i)) < n) return i;
  atomicOr(&ic_bounds_flag, 1u);
  return I(0);
}
#define IC_CHK(i, n) ::ic::ic_checked((i), (unsigned long long)(n))
#define IC_AT(p, i, j, n) ((p) + ::ic::ic_checked((i) + (j), (unsigned long long)(n)))
// host: this translation unit's flag, cleared on read
#define IC_BOUNDS_READER(name)                                            \
  unsigned name() {                                                       \
    unsigned v = 0, zero = 0;                                             \
    if (cudaMemcpyFromSymbol(&v, ic_bounds_flag, sizeof(v)) != cudaSuccess || \
        cudaMemcpyToSymbol(ic_bounds_flag, &zero, sizeof(zero)) != cudaSuccess) \
      return 2u;                                                          \
    return v;                                                             \
  }
#else
#define IC_CHK(i, n) (i)
#define IC_AT(p, i, j, n) ((p) + (i) + (j))   // p + i + j: element i + j of the array at p
#define IC_BOUNDS_READER(name) \
  unsigned name() { return 0u; }
#endif

}  // namespace ic
