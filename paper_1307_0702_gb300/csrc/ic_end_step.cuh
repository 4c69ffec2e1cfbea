// The end-of-step bookkeeping as the threads of one CTA run it (k_end_of_step
// of a box without particles, the last CTA of k_final of a box with).
#pragma once
#include <cuda_runtime.h>

#include "ic_internal.hpp"

namespace ic {

// s: shared scratch of blockDim.x doubles; blockDim.x a power of two
__device__ inline void end_of_step_cta(const EndArgs &e, double *s) {
  const int64_t n0 = e.step[0];   // read by every thread before thread 0 advances it
  double acc = 0.0;
  for (int b = threadIdx.x; b < e.nb; b += blockDim.x) acc += e.partials[b];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double A = e.has_mode ? 2.0 * s[0] * e.inv_cells : 0.0;
    const int64_t j = n0 - e.step[1];
    const double w = (j >= 0 && j < e.step[2]) ? e.weights[j] : 0.0;
    if (!isfinite(s[0])) atomicOr(e.status, kStatusNonfinite);
    e.scalars[0] += w;
    e.scalars[1] += w * A * A;
    e.scalars[2] = A;
    e.step[0] = n0 + 1;
  }
  if (threadIdx.x < 3) {
    // drive amplitudes of the RK stages of the next step (t^n, t^{n+1}, t^{n+1/2})
    const double frac = threadIdx.x == 0 ? 0.0 : (threadIdx.x == 1 ? 1.0 : 0.5);
    const double t = (double(n0 + 1) + frac) * e.dt;
    const double d = e.amp * sin(e.omega * t + e.phase);
    e.drive[threadIdx.x] = d;
    e.drive_f[threadIdx.x] = float(d);
  }
}

}  // namespace ic
