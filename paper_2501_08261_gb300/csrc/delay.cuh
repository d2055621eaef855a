// TDI delays at a grid sample from the FP64 orbit table (Sec. II.B, the X 1.5
// / 2.0 equations): shared by the TDI kernels and the heterodyned response.
#pragma once
#include "common.cuh"

namespace lisa {

// light time of link li at fractional grid position x: cubic Lagrange through
// four rows of the FP64 orbit table (stencil clamped inside the table, so the
// first and last rows extrapolate; L varies on the orbital time scale, so the
// interpolation error is far below the table's own rounding)
__device__ inline double light_time_at(const OrbitRec64* __restrict__ orb, int64_t n, int li,
                                       double x) {
  int64_t b = (int64_t)floor(x) - 1;
  b = b < 0 ? 0 : (b > n - 4 ? n - 4 : b);
  const double u = x - (double)b;
  const double w0 = -(u - 1.0) * (u - 2.0) * (u - 3.0) * (1.0 / 6.0);
  const double w1 = u * (u - 2.0) * (u - 3.0) * 0.5;
  const double w2 = -u * (u - 1.0) * (u - 3.0) * 0.5;
  const double w3 = u * (u - 1.0) * (u - 2.0) * (1.0 / 6.0);
  return w0 * orb[b].L[li] + w1 * orb[b + 1].L[li] + w2 * orb[b + 2].L[li] +
         w3 * orb[b + 3].L[li];
}

// delay D(t_i) [s] of a term: the sum of its light times at t_i, or (nested)
// tau = 0, tau += L_c(t_i - tau) over its links c in operator order
__device__ inline double term_delay_at(const TdiTerm& T, const int8_t* __restrict__ chain,
                                       const OrbitRec64* __restrict__ orb, int64_t n, int64_t i,
                                       double dt, int nested) {
  double D = 0.0;
  if (!nested) {
#pragma unroll
    for (int l = 0; l < kNLink; ++l) D += (double)T.cnt[l] * orb[i].L[l];
    return D;
  }
  for (int k = 0; k < T.ndelay; ++k) D += light_time_at(orb, n, chain[k], (double)i - D / dt);
  return D;
}

}  // namespace lisa
