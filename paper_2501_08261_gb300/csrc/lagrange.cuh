// Centred Lagrange interpolation of odd order P (K = P + 1 nodes at offsets
// -(P-1)/2 .. (P+1)/2 around floor(tau)), the fractional-delay interpolator
// used for h at retarded times and y at TDI delays (Sec. II.B; P = 1 is the
// paper's linear interpolation).
#pragma once
#include "common.cuh"

namespace lisa {

// 1 / prod_{m != j} (j - m) for nodes 0..K-1 (node j <-> offset j - (P-1)/2).
template <typename T, int K>
__host__ __device__ inline T lagrange_denom_inv(int j) {
  double d = 1.0;
  for (int m = 0; m < K; ++m)
    if (m != j) d *= (double)(j - m);
  return T(1.0 / d);
}

template <typename T, int K>
struct LagrangeConst {
  T cinv[K];
  __host__ __device__ LagrangeConst() {
    for (int j = 0; j < K; ++j) cinv[j] = lagrange_denom_inv<T, K>(j);
  }
};

// w_j(eps) = cinv_j * prod_{m<j}(e_m) * prod_{m>j}(e_m), e_m = eps - (m - (P-1)/2).
template <typename T, int K>
__device__ inline void lagrange_weights(T eps, const T* __restrict__ cinv, T* w) {
  constexpr int H = (K - 2) / 2;           // (P-1)/2
  T pre = T(1);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    w[j] = pre * cinv[j];
    pre *= eps - T(j - H);
  }
  T suf = T(1);
#pragma unroll
  for (int j = K - 1; j >= 0; --j) {
    w[j] *= suf;
    suf *= eps - T(j - H);
  }
}

}  // namespace lisa
