// Centred Lagrange interpolation of odd order P (K = P + 1 nodes at offsets
// -(P-1)/2 .. (P+1)/2 around floor(tau)), the fractional-delay interpolator
// used for h at retarded times and y at TDI delays (Sec. II.B; P = 1 is the
// paper's linear interpolation).
#pragma once
#include <math.h>

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

// Paired form (FP32, K >= 8).  Nodes o and 1 - o pair up: (eps - o)(eps - 1 + o)
// = s + c_o with s = eps (eps - 1), c_o = o (1 - o), so the K - 1 factors left
// out of each w_j are one partner factor times a product over K/2 - 1 pair
// factors.  With pair k = (node k, node K-1-k), 1/prod(j - m) antisymmetric
// between the two nodes, and Q_k = prod_{k' != k} (s + c_k'):
//   w_k = (eps - 1 + o_k) R_k,  w_{K-1-k} = (o_k - eps) R_k,  R_k = cinv_k Q_k.
// The cinv_k are absorbed into per-pair scalings lam_k = Lam / cinv_k with
// Lam^(K/2-1) = prod_k cinv_k, so that prod_{k' != k} lam_k' (s + c_k') = R_k
// directly: one FMA per pair factor, prefix and suffix products over K/2
// pairs, then two operations per weight (about 120 operations against 160 for
// the prefix / suffix form over K nodes at K = 32).
struct LagrangePairs {
  float lam[16];         // lam_k
  float lamc[16];        // lam_k c_k
};

template <int K>
inline LagrangePairs lagrange_pairs() {
  LagrangePairs T{};
  constexpr int NP = K / 2, H = (K - 2) / 2;
  if constexpr (NP >= 2) {
    double la[NP], sg[NP], sum = 0.0;
    for (int k = 0; k < NP; ++k) {
      const double ci = lagrange_denom_inv<double, K>(k);
      la[k] = log(fabs(ci));
      sg[k] = ci < 0.0 ? -1.0 : 1.0;
      sum += la[k];
    }
    const double lL = sum / (NP - 1);       // log Lam
    for (int k = 0; k < NP; ++k) {
      const double lam = sg[k] * exp(lL - la[k]);
      const double o = (double)(k - H);
      T.lam[k] = (float)lam;
      T.lamc[k] = (float)(lam * o * (1.0 - o));
    }
  }
  return T;
}

template <int K>
__device__ __forceinline__ void lagrange_weights_paired(float eps, const LagrangePairs& T,
                                                        float* w) {
  static_assert(K >= 8 && K <= 32 && K % 2 == 0, "paired weights need even K in [8, 32]");
  constexpr int NP = K / 2, H = (K - 2) / 2;
  const float s = fmaf(eps, eps, -eps);
  float P[NP], pre[NP], suf[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) P[k] = fmaf(s, T.lam[k], T.lamc[k]);
  pre[1] = P[0];
#pragma unroll
  for (int k = 2; k < NP; ++k) pre[k] = pre[k - 1] * P[k - 1];
  suf[NP - 2] = P[NP - 1];
#pragma unroll
  for (int k = NP - 3; k >= 0; --k) suf[k] = suf[k + 1] * P[k + 1];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float R = k == 0 ? suf[0] : (k == NP - 1 ? pre[NP - 1] : pre[k] * suf[k]);
    w[k] = (eps + (float)(k - H - 1)) * R;
    w[K - 1 - k] = ((float)(k - H) - eps) * R;
  }
}

}  // namespace lisa
