// Mixed-precision pieces of the stand-in waveform (Sec. II.A) shared by the
// grid waveform kernel and the heterodyned response: the quaternion power
// table of the D-matrix sums and the FP32 Planck tapers.
#pragma once
#include "common.cuh"

namespace lisa {

// Powers of the quaternion's complex components Qa = q0 + i q3, Qb = q2 + i q1
// and of their conjugates, as far as the D-matrix sum of l <= 4, |m| <= 4
// reaches (Qa^8, Qb^8, conj^2), built once per sample by repeated products.
struct QPow {
  float ar[9], ai[9], br[9], bi[9], cr[3], ci[3], dr[3], di[3];
};

__device__ inline void qpow_fill(const float* q, QPow& P) {
  P.ar[0] = 1.0f; P.ai[0] = 0.0f; P.br[0] = 1.0f; P.bi[0] = 0.0f;
  P.cr[0] = 1.0f; P.ci[0] = 0.0f; P.dr[0] = 1.0f; P.di[0] = 0.0f;
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    P.ar[k] = P.ar[k - 1] * q[0] - P.ai[k - 1] * q[3];
    P.ai[k] = P.ar[k - 1] * q[3] + P.ai[k - 1] * q[0];
    P.br[k] = P.br[k - 1] * q[2] - P.bi[k - 1] * q[1];
    P.bi[k] = P.br[k - 1] * q[1] + P.bi[k - 1] * q[2];
  }
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    P.cr[k] = P.cr[k - 1] * q[0] + P.ci[k - 1] * q[3];      // conj(Qa)^k
    P.ci[k] = -P.cr[k - 1] * q[3] + P.ci[k - 1] * q[0];
    P.dr[k] = P.dr[k - 1] * q[2] + P.di[k - 1] * q[1];      // conj(Qb)^k
    P.di[k] = -P.dr[k - 1] * q[1] + P.di[k - 1] * q[2];
  }
}

// sqrt((2l+1)/4pi) D^l_{M,2} from the power table: sum over r of
// c_r Qa^(L+M-r) conj(Qa)^(L-2-r) Qb^(2-M+r) conj(Qb)^r (ylm_from_quat's sum
// with compile-time exponents; coefficients c_r from the walker record)
template <int L, int M>
__device__ inline void ylm_pow(const QPow& P, const float* c, float& re, float& im) {
  constexpr int r0 = M - 2 > 0 ? M - 2 : 0;
  constexpr int r1 = (L + M < L - 2) ? L + M : L - 2;
  re = 0.0f;
  im = 0.0f;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int r = r0 + q;
    if (r <= r1) {
      const float xr = P.ar[L + M - r] * P.cr[L - 2 - r] - P.ai[L + M - r] * P.ci[L - 2 - r];
      const float xi = P.ar[L + M - r] * P.ci[L - 2 - r] + P.ai[L + M - r] * P.cr[L - 2 - r];
      const float yr = P.br[2 - M + r] * P.dr[r] - P.bi[2 - M + r] * P.di[r];
      const float yi = P.br[2 - M + r] * P.di[r] + P.bi[2 - M + r] * P.dr[r];
      re = fmaf(c[q], xr * yr - xi * yi, re);
      im = fmaf(c[q], xr * yi + xi * yr, im);
    }
  }
}

template <int L, int M>
__device__ inline void ylm_pair(const QPow& P, const MixMode& Md, float& ypr, float& ypi,
                                float& ymr, float& ymi) {
  ylm_pow<L, M>(P, Md.yc[0], ypr, ypi);
  ylm_pow<L, -M>(P, Md.yc[1], ymr, ymi);
}

__device__ inline float planck_up_f(float x, float T) {      // x = t - t_a
  if (x <= 0.0f) return 0.0f;
  if (x >= T) return 1.0f;
  float z = T / x - T / (T - x);
  z = fminf(fmaxf(z, -80.0f), 80.0f);
  return 1.0f / (1.0f + __expf(z));
}
__device__ inline float planck_down_ff(float f) {
  const float f1 = (float)kFhi1, f2 = (float)kFhi2;
  if (f <= f1) return 1.0f;
  if (f >= f2) return 0.0f;
  float d = f2 - f1;
  float z = d / (f2 - f) - d / (f - f1);
  z = fminf(fmaxf(z, -80.0f), 80.0f);
  return 1.0f / (1.0f + __expf(z));
}

}  // namespace lisa
