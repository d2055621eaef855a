// Double-float ("df32") arithmetic: a value is hi + lo with two floats, about
// 48 significant bits, built from the error-free transformations of Knuth
// (two-sum), Dekker (fast two-sum) and the FMA-based two-product (Ogita, Rump &
// Oishi 2005).  Used by the mixed-precision path for the absolute time and
// orbital phase, so that no FP64 instruction runs per sample.
#pragma once
#include <cuda_runtime.h>

namespace lisa {

struct df32 {
  float hi, lo;
};

__host__ __device__ inline df32 df_from_double(double x) {
  float h = (float)x;
  return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ df32 two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ df32 fast_two_sum(float a, float b) {   // |a| >= |b|
  float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df32 two_prod(float a, float b) {
  float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  df32 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + a.lo + b.lo);
}
__device__ __forceinline__ df32 df_add_f(df32 a, float b) {
  df32 s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, s.lo + a.lo);
}
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  df32 p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, p.lo + fmaf(a.hi, b.lo, a.lo * b.hi));
}
__device__ __forceinline__ df32 df_mul_f(df32 a, float b) {
  df32 p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
__device__ __forceinline__ df32 df_sqrt(df32 a) {          // a > 0
  float r = sqrtf(a.hi);
  df32 p = two_prod(r, r);
  float d = ((a.hi - p.hi) - p.lo + a.lo) * (0.5f / r);
  return fast_two_sum(r, d);
}

// x mod 2 pi in (-pi, pi] as a float, x a df32 with |x| < 4e5 (Cody-Waite
// reduction with 2 pi split in three floats, the first with 8 bits so that
// k * C1 is exact for |k| < 2^16).
__device__ __forceinline__ float df_mod_2pi(df32 x) {
  constexpr double kTwoPiD = 6.283185307179586476925286766559;
  constexpr float C1 = 6.28125f;
  constexpr float C2 = (float)(kTwoPiD - 6.28125);
  constexpr float C3 = (float)(kTwoPiD - 6.28125 - (double)(float)(kTwoPiD - 6.28125));
  float k = rintf(x.hi * (float)(1.0 / kTwoPiD));
  float r = fmaf(-k, C1, x.hi);             // exact (Sterbenz), may still be ~100
  r = fmaf(-k, C2, r);                      // one rounding, now |r| <~ pi
  r = r + x.lo;
  return fmaf(-k, C3, r);
}

}  // namespace lisa
