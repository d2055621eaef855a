// Device functions of the declared IMRPhenomT-family stand-in (Sec. II.A):
// inspiral closed form in u = x^(1/8), x = nu (t_c - t) / (5 M); C1 ringdown
// attachment at x = kXMerge; single-spin simple-precession Euler angles in
// closed form; Wigner D^l_{m,2} from a unit quaternion (Sec. II.A, quaternion
// equations, with the index and power reading documented in the design notes).
#pragma once
#include "common.cuh"

namespace lisa {

// omega [rad/s] and orbital phase of the inspiral at u (FP64)
__device__ inline void insp_omega_phase(const WalkerRec& W, double u, double& om, double& ph) {
  double iu = 1.0 / u;
  double iu2 = iu * iu, iu3 = iu2 * iu;
  om = (iu3 + W.c1 * iu2 * iu3 + W.cs * iu3 * iu3) / (8.0 * W.M);
  double u2 = u * u;
  ph = -(u2 * u2 * u + (5.0 / 3.0) * W.c1 * u2 * u + 2.5 * W.cs * u2) / W.nu;
}

__device__ inline double insp_omega_dot(const WalkerRec& W, double u) {
  double iu = 1.0 / u;
  double iu2 = iu * iu, iu4 = iu2 * iu2, iu6 = iu4 * iu2, iu7 = iu6 * iu;
  return (3.0 * iu4 + 5.0 * W.c1 * iu6 + 6.0 * W.cs * iu7) / (8.0 * W.M) * W.nu * iu7 /
         (40.0 * W.M);
}

// Hamilton product a (x) b, components (w, x, y, z)
__host__ __device__ inline void qmul(const double* a, const double* b, double* o) {
  double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
  o[0] = w; o[1] = x; o[2] = y; o[3] = z;
}

// Unit quaternion of R_z(a) R_y(b) R_z(g) from the half-angle form of the
// paper's Euler -> quaternion equations (divided by sqrt 2).
__device__ inline void quat_euler(double a, double b, double g, double* q) {
  double cb = cos(0.5 * b), sb = sin(0.5 * b);
  q[0] = cb * cos(0.5 * (a + g));
  q[1] = -sb * sin(0.5 * (a - g));
  q[2] = sb * cos(0.5 * (a - g));
  q[3] = cb * sin(0.5 * (a + g));
}

// n! and C(n, k): exact integers in double for n <= 20 and n <= 12.  Device
// code reads them from constant-memory tables (the loop and the division
// they replace give the same values, but cost FP64 multiplies and divides on
// a pipe that runs at 1/64 of FP32); the host and larger arguments compute.
static __constant__ double kFactTab[21] = {1.0, 1.0, 2.0, 6.0, 24.0, 120.0, 720.0, 5040.0, 40320.0, 362880.0, 3628800.0, 39916800.0, 479001600.0, 6227020800.0, 87178291200.0, 1307674368000.0, 20922789888000.0, 355687428096000.0, 6402373705728000.0, 1.21645100408832e+17, 2.43290200817664e+18};
static __constant__ double kBinomTab[13][13] = {
    {1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0, 2.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0, 3.0, 3.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0, 4.0, 6.0, 4.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0, 5.0, 10.0, 10.0, 5.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0, 6.0, 15.0, 20.0, 15.0, 6.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0, 7.0, 21.0, 35.0, 35.0, 21.0, 7.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0, 8.0, 28.0, 56.0, 70.0, 56.0, 28.0, 8.0, 1.0, 0.0, 0.0, 0.0, 0.0},
    {1.0, 9.0, 36.0, 84.0, 126.0, 126.0, 84.0, 36.0, 9.0, 1.0, 0.0, 0.0, 0.0},
    {1.0, 10.0, 45.0, 120.0, 210.0, 252.0, 210.0, 120.0, 45.0, 10.0, 1.0, 0.0, 0.0},
    {1.0, 11.0, 55.0, 165.0, 330.0, 462.0, 462.0, 330.0, 165.0, 55.0, 11.0, 1.0, 0.0},
    {1.0, 12.0, 66.0, 220.0, 495.0, 792.0, 924.0, 792.0, 495.0, 220.0, 66.0, 12.0, 1.0}};
__host__ __device__ inline double fact(int n) {
#ifdef __CUDA_ARCH__
  if (n >= 0 && n <= 20) return kFactTab[n];
#endif
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}
__host__ __device__ inline double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
#ifdef __CUDA_ARCH__
  if (n <= 12) return kBinomTab[n][k];
#endif
  return fact(n) / (fact(k) * fact(n - k));
}

template <typename T>
struct cplx { T re, im; };

template <typename T>
__device__ inline cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ inline cplx<T> cpow(cplx<T> a, int n) {
  cplx<T> r{T(1), T(0)};
  for (int i = 0; i < n; ++i) r = cmul(r, a);
  return r;
}

// sqrt((2l+1)/4pi) D^l_{m,2}(q) with Q_a = q0 + i q3, Q_b = q2 + i q1:
//   sqrt((l+2)!(l-2)!/((l+m)!(l-m)!)) sum_rho (-1)^rho C(l+m, rho) C(l-m, l-2-rho)
//   Q_a^{l+m-rho} conj(Q_a)^{l-2-rho} Q_b^{2-m+rho} conj(Q_b)^rho
// (every power non-negative, so no branch is needed near beta = 0 or pi).
template <typename T>
__device__ inline cplx<T> ylm_from_quat(int l, int m, const T* q) {
  cplx<T> Qa{q[0], q[3]}, Qb{q[2], q[1]};
  cplx<T> Qac{q[0], -q[3]}, Qbc{q[2], -q[1]};
  cplx<T> acc{T(0), T(0)};
  int r0 = m - 2 > 0 ? m - 2 : 0;
  int r1 = (l + m < l - 2) ? l + m : l - 2;
  for (int r = r0; r <= r1; ++r) {
    T c = T(binom(l + m, r) * binom(l - m, l - 2 - r)) * ((r & 1) ? T(-1) : T(1));
    cplx<T> t = cmul(cmul(cpow(Qa, l + m - r), cpow(Qac, l - 2 - r)),
                     cmul(cpow(Qb, 2 - m + r), cpow(Qbc, r)));
    acc.re += c * t.re;
    acc.im += c * t.im;
  }
  T pref = T(sqrt(fact(l + 2) * fact(l - 2) / (fact(l + m) * fact(l - m))) *
             sqrt((2.0 * l + 1.0) / (4.0 * kPi)));
  return {pref * acc.re, pref * acc.im};
}

// Precession stand-in: primitive G(a) of (a - S cos th1) sqrt(a^2 + b^2).
__device__ inline double prec_G(double a, double b, double Sc) {
  double J = sqrt(a * a + b * b);
  double ash = b > 0.0 ? asinh(a / b) : 0.0;
  return J * J * J / 3.0 - Sc * (0.5 * a * J + 0.5 * b * b * ash);
}

// Euler angles of the co-precessing -> J rotation at u (frozen for t >= t_m
// by the caller passing u_m).  Returns cos(beta/2), sin(beta/2), alpha, gamma.
__device__ inline void prec_angles(const WalkerRec& W, double u, double& cbh, double& sbh,
                                   double& alpha, double& gamma) {
  double Sc = W.S * W.ctilt, b = W.S * W.stilt;
  double a = 2.0 * W.nu * u + Sc;
  double J = sqrt(a * a + b * b);
  double cb = a / J, sb = b / J;          // beta in [0, pi]
  if (cb >= 0.0) {
    cbh = sqrt(0.5 * (1.0 + cb));
    sbh = sb / (2.0 * cbh);
  } else {
    sbh = sqrt(0.5 * (1.0 - cb));
    cbh = sb / (2.0 * sbh);
  }
  alpha = -(5.0 * W.kp / (32.0 * W.nu * W.nu * W.nu)) * (prec_G(a, b, Sc) - W.G_ref);
  double u2 = u * u, ur2 = W.u_ref * W.u_ref;
  gamma = W.gamma_ref + (5.0 * W.kp / (8.0 * W.nu)) *
                            (2.0 * W.nu * (u2 * u - ur2 * W.u_ref) / 3.0 + 0.5 * Sc * (u2 - ur2));
}

}  // namespace lisa
