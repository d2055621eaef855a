// Shared device-side definitions of the LISA time-domain likelihood library.
// Everything here is the library's own: constants, per-walker records, the
// orbit-table record and small numeric helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df32.cuh"

namespace lisa {

// ---- physical constants (SI) -------------------------------------------
constexpr double kC        = 299792458.0;
constexpr double kTsun     = 4.925490947641267e-06;      // G Msun / c^3 [s]
constexpr double kParsec   = 3.085677581491367e16;
constexpr double kGpcSec   = 1.0e9 * kParsec / kC;        // Gpc in light-seconds
constexpr double kAUSec    = 149597870700.0 / kC;         // AU in light-seconds
constexpr double kYear     = 31558149.763545603;          // sidereal year [s]
constexpr double kPi       = 3.141592653589793238462643383279502884;
constexpr double kOmegaOrb = 2.0 * kPi / kYear;
constexpr double kArmSec   = 2.5e9 / kC;                  // nominal light time [s]

// ---- declared waveform stand-in constants (Sec. II.A defers IMRPhenomT's)
constexpr double kFmin     = 1.0e-4;     // (2,2) start / reference frequency [Hz]
constexpr double kTaper    = 1.0e4;      // Planck start taper [s]
constexpr double kFhi1     = 0.08;       // per-mode high-frequency taper [Hz]
constexpr double kFhi2     = 0.09;
constexpr double kXMerge   = 2.0;        // x where the ringdown attaches
constexpr double kCSpin    = 0.5;        // spin-orbit coefficient of omega

constexpr int kNPar   = 15;
constexpr int kNMode  = 5;               // (2,2) (2,1) (3,3) (3,2) (4,4)
constexpr int kNLink  = 6;               // l = 1, 2, 3, -1, -2, -3

// sender / receiver spacecraft (0-based) of link index j (l = 1,2,3,-1,-2,-3)
__host__ __device__ constexpr int link_sender(int j) {
  return j == 0 ? 2 : j == 1 ? 0 : j == 2 ? 1 : j == 3 ? 1 : j == 4 ? 2 : 0;
}
__host__ __device__ constexpr int link_receiver(int j) {
  return j == 0 ? 1 : j == 1 ? 2 : j == 2 ? 0 : j == 3 ? 2 : j == 4 ? 0 : 1;
}

// ---- per-walker constants (built by the prep kernel, FP64) ---------------
struct ModeRec {
  double pref;        // (M nu / D) 8 sqrt(pi/5) * PN coefficient
  double p;           // amplitude ~ (M omega)^p
  double A_m;         // amplitude at the attachment
  double a_lm;        // ringdown (1 + a tau) slope
  double w_rd;        // ringdown angular frequency [rad/s]
  double Yp_re, Yp_im, Ym_re, Ym_im;   // aligned: -2Y_{l,m}, -2Y_{l,-m}
  int l, m;
};

// Mixed-precision copy of the per-walker constants: absolute times and the
// phase polynomial in double-float, everything else in FP32.
struct MixMode {
  float pref;          // amplitude prefactor
  int pw;              // amplitude ~ v^(2 + pw), v = (M omega)^(1/3)
  float A_m, a_lm;     // ringdown amplitude and (1 + a tau) slope
  float w_rd, dw;      // ringdown frequency and m omega_m - w_rd [rad/s]
  float ph0;           // m phi_m reduced to (-pi, pi]
  float yp_re, yp_im, ym_re, ym_im;
  int l, m;
  float yc[2][3];      // precessing: coefficients of the D-matrix sum for +m (0) and -m (1),
                       // terms r = max(+-m - 2, 0) + q, prefactor included (zero past the end)
};
struct MixRec {
  df32 T;              // t_c - t0
  df32 kap;            // nu / (5 M)
  df32 A5, A3, A2;     // phi = -(A5 u^5 + A3 u^3 + A2 u^2)
  df32 tm, tstart, ta; // t_m, t_start, t_a minus t0
  df32 dt;             // sample spacing
  float c1, cs;        // M omega = (u^-3 + c1 u^-5 + cs u^-6) / 8
  float invM;          // 1 / M [1/s]
  float tau_d;
  float c2psi, s2psi;
  float k[3], u[3], v[3];
  float aucb;          // AU cos(beta) [light-s]
  // precession stand-in, FP32 except the gamma polynomial
  float S, Sc, b, kp, alpha_c;         // alpha = alpha_c * (G(a) - Gref)
  df32 Gref;                          // G without its asinh term at the reference
  df32 g0, g3, g2;     // gamma = g0 + g3 u^3 + g2 u^2
  float twonu, um;
  float q03[4];
  MixMode mode[kNMode];
  int nmode;
};

struct WalkerRec {
  double M, nu, delta, chi, c1, cs;
  double tc, tm, t_start, t_a, um, tau_d;
  double om_m, ph_m;
  double k[3], u[3], v[3];
  double c2psi, s2psi;
  // precession stand-in
  double S, ctilt, stilt, kp, u_ref, G_ref, gamma_ref;
  double q03[4];      // inverse of the J->L0 quaternion times q(phi_ref, iota, 0)
  ModeRec mode[kNMode];
  int nmode;
  int status;         // 0 ok, 1 invalid parameters
  MixRec mx;
};

// ---- orbit table, one record per grid sample (walker-independent) --------
struct OrbitRec64 {      // absolute positions [light-s] and light times [s]
  double rr[3][3];       // spacecraft positions at t_i
  double rs[kNLink][3];  // sender position at emission, t_i - L_l
  double n[kNLink][3];   // unit vector sender -> receiver
  double L[kNLink];      // light times
};
struct OrbitRec32 {      // the same, positions relative to the guiding centre
  float rr[3][3];        // g(t) = AU (cos Omega t, sin Omega t, 0), and light
  float rs[kNLink][3];   // times as offsets L_l - kArmSec
  float n[kNLink][3];
  float L[kNLink];
};

// ---- TDI term tables (built on the host from the printed X equations) -----
struct TdiTerm {
  int8_t chan, sign, ndelay;
  int8_t cnt[kNLink];             // how many times L_l enters the delay
};
struct TdiTable {
  int nterm[kNLink];              // terms that read link l (4 for TDI 1.5, 8 for TDI 2)
  TdiTerm term[kNLink][8];
  int8_t dterm[kNLink][8];        // index among the delayed terms, -1 if undelayed
  int8_t chain[kNLink][8][8];     // term's delay links in operator order (first: at t)
  int n_dterms;
  int max_links_in_delay;
};

// ---- mixed-path TDI weights, per 64-sample tile and delayed term ------------
// Built once per context from the FP64 orbit table.  For a tile starting at
// sample i_a and a term of delay D(t): tau = i - D(t)/dt; the tile anchor
// tau_a = i_a - D(t_a)/dt = i_a + bo + eps_a.  With c = i + bo and first
// differences dy_m = y_{m+1} - y_m, the Lagrange value at eps_a is rewritten
// (summation by parts, exact) as
//   y_c + sum_{m=-15..15} C_m dy_{c+m},  C_m = sum_{o_k > m} w_k (m >= 0),
//                                        C_m = -sum_{o_k <= m} w_k (m < 0),
// with C the FP64 cumulative weights rounded to FP32.  Inside the tile the
// fraction drifts by j (a1 + j a2) samples (j = i - i_a); m1 = sum (C_f - C)
// is the first-moment error of the rounding.  The kernel evaluates
//   y_c + sum_m C_m dy_{c+m} + (j (a1 + j a2) - m1) dy_c.
// C, m1 and the s* fields carry the term's sign (+-1, exact), so the kernel
// adds them without multiplying; a1, a2, eps_a stay unsigned for positions.
constexpr int kTdiTile = 64;
struct alignas(16) TdiTileTerm {
  float C[32];           // sign * C[m + H], m = -H .. H (H = (K-2)/2); C[K-1..31] = 0
  float m1, a1, a2;      // sign * m1; drift of the fraction j (a1 + j a2)
  float eps_a;
  int bo;
  int split;             // the fraction leaves [0, 1) inside the tile
  float sa1, sa2, se;    // sign * a1, sign * a2, sign * eps_a
  int pad[3];
};

// ---- mixed-path TDI: one FIR per (channel, link) pair -----------------------
// The terms of one channel that read the same link differ only in their
// delays, and each is linear in the first differences dy of that link, so
// per tile their difference weights add into one FIR over the union of their
// windows: G[k] multiplies dy at row (output row + boff + k).  G is summed in
// FP64 and rounded to FP32 once.  The zeroth and first moments of that
// rounding error are taken out by two one-tap corrections wa, wb at the
// centre rows (offsets ma < mb) of the pair's outermost terms, so the error
// left in the FIR's response vanishes to second order in frequency.
// Each term keeps its own |y|-sized centre sample, its linear-interpolation
// part and the drift of its fraction (TdiTermLite); terms whose fraction wraps
// inside the tile (kind 2) are evaluated per sample and stay out of G.
constexpr int kTdiPairs = 12;           // 6 links x the 2 channels that read each
constexpr int kGMax = 64;               // widest combined FIR (taps)
struct TdiTermLite {
  int bo, kind;          // centre offset; 0 undelayed, 1 in G, 2 per-sample
  float sg, se, sa1, sa2;
  float eps_a, a1, a2;   // unsigned fraction and drift (kind 2)
};
struct alignas(16) TdiTilePair {
  float G[kGMax];        // signed combined weights, zero beyond ntap
  int boff, ntap4, ma, mb;
  int chan, nterm;
  float wa, wb;
  TdiTermLite t[4];
};

// ---- small helpers --------------------------------------------------------
__host__ __device__ inline double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Planck window rising from 0 at x = a to 1 at x = a + T.
__device__ inline double planck_up(double x, double a, double T) {
  if (x <= a) return 0.0;
  if (x >= a + T) return 1.0;
  double z = T / (x - a) - T / (a + T - x);
  z = fmin(fmax(z, -700.0), 700.0);
  return 1.0 / (1.0 + exp(z));
}
// Per-mode high-frequency cut: 1 below kFhi1, 0 above kFhi2.
__device__ inline double planck_down_f(double f) {
  if (f <= kFhi1) return 1.0;
  if (f >= kFhi2) return 0.0;
  double d = kFhi2 - kFhi1;
  double z = d / (kFhi2 - f) - d / (f - kFhi1);
  z = fmin(fmax(z, -700.0), 700.0);
  return 1.0 / (1.0 + exp(z));
}

}  // namespace lisa
