// Heterodyned time-domain likelihood (the speed-up route that Sec. I and
// Sec. IV of the paper name; the time-domain form is this library's and is
// stated in include/lisa_td.h).
//
// Per call, per walker:
//   node kernel   at each of B node times t_b: every TDI term of X, Y, Z reads
//                 its link at t' = t_b - D; the link response of each mode pair
//                 is formed from the waveform evaluated at the exact emission
//                 and reception times of Eq. (yslr) (two evaluations per term),
//                 then A, E, T, the demodulation by the fiducial carrier and the
//                 difference to the fiducial's own node value;
//   expand kernel at every grid sample: X0 - d + Re sum_j C_j cubic(dZ_j) per
//                 channel, written in the residual layout of the full path;
// then the full path's FFT pass 1, pass 2 + PSD-weighted norm and reduction.
// The walker-independent pieces -- the delayed times and link geometry of every
// (node, term), the carriers on the grid, X0 -- are built once per set-up.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "delay.cuh"
#include "internal.h"
#include "trace.h"
#include "standin.cuh"

namespace lisa {

namespace {

constexpr int kHetTermsMax = 16;        // terms of one channel (TDI 2)
constexpr int64_t kX0Chunk = 16384;     // grid samples per pass of the X0 set-up
constexpr int kNodeThreads = 128;

// one term of one channel: the link it reads, its sign and its delay
struct HetTerm {
  TdiTerm t;
  int8_t chain[8];
  int link;
  double sign;
};
struct HetTerms {
  int ntc;                              // terms per channel (8 or 16)
  HetTerm term[3][kHetTermsMax];
};

// delayed reception time t' of one (node, term), its light time, receiver and
// emitter positions [light-s] and unit vector, and the term's sign (0 when t'
// is off the grid: the term then reads zero)
struct HetGeom64 {
  double tp, L;
  double rr[3], rs[3], n[3];
  double sign;
};
// ---------------------------------------------------------------------------
// walker-independent tables
// ---------------------------------------------------------------------------

__global__ void het_geom_kernel(const OrbitRec64* __restrict__ orb, int64_t n, double t0,
                                double dt, const HetTerms* __restrict__ terms,
                                const int64_t* __restrict__ nodes, int64_t start, int64_t B,
                                int nested, HetGeom64* __restrict__ g64) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int q = blockIdx.y;
  const int ntc = terms->ntc;
  const HetTerm& T = terms->term[q / ntc][q % ntc];
  const int64_t ib = nodes ? nodes[b] : start + b;
  const double D = term_delay_at(T.t, T.chain, orb, n, ib, dt, nested);
  const double tp = t0 + (double)ib * dt - D;
  const bool inside = tp >= t0 && tp <= t0 + (double)(n - 1) * dt;
  // cubic Lagrange through four orbit-table rows at x = (t' - t0) / dt
  const double x = (double)ib - D / dt;
  int64_t base = (int64_t)floor(x) - 1;
  base = base < 0 ? 0 : (base > n - 4 ? n - 4 : base);
  const double u = x - (double)base;
  const double w[4] = {-(u - 1.0) * (u - 2.0) * (u - 3.0) * (1.0 / 6.0),
                       u * (u - 2.0) * (u - 3.0) * 0.5, -u * (u - 1.0) * (u - 3.0) * 0.5,
                       u * (u - 1.0) * (u - 2.0) * (1.0 / 6.0)};
  const int li = T.link, rc = link_receiver(li);
  HetGeom64 G;
  G.L = 0.0;
  for (int d = 0; d < 3; ++d) G.rr[d] = G.rs[d] = 0.0;
  for (int k = 0; k < 4; ++k) {
    const OrbitRec64& R = orb[base + k];
    G.L += w[k] * R.L[li];
    for (int d = 0; d < 3; ++d) {
      G.rr[d] += w[k] * R.rr[rc][d];
      G.rs[d] += w[k] * R.rs[li][d];
    }
  }
  const double e0 = G.rr[0] - G.rs[0], e1 = G.rr[1] - G.rs[1], e2 = G.rr[2] - G.rs[2];
  const double inv = 1.0 / sqrt(e0 * e0 + e1 * e1 + e2 * e2);
  G.n[0] = e0 * inv;
  G.n[1] = e1 * inv;
  G.n[2] = e2 * inv;
  G.tp = tp;
  G.sign = inside ? T.sign : 0.0;
  g64[(int64_t)q * B + b] = G;
}

// fiducial carriers C_j(t_i) = e^{-i Phi_j(t_i; theta0)} (the phase of
// polar_fp64: inspiral m phi(u), then the C1 ringdown phase)
__global__ void het_carrier_kernel(const WalkerRec* __restrict__ fid, int64_t n, double t0,
                                   double dt, double2* __restrict__ c64,
                                   float2* __restrict__ c32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const WalkerRec& W = *fid;
  const double t = t0 + (double)i * dt;
  const bool insp = t < W.tm;
  double ph = 0.0, tau = 0.0, dec = 1.0;
  if (insp) {
    const double x = W.nu * (W.tc - t) / (5.0 * W.M);
    double om;
    insp_omega_phase(W, sqrt(sqrt(sqrt(x))), om, ph);
  } else {
    tau = t - W.tm;
    dec = exp(-tau / W.tau_d);
  }
  for (int j = 0; j < W.nmode; ++j) {
    const ModeRec& Md = W.mode[j];
    const double phase = insp ? Md.m * ph
                              : Md.m * W.ph_m + Md.w_rd * tau +
                                    (Md.m * W.om_m - Md.w_rd) * W.tau_d * (1.0 - dec);
    double s, c;
    sincos(phase, &s, &c);
    c64[i * W.nmode + j] = make_double2(c, -s);
    c32[i * W.nmode + j] = make_float2((float)c, (float)-s);
  }
}

// bin[i] = the b with nodes[b] <= i < nodes[b + 1] (B - 2 for the last sample)
__global__ void het_bin_kernel(const int64_t* __restrict__ nodes, int64_t B, int64_t n,
                               int32_t* __restrict__ bin) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t lo = 0, hi = B - 1;                    // nodes[lo] <= i < nodes[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    if (nodes[mid] <= i) lo = mid;
    else hi = mid;
  }
  bin[i] = (int32_t)lo;
}

// base[c][i] = X0 - data (FP64 then rounded for the mixed path), or X0 alone
__global__ void het_base_kernel(int64_t m, const double* __restrict__ x0,
                                const double* __restrict__ data, double* __restrict__ b64,
                                float* __restrict__ b32, float* __restrict__ x32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double v = x0[i] - (data ? data[i] : 0.0);
  if (b64) b64[i] = v;
  if (b32) b32[i] = (float)v;
  if (x32) x32[i] = (float)x0[i];
}

// ---------------------------------------------------------------------------
// the analytic mode polarisations of one walker at one time, accumulated into
// acc[j] += h_j (ap (P_j + sg conj Q_j) + ax i (P_j - sg conj Q_j)),
// P = e^{2 i psi} Y+, Q = e^{2 i psi} Y-, h_j = A e^{-i Phi_j}: the real
// part of ap hp_j + ax hx_j for the pair's h+ = Re hp_j, hx = Re hx_j.
// FP64 throughout: the TDI sums of a node cancel the signal at low frequency
// by orders of magnitude, so every term needs far more than FP32's 24 bits
// (FP32 terms leave their rounding in A, E and, worst, T, where the PSD
// weights it by up to ~1e10 at 1e-4 Hz).
// ---------------------------------------------------------------------------

// per-walker constants of the evaluation, built once per block in shared
// memory (a block serves one walker)
struct HetMode {
  double pref, A_m, a_lm, w_rd, phm, dw;   // inspiral prefactor; ringdown constants
  double ppr, ppi, pxr, pxi;               // aligned: P + sg conj Q and i (P - sg conj Q)
  double yc[2][3];                         // precessing: D-matrix sum coefficients (+m, -m)
  int l, m, pw;                            // amplitude ~ v^(2 + pw), v = (M omega)^(1/3)
};
struct HetWalker {
  double kap, invnu, invM, c1, cs, tc, tm, t_start, t_a, tau_d, c2psi, s2psi;
  double mw_taper;                         // M omega at which the highest m reaches kFhi1
  int status, nmode;
  HetMode mode[kNMode];
};

__device__ void het_walker_fill(const WalkerRec& W, HetWalker& H) {
  H.kap = W.nu / (5.0 * W.M);
  H.invnu = 1.0 / W.nu;
  H.invM = 1.0 / W.M;
  H.c1 = W.c1;
  H.cs = W.cs;
  H.tc = W.tc;
  H.tm = W.tm;
  H.t_start = W.t_start;
  H.t_a = W.t_a;
  H.tau_d = W.tau_d;
  H.c2psi = W.c2psi;
  H.s2psi = W.s2psi;
  H.status = W.status;
  H.nmode = W.nmode;
  int mmax = 1;
  for (int j = 0; j < W.nmode; ++j) mmax = W.mode[j].m > mmax ? W.mode[j].m : mmax;
  H.mw_taper = 2.0 * kPi * kFhi1 * W.M / mmax;
  for (int j = 0; j < W.nmode; ++j) {
    const ModeRec& Md = W.mode[j];
    HetMode& D = H.mode[j];
    D.l = Md.l;
    D.m = Md.m;
    D.pw = (int)lrint(3.0 * Md.p - 2.0);
    D.pref = Md.pref;
    D.A_m = Md.A_m;
    D.a_lm = Md.a_lm;
    D.w_rd = Md.w_rd;
    D.phm = Md.m * W.ph_m;
    D.dw = Md.m * W.om_m - Md.w_rd;
    const double sg = (Md.l & 1) ? -1.0 : 1.0, c2 = W.c2psi, s2 = W.s2psi;
    const double Pr = c2 * Md.Yp_re - s2 * Md.Yp_im, Pi = c2 * Md.Yp_im + s2 * Md.Yp_re;
    const double Qr = c2 * Md.Ym_re - s2 * Md.Ym_im, Qi = c2 * Md.Ym_im + s2 * Md.Ym_re;
    D.ppr = Pr + sg * Qr;
    D.ppi = Pi - sg * Qi;
    D.pxr = -(Pi + sg * Qi);
    D.pxi = Pr - sg * Qr;
    // sqrt((2l+1)/4pi) D^l_{+-m,2}: sum over r of c_r Qa^(l+m-r) conj(Qa)^(l-2-r)
    // Qb^(2-m+r) conj(Qb)^r (the sum of ylm_from_quat, coefficients kept)
    for (int sgn = 0; sgn < 2; ++sgn) {
      const int l = Md.l, mm = sgn ? -Md.m : Md.m;
      const int r0 = mm - 2 > 0 ? mm - 2 : 0;
      const int r1 = (l + mm < l - 2) ? l + mm : l - 2;
      const double pref = sqrt(fact(l + 2) * fact(l - 2) / (fact(l + mm) * fact(l - mm))) *
                          sqrt((2.0 * l + 1.0) / (4.0 * kPi));
      for (int q = 0; q < 3; ++q) {
        const int r = r0 + q;
        D.yc[sgn][q] = r <= r1 ? binom(l + mm, r) * binom(l - mm, l - 2 - r) *
                                     ((r & 1) ? -1.0 : 1.0) * pref
                               : 0.0;
      }
    }
  }
}

// powers of Qa = q0 + i q3, Qb = q2 + i q1 (to 8) and of their conjugates (to 2)
struct QPowD {
  double ar[9], ai[9], br[9], bi[9], cr[3], ci[3], dr[3], di[3];
};

__device__ inline void qpowd_fill(const double* q, QPowD& P) {
  P.ar[0] = 1.0; P.ai[0] = 0.0; P.br[0] = 1.0; P.bi[0] = 0.0;
  P.cr[0] = 1.0; P.ci[0] = 0.0; P.dr[0] = 1.0; P.di[0] = 0.0;
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    P.ar[k] = P.ar[k - 1] * q[0] - P.ai[k - 1] * q[3];
    P.ai[k] = P.ar[k - 1] * q[3] + P.ai[k - 1] * q[0];
    P.br[k] = P.br[k - 1] * q[2] - P.bi[k - 1] * q[1];
    P.bi[k] = P.br[k - 1] * q[1] + P.bi[k - 1] * q[2];
  }
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    P.cr[k] = P.cr[k - 1] * q[0] + P.ci[k - 1] * q[3];
    P.ci[k] = -P.cr[k - 1] * q[3] + P.ci[k - 1] * q[0];
    P.dr[k] = P.dr[k - 1] * q[2] + P.di[k - 1] * q[1];
    P.di[k] = -P.dr[k - 1] * q[1] + P.di[k - 1] * q[2];
  }
}

template <int L, int M>
__device__ inline void ylmd_pow(const QPowD& P, const double* c, double& re, double& im) {
  constexpr int r0 = M - 2 > 0 ? M - 2 : 0;
  constexpr int r1 = (L + M < L - 2) ? L + M : L - 2;
  re = 0.0;
  im = 0.0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int r = r0 + q;
    if (r <= r1) {
      const double xr = P.ar[L + M - r] * P.cr[L - 2 - r] - P.ai[L + M - r] * P.ci[L - 2 - r];
      const double xi = P.ar[L + M - r] * P.ci[L - 2 - r] + P.ai[L + M - r] * P.cr[L - 2 - r];
      const double yr = P.br[2 - M + r] * P.dr[r] - P.bi[2 - M + r] * P.di[r];
      const double yi = P.br[2 - M + r] * P.di[r] + P.bi[2 - M + r] * P.dr[r];
      re += c[q] * (xr * yr - xi * yi);
      im += c[q] * (xr * yi + xi * yr);
    }
  }
}

template <int L, int M>
__device__ inline void ylmd_pair(const QPowD& P, const HetMode& D, double& ypr, double& ypi,
                                 double& ymr, double& ymi) {
  ylmd_pow<L, M>(P, D.yc[0], ypr, ypi);
  ylmd_pow<L, -M>(P, D.yc[1], ymr, ymi);
}

// FP64 roots and reciprocals from an FP32 seed refined by two Newton steps
// whose slope is kept from the seed: each step multiplies the relative error
// by ~1e-7 (plus the quadratic term), so the results land at FP64 rounding
// (one step leaves ~1e-14: random per evaluation, which the TDI sums do not
// cancel) at a fraction of the FP64 pipe's cost of sqrt, cbrt and division
__device__ __forceinline__ double rcp_nr(double a) {          // 1 / a, a > 0 normal
  double r = (double)__frcp_rn((float)a);
#pragma unroll
  for (int k = 0; k < 2; ++k) r = fma(r, fma(-a, r, 1.0), r);
  return r;
}
__device__ __forceinline__ double root8_nr(double x) {        // x^(1/8), x > 0
  const float xf = (float)x;
  const float uf = sqrtf(sqrtf(sqrtf(xf)));
  const double slope = (double)(uf / (8.0f * xf));            // 1 / (8 u^7) = u / (8 x)
  double u = (double)uf;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double u2 = u * u, u4 = u2 * u2;
    u = fma(x - u4 * u4, slope, u);
  }
  return u;
}
__device__ __forceinline__ double cbrt_nr(double a) {         // a^(1/3), a > 0
  const float vf = cbrtf((float)a);
  const double slope = (double)(1.0f / (3.0f * vf * vf));
  double v = (double)vf;
#pragma unroll
  for (int k = 0; k < 2; ++k) v = fma(a - v * v * v, slope, v);
  return v;
}

// x - 2 pi k with k = rint(x / 2 pi): |result| <= pi, for the phases of
// months-long chirps (up to ~1e6 rad); 2 pi split into its double and the
// double of the remainder (2 pi - 6.283185307179586 = 2.449293598294706e-16)
__device__ __forceinline__ double reduce_2pi(double x) {
  const double k = rint(x * 0.15915494309189535);
  const double r = fma(-k, 6.283185307179586, x);
  return fma(-k, 2.4492935982947064e-16, r);
}

// absolute time t; zero outside [t0, t_end].  RAW (aligned spins only):
// acc[j] += ap h_j, the angular weights left to the caller, which applies them
// once to the difference of a link's two ends
template <bool PREC, bool RAW = false>
__device__ __forceinline__ void modes_fp64(const HetWalker& H, const WalkerRec& W, double t,
                                           double t0, double t_end, double ap, double ax,
                                           double2 (&acc)[kNMode]) {
  if (H.status != 0 || t < t0 || t > t_end || t < H.t_start) return;
  const double win = planck_up(t, H.t_a, kTaper);
  if (win == 0.0) return;
  const bool insp = t < H.tm;
  double u = W.um, Mw = 0.0, tau = 0.0, dec = 1.0, e1r = 1.0, e1i = 0.0, v = 0.0;
  if (insp) {
    u = root8_nr(H.kap * (H.tc - t));
    const double iu = rcp_nr(u);
    const double iu2 = iu * iu, iu3 = iu2 * iu;
    Mw = 0.125 * (iu3 + H.c1 * iu2 * iu3 + H.cs * iu3 * iu3);        // M omega
    const double u2 = u * u;
    const double ph = -(u2 * u2 * u + (5.0 / 3.0) * H.c1 * u2 * u + 2.5 * H.cs * u2) * H.invnu;
    double s1, c1;
    sincos(reduce_2pi(ph), &s1, &c1);
    e1r = c1;                                    // e^{-i phi}
    e1i = -s1;
    v = cbrt_nr(Mw);
  } else {
    tau = t - H.tm;
    dec = exp(-tau / H.tau_d);
  }
  if (RAW && insp) {
    // acc[j] += ap A_j e^{-i m_j phi}: one multiply and two FMAs per mode; the
    // high-frequency taper is looked at only once some mode can reach it
    const bool taper = Mw > H.mw_taper;
    const double v2 = v * v;
    const double w0 = ap * win * v2, w1 = w0 * v, w2 = w1 * v;
    double pr[5], pim[5];
    pr[1] = e1r; pim[1] = e1i;
#pragma unroll
    for (int m = 2; m <= 4; ++m) {
      pr[m] = pr[m - 1] * e1r - pim[m - 1] * e1i;
      pim[m] = pr[m - 1] * e1i + pim[m - 1] * e1r;
    }
#pragma unroll
    for (int j = 0; j < kNMode; ++j) {
      if (j >= H.nmode) continue;
      const HetMode& D = H.mode[j];
      double a = D.pref * (D.pw == 0 ? w0 : (D.pw == 1 ? w1 : w2));
      if (taper) a *= planck_down_f(D.m * Mw * H.invM * (0.5 / kPi));
      double hr = pr[1], hi = pim[1];
#pragma unroll
      for (int k = 2; k <= 4; ++k)
        if (k == D.m) {
          hr = pr[k];
          hi = pim[k];
        }
      acc[j].x = fma(a, hr, acc[j].x);
      acc[j].y = fma(a, hi, acc[j].y);
    }
    return;
  }
  QPowD P;
  if (PREC) {
    double cbh, sbh, al, ga;
    prec_angles(W, u, cbh, sbh, al, ga);
    double sp, cp, sm, cm;
    sincos(0.5 * (al + ga), &sp, &cp);
    sincos(0.5 * (al - ga), &sm, &cm);
    const double q1[4] = {cbh * cp, sbh * sm, -sbh * cm, -cbh * sp};   // q(al, be, ga)^-1
    double qT[4];
    qmul(q1, W.q03, qT);
    qpowd_fill(qT, P);
  }
  // e^{-i m phi}, m = 1..4
  double pr[5], pim[5];
  pr[1] = e1r; pim[1] = e1i;
#pragma unroll
  for (int m = 2; m <= 4; ++m) {
    pr[m] = pr[m - 1] * e1r - pim[m - 1] * e1i;
    pim[m] = pr[m - 1] * e1i + pim[m - 1] * e1r;
  }
  const double v2 = v * v;
#pragma unroll
  for (int j = 0; j < kNMode; ++j) {
    if (j >= H.nmode) continue;
    const HetMode& D = H.mode[j];
    double amp, hr, hi, freq;
    if (insp) {
      amp = D.pref * (D.pw == 0 ? v2 : (D.pw == 1 ? v2 * v : v2 * v2));
      freq = D.m * Mw * H.invM;
      hr = pr[1];
      hi = pim[1];
#pragma unroll
      for (int k = 2; k <= 4; ++k)
        if (k == D.m) {
          hr = pr[k];
          hi = pim[k];
        }
    } else {
      amp = D.A_m * (1.0 + D.a_lm * tau) * dec;
      const double phase = D.phm + D.w_rd * tau + D.dw * H.tau_d * (1.0 - dec);
      freq = D.w_rd + D.dw * dec;
      double s, c;
      sincos(phase, &s, &c);
      hr = c;
      hi = -s;
    }
    const double f = freq * (0.5 / kPi);
    amp *= f > kFhi1 ? win * planck_down_f(f) : win;
    if (amp == 0.0) continue;
    if (RAW) {
      const double a = ap * amp;
      acc[j].x = fma(a, hr, acc[j].x);
      acc[j].y = fma(a, hi, acc[j].y);
      continue;
    }
    double ppr, ppi, pxr, pxi;
    if (PREC) {
      double ypr, ypi, ymr, ymi;
      const int lm = D.l * 8 + D.m;
      if (lm == 2 * 8 + 2) ylmd_pair<2, 2>(P, D, ypr, ypi, ymr, ymi);
      else if (lm == 2 * 8 + 1) ylmd_pair<2, 1>(P, D, ypr, ypi, ymr, ymi);
      else if (lm == 3 * 8 + 3) ylmd_pair<3, 3>(P, D, ypr, ypi, ymr, ymi);
      else if (lm == 3 * 8 + 2) ylmd_pair<3, 2>(P, D, ypr, ypi, ymr, ymi);
      else ylmd_pair<4, 4>(P, D, ypr, ypi, ymr, ymi);
      const double sg = (D.l & 1) ? -1.0 : 1.0, c2 = H.c2psi, s2 = H.s2psi;
      const double Pr = c2 * ypr - s2 * ypi, Pi = c2 * ypi + s2 * ypr;
      const double Qr = c2 * ymr - s2 * ymi, Qi = c2 * ymi + s2 * ymr;
      ppr = Pr + sg * Qr;
      ppi = Pi - sg * Qi;
      pxr = -(Pi + sg * Qi);
      pxi = Pr - sg * Qr;
    } else {
      ppr = D.ppr; ppi = D.ppi; pxr = D.pxr; pxi = D.pxi;
    }
    const double wr = amp * (ap * ppr + ax * pxr), wi = amp * (ap * ppi + ax * pxi);
    acc[j].x += hr * wr - hi * wi;
    acc[j].y += hr * wi + hi * wr;
  }
}

// ---------------------------------------------------------------------------
// node kernels: one thread per (node, walker), blocks of consecutive nodes of
// one walker (the walker's record is read by every thread of the block).
//   mode 0: out[((b nm + j) 3 + c) ldw + w] = conj(C_j(t_b)) X_jc - z0[(b nm + j) 3 + c]
//   mode 1: out[(b nm + j) 3 + c] = conj(C_j(t_b)) X_jc                (fiducial)
//   mode 2: x0[c n + i_b] = Re sum_j X_jc                             (fiducial)
// ---------------------------------------------------------------------------

template <typename C2>
__device__ __forceinline__ void add_channel(int c, const C2 (&t)[kNMode], C2 (&ax)[kNMode],
                                            C2 (&ay)[kNMode], C2 (&az)[kNMode]) {
#pragma unroll
  for (int j = 0; j < kNMode; ++j) {
    if (c == 0) { ax[j].x += t[j].x; ax[j].y += t[j].y; }
    else if (c == 1) { ay[j].x += t[j].x; ay[j].y += t[j].y; }
    else { az[j].x += t[j].x; az[j].y += t[j].y; }
  }
}

template <typename OutT>
__device__ __forceinline__ OutT to_out(double x, double y);
template <>
__device__ __forceinline__ double2 to_out<double2>(double x, double y) { return make_double2(x, y); }
template <>
__device__ __forceinline__ float2 to_out<float2>(double x, double y) {
  return make_float2((float)x, (float)y);
}

// FP64 throughout; OutT is double2 for FP64 contexts and float2 for mixed ones
// (the node differences are rounded once, after the subtraction)
template <typename OutT, bool PREC>
__global__ void __launch_bounds__(kNodeThreads) het_nodes_kernel(
    const WalkerRec* __restrict__ walkers, const HetGeom64* __restrict__ g, int ntc,
    const int64_t* __restrict__ nodes, int64_t start, int64_t B, int64_t n, double t0,
    double t_end, const double2* __restrict__ car, int mode,
    const double2* __restrict__ z0, void* __restrict__ outv, int ldw,
    double* __restrict__ x0) {
  __shared__ HetWalker H;
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int w = blockIdx.y;
  const WalkerRec& W = walkers[w];
  if (threadIdx.x == 0) het_walker_fill(W, H);
  __syncthreads();
  if (b >= B) return;
  double2 ax[kNMode], ay[kNMode], az[kNMode];
#pragma unroll
  for (int j = 0; j < kNMode; ++j) ax[j] = ay[j] = az[j] = make_double2(0.0, 0.0);
  const double k0 = W.k[0], k1 = W.k[1], k2 = W.k[2];
  // aligned spins: per channel, S1_j = sum_terms ap dh_j and S2_j = sum_terms ax dh_j
  // (dh = h(t_s) - h(t_r)); the constant angular weights are applied once per
  // channel: X_j = (P + sg conj Q)_j S1_j + i (P - sg conj Q)_j S2_j
  double2 s1[kNMode], s2[kNMode];
#pragma unroll
  for (int j = 0; j < kNMode; ++j) s1[j] = s2[j] = make_double2(0.0, 0.0);
  for (int q = 0; q < 3 * ntc; ++q) {
    const HetGeom64 G = g[(int64_t)q * B + b];
    if (G.sign != 0.0) {
      const double kr = k0 * G.rr[0] + k1 * G.rr[1] + k2 * G.rr[2];
      const double ks = k0 * G.rs[0] + k1 * G.rs[1] + k2 * G.rs[2];
      const double kn = k0 * G.n[0] + k1 * G.n[1] + k2 * G.n[2];
      const double un = dot3(W.u, G.n), vn = dot3(W.v, G.n);
      const double den = 0.5 * G.sign * rcp_nr(1.0 - kn);
      const double ap = den * (un * un - vn * vn), axx = den * 2.0 * un * vn;
      double2 tmp[kNMode];
#pragma unroll
      for (int j = 0; j < kNMode; ++j) tmp[j] = make_double2(0.0, 0.0);
      if (PREC) {
        modes_fp64<PREC>(H, W, G.tp - G.L - ks, t0, t_end, ap, axx, tmp);
        modes_fp64<PREC>(H, W, G.tp - kr, t0, t_end, -ap, -axx, tmp);
        add_channel(q / ntc, tmp, ax, ay, az);
      } else {
        modes_fp64<PREC, true>(H, W, G.tp - G.L - ks, t0, t_end, 1.0, 0.0, tmp);
        modes_fp64<PREC, true>(H, W, G.tp - kr, t0, t_end, -1.0, 0.0, tmp);
#pragma unroll
        for (int j = 0; j < kNMode; ++j) {
          s1[j].x = fma(ap, tmp[j].x, s1[j].x);
          s1[j].y = fma(ap, tmp[j].y, s1[j].y);
          s2[j].x = fma(axx, tmp[j].x, s2[j].x);
          s2[j].y = fma(axx, tmp[j].y, s2[j].y);
        }
      }
    }
    if (!PREC && (q + 1) % ntc == 0) {             // end of channel q / ntc
      double2 t2[kNMode];
#pragma unroll
      for (int j = 0; j < kNMode; ++j) {
        t2[j] = make_double2(0.0, 0.0);
        if (j < H.nmode) {
          const HetMode& D = H.mode[j];
          t2[j].x = D.ppr * s1[j].x - D.ppi * s1[j].y + D.pxr * s2[j].x - D.pxi * s2[j].y;
          t2[j].y = D.ppr * s1[j].y + D.ppi * s1[j].x + D.pxr * s2[j].y + D.pxi * s2[j].x;
        }
        s1[j] = s2[j] = make_double2(0.0, 0.0);
      }
      add_channel(q / ntc, t2, ax, ay, az);
    }
  }
  const int64_t ib = nodes ? nodes[b] : start + b;
  const int nm = H.nmode;
  const double r2 = 0.70710678118654752440, r6 = 0.40824829046386301637,
               r3 = 0.57735026918962576451;
  double sum[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < kNMode; ++j) {
    if (j >= nm) continue;
    const double2 X = ax[j], Y = ay[j], Z = az[j];
    const double2 aet[3] = {make_double2((Z.x - X.x) * r2, (Z.y - X.y) * r2),
                            make_double2((X.x - 2.0 * Y.x + Z.x) * r6, (X.y - 2.0 * Y.y + Z.y) * r6),
                            make_double2((X.x + Y.x + Z.x) * r3, (X.y + Y.y + Z.y) * r3)};
    if (mode == 2) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sum[c] += aet[c].x;
      continue;
    }
    const double2 C = car[ib * nm + j];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // conj(C) * aet
      const double vr = C.x * aet[c].x + C.y * aet[c].y, vi = C.x * aet[c].y - C.y * aet[c].x;
      const int64_t o = (b * nm + j) * 3 + c;
      if (mode == 1) {
        ((double2*)outv)[o] = make_double2(vr, vi);
      } else {
        const double2 f = z0[o];
        ((OutT*)outv)[o * ldw + w] = to_out<OutT>(vr - f.x, vi - f.y);
      }
    }
  }
  if (mode == 2)
    for (int c = 0; c < 3; ++c) x0[c * n + ib] = sum[c];
}

// ---------------------------------------------------------------------------
// expansion: r[c][i][ldr] = base[c][i] + Re sum_j C_j(i) sum_q w_q(i) dZ_j,a+q,
// the cubic Lagrange polynomial through the nodes a .. a + 3 around sample i
// (a = min(max(b - 1, 0), B - 4), b the node interval holding i).  Lane =
// walker; each warp a run of `chunk` consecutive samples, the four nodes'
// values kept in registers while the interval does not change.
// ---------------------------------------------------------------------------

constexpr int kExpandWarps = 4;       // warps per block of the expansion
constexpr int kExpandMinBlocks = 4;   // resident blocks per SM it is compiled for

template <typename R, typename C2, int NM>
__global__ void __launch_bounds__(32 * kExpandWarps, kExpandMinBlocks) het_expand_kernel(
    int64_t n, int chunk, const int32_t* __restrict__ bin, const int64_t* __restrict__ nodes,
    int B, const C2* __restrict__ car, const R* __restrict__ base, const C2* __restrict__ dz,
    int ldz, R* __restrict__ r, int ldr, int W) {
  const int w = blockIdx.y * 32 + threadIdx.x;
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.y + threadIdx.y) * chunk;
  if (i0 >= n) return;
  const int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
  // one channel at a time, so that only its modes' four node values occupy
  // registers.  Lagrange form: the weights of a sample within its interval
  // stay O(1), so FP32 rounding stays at ~1e-7 of the node values even where
  // an envelope far from the fiducial's is not smooth (the Newton form's
  // divided differences are not bounded there and lose more)
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    int cur = -1;
    C2 z[NM][4];
    R xs[4], dinv[4];
    for (int64_t i = i0; i < i1; ++i) {
      const int b = bin[i];
      if (b != cur) {
        cur = b;
        int a = b - 1 < 0 ? 0 : b - 1;
        a = a > B - 4 ? B - 4 : a;
        // 32-bit sample indices (n < 2^24): a 64-bit integer conversion would
        // run on the FP64 pipe
#pragma unroll
        for (int q = 0; q < 4; ++q) xs[q] = (R)(int)nodes[a + q];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          R den = R(1);
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (t != q) den *= xs[q] - xs[t];
          dinv[q] = R(1) / den;
        }
#pragma unroll
        for (int j = 0; j < NM; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            z[j][q] = dz[(((int64_t)(a + q) * NM + j) * 3 + c) * ldz + w];
      }
      const R xi = (R)(int)i;
      const R e0 = xi - xs[0], e1 = xi - xs[1], e2 = xi - xs[2], e3 = xi - xs[3];
      const R e01 = e0 * e1, e23 = e2 * e3;
      const R wq[4] = {e1 * e23 * dinv[0], e0 * e23 * dinv[1], e01 * e3 * dinv[2],
                       e01 * e2 * dinv[3]};
      R acc = base[c * n + i];
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        const C2 cj = car[i * NM + j];
        R er = R(0), ei = R(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          er += wq[q] * z[j][q].x;
          ei += wq[q] * z[j][q].y;
        }
        acc += cj.x * er - cj.y * ei;
      }
      if (w < W) r[(c * n + i) * ldr + w] = acc;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct HetState {
  int64_t B;
  int nm, ntc;
  int64_t* nodes;          // [B]
  int32_t* bin;            // [n]
  HetTerms* terms;         // device copy
  HetGeom64* g64;          // [3 ntc][max(B, kX0Chunk)]
  double2* car64;          // [n][nm]
  float2* car32;           // [n][nm]
  double* x0;              // [3][n] FP64
  float* x0f;              // [3][n] X0 rounded to FP32
  double* base64;          // [3][n] X0 - data
  float* base32;           // [3][n]
  double2* z0;             // [B][nm][3] the fiducial's node values (FP64)
  void* dz;                // [B][nm][3][wmax_pad] complex
  WalkerRec* fid;          // [1]
  double* theta0;          // [15]
  int data_version;        // version of the data in base64 / base32 (-1: none)
};

void free_het(lisa_td_ctx* c) {
  HetState* h = (HetState*)c->het;
  if (!h) return;
  void* ptrs[] = {h->nodes, h->bin, h->terms, h->g64, h->car64, h->car32, h->x0,
                  h->x0f, h->base64, h->base32, h->z0, h->dz, h->fid, h->theta0};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free(h);
  c->het = nullptr;
}

namespace {

inline int pad32(int w) { return (w + 31) / 32 * 32; }

HetTerms build_terms(int gen, int* ntc) {
  const TdiTable tab = build_tdi_table(gen);
  HetTerms T;
  memset(&T, 0, sizeof(T));
  int cnt[3] = {0, 0, 0};
  for (int j = 0; j < kNLink; ++j)
    for (int k = 0; k < tab.nterm[j]; ++k) {
      const TdiTerm& t = tab.term[j][k];
      HetTerm& h = T.term[t.chan][cnt[t.chan]++];
      h.t = t;
      memcpy(h.chain, tab.chain[j][k], sizeof(h.chain));
      h.link = j;
      h.sign = (double)t.sign;
    }
  T.ntc = cnt[0];
  *ntc = cnt[0];
  return T;
}

template <typename OutT, bool PREC>
void nodes_launch(const lisa_td_ctx* c, const HetState* h, const WalkerRec* walkers,
                  const int64_t* nodes, int64_t start, int64_t B, int W, int mode, void* out,
                  int ldw, double* x0, cudaStream_t s) {
  dim3 grid((unsigned)((B + kNodeThreads - 1) / kNodeThreads), (unsigned)W);
  const double t_end = c->cfg.t0 + (double)(c->n - 1) * c->cfg.dt;
  het_nodes_kernel<OutT, PREC><<<grid, kNodeThreads, 0, s>>>(
      walkers, h->g64, h->ntc, nodes, start, B, c->n, c->cfg.t0, t_end, h->car64, mode, h->z0,
      out, ldw, x0);
}

// node kernel over the B nodes (mode 0 / 1), or over the samples start ..
// start + B - 1 with the geometry built for them (mode 2, FP64 output)
cudaError_t launch_nodes_ex(const lisa_td_ctx* c, const HetState* h, const WalkerRec* walkers,
                            const int64_t* nodes, int64_t start, int64_t B, int W, int mode,
                            void* out, int ldw, double* x0, cudaStream_t s) {
  const bool f64 = c->cfg.precision == 0 || mode != 0;
  if (c->cfg.precessing) {
    if (f64) nodes_launch<double2, true>(c, h, walkers, nodes, start, B, W, mode, out, ldw, x0, s);
    else nodes_launch<float2, true>(c, h, walkers, nodes, start, B, W, mode, out, ldw, x0, s);
  } else {
    if (f64) nodes_launch<double2, false>(c, h, walkers, nodes, start, B, W, mode, out, ldw, x0, s);
    else nodes_launch<float2, false>(c, h, walkers, nodes, start, B, W, mode, out, ldw, x0, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_nodes(const lisa_td_ctx* c, const HetState* h, const WalkerRec* walkers,
                         int W, int mode, void* out, int ldw, cudaStream_t s) {
  return launch_nodes_ex(c, h, walkers, h->nodes, 0, h->B, W, mode, out, ldw, nullptr, s);
}

template <typename R, typename C2>
cudaError_t launch_expand_t(const lisa_td_ctx* c, const HetState* h, const C2* car,
                            const R* base, const C2* dz, int ldz, R* r, int ldr, int W, int Wgrid,
                            cudaStream_t s) {
  const int chunk = 128;
  dim3 block(32, kExpandWarps);
  dim3 grid((unsigned)((c->n + kExpandWarps * chunk - 1) / (kExpandWarps * chunk)),
            (unsigned)(Wgrid / 32));
#define HET_EXPAND(NM)                                                                        \
  het_expand_kernel<R, C2, NM><<<grid, block, 0, s>>>(c->n, chunk, h->bin, h->nodes,            \
                                                      (int)h->B, car, base, dz, ldz, r, ldr, W)
  switch (h->nm) {
    case 1: HET_EXPAND(1); break;
    case 2: HET_EXPAND(2); break;
    case 3: HET_EXPAND(3); break;
    case 4: HET_EXPAND(4); break;
    default: HET_EXPAND(5); break;
  }
#undef HET_EXPAND
  return cudaGetLastError();
}

// model (base = X0) or residual (base = X0 - d) of Wgrid padded walkers into r
cudaError_t launch_expand(const lisa_td_ctx* c, const HetState* h, bool resid, void* r, int ldr,
                          int W, int Wgrid, cudaStream_t s) {
  if (c->cfg.precision == 0)
    return launch_expand_t<double, double2>(c, h, h->car64, resid ? h->base64 : h->x0,
                                            (const double2*)h->dz, Wgrid, (double*)r, ldr, W,
                                            Wgrid, s);
  return launch_expand_t<float, float2>(c, h, h->car32, resid ? h->base32 : h->x0f,
                                        (const float2*)h->dz, Wgrid, (float*)r, ldr, W, Wgrid, s);
}

cudaError_t refresh_base(lisa_td_ctx* c, HetState* h, cudaStream_t s) {
  if (h->data_version == c->data_version) return cudaSuccess;
  const int64_t m = 3 * c->n;
  het_base_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, h->x0, c->data64, h->base64,
                                                              h->base32, nullptr);
  h->data_version = c->data_version;
  return cudaGetLastError();
}

// prep + node differences of W walkers (padded to Wp) into h->dz
cudaError_t run_nodes(lisa_td_ctx* c, HetState* h, const double* params, int W, int Wp,
                      cudaStream_t s) {
  cudaError_t e = launch_prep(c, params, W, Wp, s);
  if (e == cudaSuccess) e = launch_nodes(c, h, c->walkers, Wp, 0, h->dz, Wp, s);
  return e;
}

}  // namespace

}  // namespace lisa

namespace lisa {
const char* const kHetStageRange[7] = {"lisa_td_het/prep", "lisa_td_het/nodes",
                                       "lisa_td_het/expand", "lisa_td_het/empty",
                                       "lisa_td_het/fft_pass1", "lisa_td_het/fft_pass2_norm",
                                       "lisa_td_het/reduce"};
}  // namespace lisa

extern "C" {

int lisa_td_het_setup(lisa_td_ctx* c, const double* theta0_host, const int64_t* nodes_host,
                      int64_t B, void* stream) {
  using namespace lisa;
  if (!c || !theta0_host || !nodes_host)
    return report_error(LISA_TD_EINVAL, "lisa_td_het_setup: NULL argument");
  for (int k = 0; k < kNPar; ++k)
    if (!isfinite(theta0_host[k]))
      return report_error(LISA_TD_EINVAL, "lisa_td_het_setup: fiducial entry %d is not finite", k);
  if (B < 4 || nodes_host[0] != 0 || nodes_host[B - 1] != c->n - 1)
    return report_error(LISA_TD_EINVAL,
                        "lisa_td_het_setup: nodes must hold at least 4 indices from 0 to n - 1");
  for (int64_t b = 1; b < B; ++b)
    if (nodes_host[b] <= nodes_host[b - 1])
      return report_error(LISA_TD_EINVAL, "lisa_td_het_setup: nodes must rise strictly (index %lld)",
                          (long long)b);
  if (B > (int64_t)INT32_MAX / 2)
    return report_error(LISA_TD_ERANGE, "lisa_td_het_setup: too many nodes");
  free_het(c);
  cudaStream_t s = (cudaStream_t)stream;
  HetState* h = (HetState*)calloc(1, sizeof(HetState));
  if (!h) return report_error(LISA_TD_ENOMEM, "lisa_td_het_setup: host allocation failed");
  c->het = h;
  h->B = B;
  h->data_version = -1;
  int ntc = 0;
  const HetTerms terms = build_terms(c->cfg.tdi_gen, &ntc);
  h->ntc = ntc;
  int nm = 0;
  for (int j = 0; j < kNMode; ++j) nm += (c->cfg.mode_mask >> j) & 1;
  h->nm = nm;
  const int64_t n = c->n;
  const size_t cs = 2 * (size_t)c->esize;
  const int64_t grows = B > kX0Chunk ? B : kX0Chunk;
  struct { void** p; size_t bytes; } allocs[] = {
      {(void**)&h->nodes, sizeof(int64_t) * B},
      {(void**)&h->bin, sizeof(int32_t) * n},
      {(void**)&h->terms, sizeof(HetTerms)},
      {(void**)&h->g64, sizeof(HetGeom64) * 3 * ntc * grows},
      {(void**)&h->car64, sizeof(double2) * n * nm},
      {(void**)&h->car32, sizeof(float2) * n * nm},
      {(void**)&h->x0, sizeof(double) * 3 * n},
      {(void**)&h->x0f, sizeof(float) * 3 * n},
      {(void**)&h->base64, sizeof(double) * 3 * n},
      {(void**)&h->base32, sizeof(float) * 3 * n},
      {(void**)&h->z0, sizeof(double2) * B * nm * 3},
      {(void**)&h->dz, cs * B * nm * 3 * (size_t)c->wmax_pad},
      {(void**)&h->fid, sizeof(WalkerRec)},
      {(void**)&h->theta0, sizeof(double) * kNPar},
  };
  for (auto& a : allocs) {
    cudaError_t e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      *a.p = nullptr;
      free_het(c);
      cudaGetLastError();
      return report_error(e == cudaErrorMemoryAllocation ? LISA_TD_ENOMEM : LISA_TD_ECUDA,
                          "lisa_td_het_setup: cudaMalloc: %s", cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaMemcpyAsync(h->nodes, nodes_host, sizeof(int64_t) * B, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->terms, &terms, sizeof(terms), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->theta0, theta0_host, sizeof(double) * kNPar, cudaMemcpyHostToDevice, s);
  // the fiducial's record: the prep kernel writes walker 0 of the workspace
  if (e == cudaSuccess) e = launch_prep(c, h->theta0, 1, 1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->fid, c->walkers, sizeof(WalkerRec), cudaMemcpyDeviceToDevice, s);
  int32_t fstatus = 1;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&fstatus, &h->fid->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && fstatus != 0) {
    free_het(c);
    return report_error(LISA_TD_EINVAL, "lisa_td_het_setup: the fiducial parameters are invalid");
  }
  const unsigned gb = (unsigned)((n + 255) / 256);
  if (e == cudaSuccess) {
    het_carrier_kernel<<<gb, 256, 0, s>>>(h->fid, n, c->cfg.t0, c->cfg.dt, h->car64, h->car32);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    het_bin_kernel<<<gb, 256, 0, s>>>(h->nodes, B, n, h->bin);
    e = cudaGetLastError();
  }
  // X0: the fiducial's continuous-time response at every sample, FP64, in chunks
  for (int64_t a = 0; a < n && e == cudaSuccess; a += kX0Chunk) {
    const int64_t cnt = n - a < kX0Chunk ? n - a : kX0Chunk;
    dim3 gg((unsigned)((cnt + 127) / 128), (unsigned)(3 * ntc));
    het_geom_kernel<<<gg, 128, 0, s>>>(c->orb64, n, c->cfg.t0, c->cfg.dt, h->terms, nullptr, a,
                                       cnt, c->cfg.tdi_nested, h->g64);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    e = launch_nodes_ex(c, h, h->fid, nullptr, a, cnt, 1, 2, nullptr, 0, h->x0, s);
  }
  if (e == cudaSuccess) {
    const int64_t m = 3 * n;
    het_base_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, h->x0, nullptr, nullptr,
                                                                nullptr, h->x0f);
    e = cudaGetLastError();
  }
  // the nodes' geometry, then the fiducial's node values z0
  if (e == cudaSuccess) {
    dim3 gg((unsigned)((B + 127) / 128), (unsigned)(3 * ntc));
    het_geom_kernel<<<gg, 128, 0, s>>>(c->orb64, n, c->cfg.t0, c->cfg.dt, h->terms, h->nodes, 0,
                                       B, c->cfg.tdi_nested, h->g64);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_nodes(c, h, h->fid, 1, 1, h->z0, 0, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_het(c);
    return report_error(LISA_TD_ECUDA, "lisa_td_het_setup: %s", cudaGetErrorString(e));
  }
  return LISA_TD_OK;
}

static int het_check(lisa_td_ctx* c, const void* a, const void* b, int32_t W, const char* who) {
  if (!c || !a || !b) return lisa::report_error(LISA_TD_EINVAL, "%s: NULL argument", who);
  if (!c->het) return lisa::report_error(LISA_TD_EINVAL, "%s: lisa_td_het_setup has not been called", who);
  if (W < 1) return lisa::report_error(LISA_TD_EINVAL, "%s: W must be >= 1", who);
  if (W > c->cfg.max_walkers)
    return lisa::report_error(LISA_TD_ERANGE, "%s: W=%d above max_walkers=%d", who, W, c->cfg.max_walkers);
  return LISA_TD_OK;
}

int lisa_td_het_loglike(lisa_td_ctx* c, const double* params_dev, int32_t W, double* logl_dev,
                        int32_t* status_dev, void* stream) {
  using namespace lisa;
  int rc = het_check(c, params_dev, logl_dev, W, "lisa_td_het_loglike");
  if (rc) return rc;
  if (!c->has_data) return report_error(LISA_TD_EINVAL, "lisa_td_het_loglike: lisa_td_set_data has not been called");
  HetState* h = (HetState*)c->het;
  cudaStream_t s = (cudaStream_t)stream;
  const int Wp = pad32(W);
  cudaEvent_t* ev = nullptr;
  if (c->prof_on && c->prof_calls < LISA_TD_PROF_CALLS)
    ev = c->prof_ev + (size_t)(c->prof_calls++) * (LISA_TD_NSTAGE + 1);
  cudaError_t e = refresh_base(c, h, s);
#define STAGE(k, call)                                                   \
  do {                                                                   \
    TraceRange range_(kHetStageRange[k]);                                \
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[k], s);           \
    if (e == cudaSuccess) e = (call);                                    \
  } while (0)
  STAGE(0, launch_prep(c, params_dev, W, Wp, s));
  STAGE(1, launch_nodes(c, h, c->walkers, Wp, 0, h->dz, Wp, s));
  STAGE(2, launch_expand(c, h, true, c->r, Wp, Wp, Wp, s));
  STAGE(3, cudaSuccess);
  STAGE(4, launch_fft_pass1(c, Wp, c->r, s));
  STAGE(5, launch_fft_pass2(c, Wp, s));
  STAGE(6, launch_reduce(c, W, Wp, logl_dev, status_dev, s));
#undef STAGE
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[LISA_TD_NSTAGE], s);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "lisa_td_het_loglike: %s", cudaGetErrorString(e));
  return LISA_TD_OK;
}

int lisa_td_het_deltas(lisa_td_ctx* c, const double* params_dev, int32_t W, void* dz_dev,
                       void* stream) {
  using namespace lisa;
  int rc = het_check(c, params_dev, dz_dev, W, "lisa_td_het_deltas");
  if (rc) return rc;
  HetState* h = (HetState*)c->het;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_prep(c, params_dev, W, pad32(W), s);
  if (e == cudaSuccess) e = launch_nodes(c, h, c->walkers, W, 0, dz_dev, W, s);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "lisa_td_het_deltas: %s", cudaGetErrorString(e));
  return LISA_TD_OK;
}

int lisa_td_het_aet(lisa_td_ctx* c, const double* params_dev, int32_t W, void* aet_dev,
                    void* stream) {
  using namespace lisa;
  int rc = het_check(c, params_dev, aet_dev, W, "lisa_td_het_aet");
  if (rc) return rc;
  HetState* h = (HetState*)c->het;
  cudaStream_t s = (cudaStream_t)stream;
  const int Wp = pad32(W);
  cudaError_t e = run_nodes(c, h, params_dev, W, Wp, s);
  if (e == cudaSuccess) e = launch_expand(c, h, false, aet_dev, W, W, Wp, s);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "lisa_td_het_aet: %s", cudaGetErrorString(e));
  return LISA_TD_OK;
}

}  // extern "C"
