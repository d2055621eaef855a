// Per-walker constants of the stand-in waveform, source frame and precession
// (Sec. II.A, II.B).  One thread per walker, FP64; walkers W..Wpad-1 repeat
// walker 0 so that padded lanes of later kernels compute finite values.
#include <math.h>

#include "internal.h"
#include "standin.cuh"

namespace lisa {

namespace {

__device__ void mode_coeff(int j, double nu, double delta, int& l, int& m, double& coef,
                           int& extra, double& rd_ratio) {
  switch (j) {
    case 0: l = 2; m = 2; coef = 1.0; extra = 0; rd_ratio = 1.0; break;
    case 1: l = 2; m = 1; coef = delta / 3.0; extra = 1; rd_ratio = 0.75; break;
    case 2: l = 3; m = 3; coef = 0.75 * sqrt(15.0 / 14.0) * delta; extra = 1; rd_ratio = 1.55; break;
    case 3: l = 3; m = 2; coef = sqrt(5.0 / 7.0) * (1.0 - 3.0 * nu) / 3.0; extra = 2; rd_ratio = 1.25; break;
    default: l = 4; m = 4; coef = 8.0 / 9.0 * sqrt(5.0 / 7.0) * (1.0 - 3.0 * nu); extra = 2; rd_ratio = 2.1; break;
  }
}

__global__ void prep_kernel(const double* __restrict__ params, int W, int Wpad, double t0,
                            double dt, const int64_t* __restrict__ woff, int mode_mask,
                            int precessing, WalkerRec* __restrict__ out) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wpad) return;
  int src_w = w < W ? w : 0;
  double p[kNPar];
  bool ok = true;
  for (int j = 0; j < kNPar; ++j) {
    p[j] = params[(int64_t)src_w * kNPar + j];
    ok = ok && isfinite(p[j]);
  }
  WalkerRec R;
  memset(&R, 0, sizeof(R));
  double m1 = p[0], m2 = p[1];
  double a1 = p[2], th1 = p[3], ph1 = p[4], a2 = p[5], th2 = p[6], ph2 = p[7];
  if (m2 > m1) {                                   // m1 >= m2 by swapping the bodies
    double t;
    t = m1; m1 = m2; m2 = t;
    t = a1; a1 = a2; a2 = t;
    t = th1; th1 = th2; th2 = t;
    t = ph1; ph1 = ph2; ph2 = t;
  }
  ok = ok && m1 > 0.0 && m2 > 0.0 && p[8] > 0.0 && fabs(a1) < 1.0 && fabs(a2) < 1.0;
  if (precessing) ok = ok && a1 >= 0.0 && a2 >= 0.0;
  if (!ok) {                                       // harmless finite stand-in values
    m1 = m2 = 5.0e5; a1 = a2 = 0.0; th1 = th2 = ph1 = ph2 = 0.0;
    p[8] = 1.0; p[14] = 0.0;
  }
  double mt = m1 + m2;
  R.M = mt * kTsun;
  R.nu = m1 * m2 / (mt * mt);
  R.delta = (m1 - m2) / mt;
  double chi1 = precessing ? a1 * cos(th1) : a1;
  double chi2 = precessing ? a2 * cos(th2) : a2;
  R.chi = (m1 * chi1 + m2 * chi2) / mt;
  R.c1 = 743.0 / 2688.0 + 11.0 * R.nu / 32.0;
  R.cs = kCSpin * R.chi;
  R.tc = p[14];
  R.um = pow(kXMerge, 0.125);
  R.tm = R.tc - 5.0 * R.M * kXMerge / R.nu;
  double af = 0.686 + 0.25 * R.chi;
  double wrd22 = (1.5251 - 1.1568 * pow(1.0 - af, 0.1292)) / R.M;
  double Q = 0.7 + 1.4187 * pow(1.0 - af, -0.4990);
  R.tau_d = 2.0 * Q / wrd22;
  double us = pow(8.0 * kPi * R.M * kFmin, -1.0 / 3.0);
  double us2 = us * us, us4 = us2 * us2;
  R.t_start = R.tc - 5.0 * R.M * us4 * us4 / R.nu;
  // the start taper begins at the later of the signal start and the start of
  // the walker's window (the grid start, or its own window in ragged batches)
  const double t0w = t0 + (woff ? (double)woff[w] * dt : 0.0);   // the window's first sample
  R.t_a = fmax(t0w, R.t_start);
  insp_omega_phase(R, R.um, R.om_m, R.ph_m);
  double omdot = insp_omega_dot(R, R.um);
  double D = p[8] * kGpcSec;
  double iota = p[9], phr = p[10], beta = p[11], lam = p[12], psi = p[13];

  // aligned spherical harmonics through the quaternion of R(phi_ref, iota, 0)
  double qy[4];
  quat_euler(phr, iota, 0.0, qy);
  int nm = 0;
  for (int j = 0; j < kNMode; ++j) {
    if (!((mode_mask >> j) & 1)) continue;
    int l, m, extra;
    double coef, ratio;
    mode_coeff(j, R.nu, R.delta, l, m, coef, extra, ratio);
    ModeRec& M = R.mode[nm++];
    M.l = l;
    M.m = m;
    M.pref = R.M * R.nu / D * 8.0 * sqrt(kPi / 5.0) * coef;
    M.p = (2.0 + extra) / 3.0;
    M.A_m = M.pref * pow(R.M * R.om_m, M.p);
    M.a_lm = M.p * omdot / R.om_m + 1.0 / R.tau_d;
    M.w_rd = ratio * wrd22;
    cplx<double> yp = ylm_from_quat<double>(l, m, qy);
    cplx<double> ym = ylm_from_quat<double>(l, -m, qy);
    M.Yp_re = yp.re; M.Yp_im = yp.im;
    M.Ym_re = ym.re; M.Ym_im = ym.im;
  }
  R.nmode = nm;

  // source frame (Sec. II.B): propagation vector k, polarisation vectors u, v
  double cb = cos(beta), sb = sin(beta), cl = cos(lam), sl = sin(lam);
  R.k[0] = -cb * cl; R.k[1] = -cb * sl; R.k[2] = -sb;
  R.v[0] = -sb * cl; R.v[1] = -sb * sl; R.v[2] = cb;
  R.u[0] = sl;       R.u[1] = -cl;      R.u[2] = 0.0;
  R.c2psi = cos(2.0 * psi);
  R.s2psi = sin(2.0 * psi);

  // precession stand-in (single spin): S, tilt, reference values, J -> L0
  R.S = a1 * (m1 / mt) * (m1 / mt);
  R.ctilt = cos(th1);
  R.stilt = sin(th1);
  R.kp = 2.0 + 1.5 * m2 / m1;
  R.u_ref = us;
  double Sc = R.S * R.ctilt, b = R.S * R.stilt;
  double aref = 2.0 * R.nu * us + Sc;
  R.G_ref = prec_G(aref, b, Sc);
  R.gamma_ref = kPi - ph1;
  double beta_ref = atan2(b, aref);
  // inverse of q(alpha0, beta0, gamma0), the J -> L0 rotation with
  // (alpha0, beta0, gamma0) = (phi1 - pi, -beta_ref, 0), composed with
  // q(phi_ref, iota, 0)
  double q0[4], q0i[4];
  quat_euler(ph1 - kPi, -beta_ref, 0.0, q0);
  q0i[0] = q0[0]; q0i[1] = -q0[1]; q0i[2] = -q0[2]; q0i[3] = -q0[3];
  qmul(q0i, qy, R.q03);
  R.status = ok ? 0 : 1;

  // ---- mixed-precision copy ----
  MixRec& X = R.mx;
  X.T = df_from_double(R.tc - t0w);
  X.kap = df_from_double(R.nu / (5.0 * R.M));
  X.A5 = df_from_double(1.0 / R.nu);
  X.A3 = df_from_double((5.0 / 3.0) * R.c1 / R.nu);
  X.A2 = df_from_double(2.5 * R.cs / R.nu);
  X.tm = df_from_double(R.tm - t0w);
  X.tstart = df_from_double(R.t_start - t0w);
  X.ta = df_from_double(R.t_a - t0w);
  X.dt = df_from_double(dt);
  X.c1 = (float)R.c1;
  X.cs = (float)R.cs;
  X.invM = (float)(1.0 / R.M);
  X.tau_d = (float)R.tau_d;
  X.c2psi = (float)R.c2psi;
  X.s2psi = (float)R.s2psi;
  for (int d = 0; d < 3; ++d) {
    X.k[d] = (float)R.k[d];
    X.u[d] = (float)R.u[d];
    X.v[d] = (float)R.v[d];
  }
  X.aucb = (float)(kAUSec * cos(beta));
  X.S = (float)R.S;
  X.Sc = (float)Sc;
  X.b = (float)b;
  X.kp = (float)R.kp;
  {
    // G_ref split: the double-float part excludes the asinh term, which the
    // kernel evaluates in FP32 with the asinh term of the reference folded in
    double Jr = sqrt(aref * aref + b * b);
    double ashr = b > 0.0 ? asinh(aref / b) : 0.0;
    X.Gref = df_from_double(Jr * Jr * Jr / 3.0 - Sc * 0.5 * aref * Jr - Sc * 0.5 * b * b * ashr);
  }
  X.alpha_c = (float)(-(5.0 * R.kp / (32.0 * R.nu * R.nu * R.nu)));
  {
    double C = 5.0 * R.kp / (8.0 * R.nu);
    double ur = R.u_ref;
    X.g3 = df_from_double(C * 2.0 * R.nu / 3.0);
    X.g2 = df_from_double(C * 0.5 * Sc);
    X.g0 = df_from_double(R.gamma_ref - C * (2.0 * R.nu * ur * ur * ur / 3.0 + 0.5 * Sc * ur * ur));
  }
  X.twonu = (float)(2.0 * R.nu);
  X.um = (float)R.um;
  for (int d = 0; d < 4; ++d) X.q03[d] = (float)R.q03[d];
  X.nmode = R.nmode;
  for (int j = 0; j < R.nmode; ++j) {
    const ModeRec& Md = R.mode[j];
    MixMode& Q = X.mode[j];
    Q.pref = (float)Md.pref;
    Q.pw = (int)lround(3.0 * Md.p) - 2;
    Q.A_m = (float)Md.A_m;
    Q.a_lm = (float)Md.a_lm;
    Q.w_rd = (float)Md.w_rd;
    Q.dw = (float)(Md.m * R.om_m - Md.w_rd);
    Q.ph0 = (float)remainder(Md.m * R.ph_m, 2.0 * kPi);
    Q.yp_re = (float)Md.Yp_re;
    Q.yp_im = (float)Md.Yp_im;
    Q.ym_re = (float)Md.Ym_re;
    Q.ym_im = (float)Md.Ym_im;
    Q.l = Md.l;
    Q.m = Md.m;
    for (int sg = 0; sg < 2; ++sg) {
      const int l = Md.l, mm = sg ? -Md.m : Md.m;
      const int r0 = mm - 2 > 0 ? mm - 2 : 0;
      const int r1 = (l + mm < l - 2) ? l + mm : l - 2;
      const double pref = sqrt(fact(l + 2) * fact(l - 2) / (fact(l + mm) * fact(l - mm))) *
                          sqrt((2.0 * l + 1.0) / (4.0 * kPi));
      for (int q = 0; q < 3; ++q) {
        const int r = r0 + q;
        Q.yc[sg][q] = r <= r1 ? (float)(binom(l + mm, r) * binom(l - mm, l - 2 - r) *
                                         ((r & 1) ? -1.0 : 1.0) * pref)
                              : 0.0f;
      }
    }
  }
  out[w] = R;
}

}  // namespace

cudaError_t launch_prep(const lisa_td_ctx* c, const double* params, int W, int Wpad,
                        cudaStream_t s) {
  int threads = 64;
  int blocks = (Wpad + threads - 1) / threads;
  prep_kernel<<<blocks, threads, 0, s>>>(params, W, Wpad, c->cfg.t0, c->cfg.dt, c->woff,
                                         c->cfg.mode_mask, c->cfg.precessing, c->walkers);
  return cudaGetLastError();
}

}  // namespace lisa
