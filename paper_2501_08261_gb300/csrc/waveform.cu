// Polarisations h+, hx of the stand-in model on the grid (Sec. II.A), FP64
// path: every sample evaluates the closed forms directly.  Aligned spins use
// the spin-weighted harmonics -2Y_lm(iota, phi_ref); precessing spins use the
// single sum of Eq. (newtwistup) with the quaternion-built D^l_{m,2}.
#include <math.h>

#include "internal.h"
#include "mixed_wave.cuh"
#include "standin.cuh"

namespace lisa {

namespace {

// h+ - i hx (before the psi rotation) at time t, FP64.
__device__ void polar_fp64(const WalkerRec& W, double t, int precessing, double& re,
                           double& im) {
  re = 0.0;
  im = 0.0;
  if (W.status != 0 || t < W.t_start) return;
  double win = planck_up(t, W.t_a, kTaper);
  if (win == 0.0) return;
  bool insp = t < W.tm;
  double u = W.um, om = 0.0, ph = 0.0, tau = 0.0, dec = 1.0;
  if (insp) {
    double x = W.nu * (W.tc - t) / (5.0 * W.M);
    u = sqrt(sqrt(sqrt(x)));
    insp_omega_phase(W, u, om, ph);
  } else {
    tau = t - W.tm;
    dec = exp(-tau / W.tau_d);
  }
  // rotation of the co-precessing modes (precessing) : quaternion q_T
  double qT[4];
  if (precessing) {
    double cbh, sbh, al, ga;
    prec_angles(W, u, cbh, sbh, al, ga);
    double sp, cp, sm, cm;
    sincos(0.5 * (al + ga), &sp, &cp);
    sincos(0.5 * (al - ga), &sm, &cm);
    double q1[4] = {cbh * cp, sbh * sm, -sbh * cm, -cbh * sp};   // q(al, be, ga)^-1
    qmul(q1, W.q03, qT);
  }
  for (int j = 0; j < W.nmode; ++j) {
    const ModeRec& Md = W.mode[j];
    double amp, phase, freq;
    if (insp) {
      amp = Md.pref * pow(W.M * om, Md.p);
      phase = Md.m * ph;
      freq = Md.m * om;
    } else {
      amp = Md.A_m * (1.0 + Md.a_lm * tau) * dec;
      phase = Md.m * W.ph_m + Md.w_rd * tau + (Md.m * W.om_m - Md.w_rd) * W.tau_d * (1.0 - dec);
      freq = Md.w_rd + (Md.m * W.om_m - Md.w_rd) * dec;
    }
    amp *= win * planck_down_f(freq / (2.0 * kPi));
    if (amp == 0.0) continue;
    double s, c;
    sincos(phase, &s, &c);
    double hr = amp * c, hi = -amp * s;                 // h_lm = A e^{-i Phi}
    double sg = (Md.l & 1) ? -1.0 : 1.0;                 // h_{l,-m} = (-1)^l conj(h_lm)
    double ypr, ypi, ymr, ymi;
    if (precessing) {
      cplx<double> a = ylm_from_quat<double>(Md.l, Md.m, qT);
      cplx<double> b = ylm_from_quat<double>(Md.l, -Md.m, qT);
      ypr = a.re; ypi = a.im; ymr = b.re; ymi = b.im;
    } else {
      ypr = Md.Yp_re; ypi = Md.Yp_im; ymr = Md.Ym_re; ymi = Md.Ym_im;
    }
    re += hr * ypr - hi * ypi + sg * (hr * ymr + hi * ymi);
    im += hr * ypi + hi * ypr + sg * (hr * ymi - hi * ymr);
  }
}

__global__ void waveform_fp64_kernel(const WalkerRec* __restrict__ walkers, int64_t n,
                                     double t0, double dt, int precessing, double2* h,
                                     const int64_t* __restrict__ woff) {
  int w = blockIdx.y;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (woff && i < woff[w]) return;             // before the walker's window: never read
  const WalkerRec& W = walkers[w];
  double re, im;
  polar_fp64(W, t0 + (double)i * dt, precessing, re, im);
  // (h+ - i hx) e^{2 i psi}
  double Hr = re * W.c2psi - im * W.s2psi;
  double Hi = re * W.s2psi + im * W.c2psi;
  h[(int64_t)w * n + i] = make_double2(Hr, -Hi);
}

// ---------------------------------------------------------------------------
// Mixed path: the absolute time and the orbital phase in double-float (so the
// phase of a months-long signal keeps ~1e-7 rad), reduced mod 2 pi, then FP32.
// ---------------------------------------------------------------------------

// h+ - i hx before the psi rotation at sample i (time t0 + i dt), mixed precision.
__device__ void polar_mixed(const MixRec& X, int status, int i, int precessing, float& re,
                            float& im) {
  re = 0.0f;
  im = 0.0f;
  if (status != 0) return;
  // t - t0 = i * dt exactly in double-float (i < 2^24: exact in FP32, and a
  // 32-bit conversion keeps the FP64 pipe out of the per-sample work)
  float fi = (float)i;
  df32 t = two_prod(fi, X.dt.hi);
  t = fast_two_sum(t.hi, fmaf(fi, X.dt.lo, t.lo));
  if (df_add(t, {-X.tstart.hi, -X.tstart.lo}).hi < 0.0f) return;
  float xa = df_add(t, {-X.ta.hi, -X.ta.lo}).hi;
  float win = planck_up_f(xa, (float)kTaper);
  if (win == 0.0f) return;
  float tau = df_add(t, {-X.tm.hi, -X.tm.lo}).hi;          // t - t_m
  const bool insp = tau < 0.0f;
  float uf = X.um, Mw = 0.0f, e1r = 1.0f, e1i = 0.0f, dec = 1.0f;
  df32 udf = {X.um, 0.0f};
  if (insp) {
    df32 x = df_mul(X.kap, df_add(X.T, {-t.hi, -t.lo}));
    df32 u = df_sqrt(df_sqrt(df_sqrt(x)));
    df32 u2 = df_mul(u, u);
    df32 ph = df_mul(u2, df_add(df_mul(u, df_add(df_mul(X.A5, u2), X.A3)), X.A2));
    float r = df_mod_2pi(ph);              // phi = -ph; e^{-i phi} = e^{+i r}
    sincosf(r, &e1i, &e1r);
    uf = u.hi;
    udf = u;
    float iu = 1.0f / uf;
    float iu2 = iu * iu, iu3 = iu2 * iu;
    Mw = 0.125f * (iu3 + X.c1 * iu2 * iu3 + X.cs * iu3 * iu3);
  } else {
    dec = __expf(-tau / X.tau_d);
  }
  float v = insp ? cbrtf(Mw) : 0.0f;
  float v2 = v * v;
  float qT[4];
  QPow P;
  if (precessing) {
    // a = 2 nu u + S cos(th1) and G(a) - G_ref in double-float: alpha_c can
    // reach ~400 for q = 8, so G needs more than FP32's 24 bits
    df32 ad = df_add_f(df_mul_f(udf, X.twonu), X.Sc);
    df32 J2 = df_add(df_mul(ad, ad), two_prod(X.b, X.b));
    df32 Jd = df_sqrt(J2);
    float a = ad.hi, J = Jd.hi;
    float cb = a / J, sb = X.b / J, cbh, sbh;
    if (cb >= 0.0f) {
      cbh = sqrtf(0.5f * (1.0f + cb));
      sbh = sb / (2.0f * cbh);
    } else {
      sbh = sqrtf(0.5f * (1.0f - cb));
      cbh = sb / (2.0f * sbh);
    }
    float ash = X.b > 0.0f ? asinhf(a / X.b) : 0.0f;
    df32 J3 = df_mul(df_mul(Jd, Jd), Jd);
    df32 G = df_add(df_mul_f(J3, 1.0f / 3.0f), df_mul_f(df_mul(ad, Jd), -0.5f * X.Sc));
    G = df_add(G, {-X.Gref.hi, -X.Gref.lo});
    float al = X.alpha_c * (G.hi + (G.lo - X.Sc * 0.5f * X.b * X.b * ash));
    df32 u2 = df_mul(udf, udf);
    df32 gam = df_add(X.g0, df_add(df_mul(X.g3, df_mul(u2, udf)), df_mul(X.g2, u2)));
    float sp, cp, sm, cm;
    // (alpha +- gamma)/2 with gamma in double-float
    df32 sp2 = df_add_f(gam, al), sm2 = df_add_f({-gam.hi, -gam.lo}, al);
    float hp = df_mod_2pi({0.5f * sp2.hi, 0.5f * sp2.lo});
    float hm = df_mod_2pi({0.5f * sm2.hi, 0.5f * sm2.lo});
    sincosf(hp, &sp, &cp);
    sincosf(hm, &sm, &cm);
    float q1[4] = {cbh * cp, sbh * sm, -sbh * cm, -cbh * sp};   // q(al, be, ga)^-1
    const float* b = X.q03;
    qT[0] = q1[0] * b[0] - q1[1] * b[1] - q1[2] * b[2] - q1[3] * b[3];
    qT[1] = q1[0] * b[1] + q1[1] * b[0] + q1[2] * b[3] - q1[3] * b[2];
    qT[2] = q1[0] * b[2] - q1[1] * b[3] + q1[2] * b[0] + q1[3] * b[1];
    qT[3] = q1[0] * b[3] + q1[1] * b[2] - q1[2] * b[1] + q1[3] * b[0];
    qpow_fill(qT, P);
  }
  // powers e^{-i m phi}, m = 1..4
  float pr[5], pi_[5];
  pr[0] = 1.0f; pi_[0] = 0.0f;
  pr[1] = e1r; pi_[1] = e1i;
#pragma unroll
  for (int m = 2; m <= 4; ++m) {
    pr[m] = pr[m - 1] * e1r - pi_[m - 1] * e1i;
    pi_[m] = pr[m - 1] * e1i + pi_[m - 1] * e1r;
  }
  for (int j = 0; j < X.nmode; ++j) {
    const MixMode& Md = X.mode[j];
    float amp, hr, hi, freq;
    if (insp) {
      float vp = Md.pw == 0 ? v2 : (Md.pw == 1 ? v2 * v : v2 * v2);
      amp = Md.pref * vp;
      freq = (float)Md.m * Mw * X.invM;
      hr = pr[1];
      hi = pi_[1];
#pragma unroll
      for (int k = 2; k <= 4; ++k)                 // register select of e^{-i m phi}
        if (k == Md.m) {
          hr = pr[k];
          hi = pi_[k];
        }
    } else {
      amp = Md.A_m * (1.0f + Md.a_lm * tau) * dec;
      float ph = Md.ph0 + Md.w_rd * tau + Md.dw * X.tau_d * (1.0f - dec);
      freq = Md.w_rd + Md.dw * dec;
      float s, c;
      sincosf(ph, &s, &c);
      hr = c;
      hi = -s;
    }
    amp *= win * planck_down_ff(freq * (float)(0.5 / kPi));
    hr *= amp;
    hi *= amp;
    float sg = (Md.l & 1) ? -1.0f : 1.0f;
    float ypr, ypi, ymr, ymi;
    if (precessing) {
      const int lm = Md.l * 8 + Md.m;
      if (lm == 2 * 8 + 2) ylm_pair<2, 2>(P, Md, ypr, ypi, ymr, ymi);
      else if (lm == 2 * 8 + 1) ylm_pair<2, 1>(P, Md, ypr, ypi, ymr, ymi);
      else if (lm == 3 * 8 + 3) ylm_pair<3, 3>(P, Md, ypr, ypi, ymr, ymi);
      else if (lm == 3 * 8 + 2) ylm_pair<3, 2>(P, Md, ypr, ypi, ymr, ymi);
      else ylm_pair<4, 4>(P, Md, ypr, ypi, ymr, ymi);
    } else {
      ypr = Md.yp_re; ypi = Md.yp_im; ymr = Md.ym_re; ymi = Md.ym_im;
    }
    re += hr * ypr - hi * ypi + sg * (hr * ymr + hi * ymi);
    im += hr * ypi + hi * ypr + sg * (hr * ymi - hi * ymr);
  }
}

__global__ void __launch_bounds__(128) waveform_mixed_kernel(
    const WalkerRec* __restrict__ walkers, int64_t n, int precessing, float2* __restrict__ h,
    const int64_t* __restrict__ woff) {
  const int w = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t lo = woff ? woff[w] : 0;
  if (i < lo) return;                          // before the walker's window: never read
  const MixRec& X = walkers[w].mx;
  float re, im;
  // the double-float time anchors are relative to the window start
  polar_mixed(X, walkers[w].status, (int)(i - lo), precessing, re, im);
  float Hr = re * X.c2psi - im * X.s2psi;
  float Hi = re * X.s2psi + im * X.c2psi;
  h[(int64_t)w * n + i] = make_float2(Hr, -Hi);
}

}  // namespace

cudaError_t launch_waveform(const lisa_td_ctx* c, int W, void* h, cudaStream_t s) {
  dim3 grid((unsigned)((c->n + 127) / 128), (unsigned)W);
  if (c->cfg.precision == 0) {
    waveform_fp64_kernel<<<grid, 128, 0, s>>>(c->walkers, c->n, c->cfg.t0, c->cfg.dt,
                                              c->cfg.precessing, (double2*)h, c->woff);
  } else {
    waveform_mixed_kernel<<<grid, 128, 0, s>>>(c->walkers, c->n, c->cfg.precessing, (float2*)h,
                                               c->woff);
  }
  return cudaGetLastError();
}

}  // namespace lisa
