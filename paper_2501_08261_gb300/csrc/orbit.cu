// Create-time tables (Sec. II.B: the orbit quantities are computed once, not
// per likelihood call):
// spacecraft positions, emission positions and light times per grid sample,
// the PSD weights of the band bins, FFT twiddles, and the data copy.
#include <math.h>

#include "internal.h"

namespace lisa {

namespace {

// Rigid equal-arm model: centre on the 1 AU circle, triangle of side L in a
// plane tilted 60 deg, cartwheeling at -Omega.
__device__ void rigid_pos(int craft, double t, double* r) {
  double a = kOmegaOrb * t;
  double ca = cos(a), sa = sin(a);
  double er[3] = {ca, sa, 0.0}, ephi[3] = {-sa, ca, 0.0};
  double uh[3] = {0.5 * ca, 0.5 * sa, 0.5 * sqrt(3.0)};
  double ang = a - 2.0 * kPi * craft / 3.0;
  double rho = kArmSec / sqrt(3.0);
  double c = cos(ang), s = sin(ang);
  for (int d = 0; d < 3; ++d) r[d] = kAUSec * er[d] + rho * (-c * uh[d] + s * ephi[d]);
}

// Keplerian model: ellipse a = 1 AU, e_k = e0 (1 + eta_k), inclination
// sqrt(3) e_k about the perihelion-normal axis, node 2 pi k / 3.
__device__ void kepler_pos(int craft, double t, double* r) {
  const double e0 = 2.5e9 / (2.0 * sqrt(3.0) * 149597870700.0);
  const double eta = craft == 0 ? 0.0 : (craft == 1 ? 0.01 : -0.01);
  double e = e0 * (1.0 + eta);
  double inc = sqrt(3.0) * e;
  double node = 2.0 * kPi * craft / 3.0;
  double Mean = kOmegaOrb * t - node;
  double E = Mean;
  for (int it = 0; it < 30; ++it) {              // Newton, bounded
    double dE = (E - e * sin(E) - Mean) / (1.0 - e * cos(E));
    E -= dE;
    if (fabs(dE) < 1e-16) break;
  }
  double X = kAUSec * (cos(E) - e);
  double Y = kAUSec * sqrt(1.0 - e * e) * sin(E);
  double xt = X * cos(inc), zt = -X * sin(inc);
  r[0] = xt * cos(node) - Y * sin(node);
  r[1] = xt * sin(node) + Y * cos(node);
  r[2] = zt;
}

// The caller's table (positions [rows][3][3] in light-seconds, row j at
// T0 + j Tdt): centred 8-point Lagrange interpolation in the row index, nodes
// j - 3 .. j + 4 around j = floor((t - T0) / Tdt), the stencil shifted inwards
// at the table's ends.
struct OrbitTableView {
  const double* pos;
  int64_t rows;
  double t0, dt;
};

__device__ void table_pos(const OrbitTableView& T, int craft, double t, double* r) {
  const double x = (t - T.t0) / T.dt;
  int64_t j = (int64_t)floor(x);
  int64_t b = j - 3;
  b = b < 0 ? 0 : (b > T.rows - 8 ? T.rows - 8 : b);
  const double u = x - (double)b;                  // position in node units, nodes 0..7
  double w[8];
  for (int k = 0; k < 8; ++k) {
    double num = 1.0, den = 1.0;
    for (int m = 0; m < 8; ++m) {
      if (m == k) continue;
      num *= u - (double)m;
      den *= (double)(k - m);
    }
    w[k] = num / den;
  }
  for (int d = 0; d < 3; ++d) {
    double acc = 0.0;
    for (int k = 0; k < 8; ++k) acc += w[k] * T.pos[((b + k) * 3 + craft) * 3 + d];
    r[d] = acc;
  }
}

__device__ void craft_pos(int kind, const OrbitTableView& T, int craft, double t, double* r) {
  if (kind == 0) rigid_pos(craft, t, r);
  else if (kind == 1) kepler_pos(craft, t, r);
  else table_pos(T, craft, t, r);
}

__global__ void orbit_kernel(int64_t n, double t0, double dt, int kind, OrbitTableView T,
                             double phase, OrbitRec64* o64, OrbitRec32* o32) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = t0 + (double)i * dt;
  OrbitRec64 R;
  for (int k = 0; k < 3; ++k) craft_pos(kind, T, k, t, R.rr[k]);
  for (int j = 0; j < kNLink; ++j) {
    int sidx = link_sender(j), ridx = link_receiver(j);
    double L, rs[3];
    if (kind == 0) {
      L = kArmSec;
    } else {                                      // light-time fixed point
      craft_pos(kind, T, sidx, t, rs);
      double d0 = R.rr[ridx][0] - rs[0], d1 = R.rr[ridx][1] - rs[1], d2 = R.rr[ridx][2] - rs[2];
      L = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      for (int it = 0; it < 8; ++it) {
        craft_pos(kind, T, sidx, t - L, rs);
        d0 = R.rr[ridx][0] - rs[0]; d1 = R.rr[ridx][1] - rs[1]; d2 = R.rr[ridx][2] - rs[2];
        L = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      }
    }
    craft_pos(kind, T, sidx, t - L, rs);
    double d[3] = {R.rr[ridx][0] - rs[0], R.rr[ridx][1] - rs[1], R.rr[ridx][2] - rs[2]};
    double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int q = 0; q < 3; ++q) {
      R.rs[j][q] = rs[q];
      R.n[j][q] = d[q] / nn;
    }
    R.L[j] = L;
  }
  o64[i] = R;
  // FP32 copy relative to the guiding centre g(t) = AU (cos(Omega t + phase),
  // sin(Omega t + phase), 0)
  double a = kOmegaOrb * t + phase;
  double g[3] = {kAUSec * cos(a), kAUSec * sin(a), 0.0};
  OrbitRec32 F;
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 3; ++q) F.rr[k][q] = (float)(R.rr[k][q] - g[q]);
  for (int j = 0; j < kNLink; ++j) {
    for (int q = 0; q < 3; ++q) {
      F.rs[j][q] = (float)(R.rs[j][q] - g[q]);
      F.n[j][q] = (float)R.n[j][q];
    }
    F.L[j] = (float)(R.L[j] - kArmSec);       // offset from the nominal light time
  }
  o32[i] = F;
}

// dt^2 * 4 df / S_c(f_k) for bins in [f_lo, f_hi], else 0 (Sangria PSD,
// x = 2 pi f L / c, A_acc = 2.4e-15; TDI 2: times 4 sin^2 2x).
__global__ void psd_kernel(int64_t nb, int64_t n, double dt, double flo, double fhi, int gen,
                           double* w) {
  float* w32 = reinterpret_cast<float*>(w + 2 * nb);      // x 2^-160, see psd_bytes
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  double f = (double)k / ((double)n * dt);
  double wae = 0.0, wt = 0.0;
  if (f >= flo && f <= fhi && f > 0.0) {
    double om = 2.0 * kPi * f;
    double oc = om / kC;
    double sacc = 2.4e-15 * 2.4e-15 * (1.0 + (4e-4 / f) * (4e-4 / f)) *
                  (1.0 + pow(f / 8e-3, 4.0)) / (om * om * om * om) * oc * oc;
    double sop = 7.9e-12 * 7.9e-12 * (1.0 + pow(2e-3 / f, 4.0)) * oc * oc;
    double x = om * kArmSec;
    double sx = sin(x), cx = cos(x);
    double sae = 8.0 * sx * sx * (2.0 * sacc * (3.0 + 2.0 * cx + cos(2.0 * x)) + sop * (2.0 + cx));
    double sh = sin(0.5 * x);
    double st = 16.0 * sop * (1.0 - cx) * sx * sx + 128.0 * sacc * sx * sx * sh * sh * sh * sh;
    if (gen == 20) {
      double s2 = sin(2.0 * x);
      sae *= 4.0 * s2 * s2;
      st *= 4.0 * s2 * s2;
    }
    double df = 1.0 / ((double)n * dt);
    wae = dt * dt * 4.0 * df / sae;
    wt = dt * dt * 4.0 * df / st;
  }
  w[k] = wae;
  w[nb + k] = wt;
  w32[k] = (float)(wae * 0x1p-160);
  w32[nb + k] = (float)(wt * 0x1p-160);
}

template <typename C>
__global__ void twiddle_kernel(int64_t n, C* tw) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  // exp(-2 pi i j / n), argument reduced exactly in integers
  double s, c;
  sincospi(-2.0 * (double)j / (double)n, &s, &c);
  tw[j].x = c;
  tw[j].y = s;
}

__global__ void data_copy_kernel(int64_t m, const double* __restrict__ src, double* d64,
                                 float* d32) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double v = src[i];
  d64[i] = v;
  d32[i] = (float)v;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_orbit_tables(const lisa_td_ctx* c, cudaStream_t s) {
  OrbitTableView T{c->orb_table, c->orb_rows, c->orb_t0, c->orb_dt};
  orbit_kernel<<<nblk(c->n, 128), 128, 0, s>>>(c->n, c->cfg.t0, c->cfg.dt, c->cfg.orbit_kind, T,
                                                c->orb_phase, c->orb64, c->orb32);
  return cudaGetLastError();
}

cudaError_t launch_psd_weights(const lisa_td_ctx* c, cudaStream_t s) {
  int64_t nb = c->n / 2 + 1;
  psd_kernel<<<nblk(nb, 256), 256, 0, s>>>(nb, c->n, c->cfg.dt, c->cfg.f_lo, c->cfg.f_hi,
                                            c->cfg.tdi_gen, c->psdw);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(const lisa_td_ctx* c, cudaStream_t s) {
  const FftPlan& p = c->plan;
  if (c->cfg.precision == 0) {
    twiddle_kernel<double2><<<nblk(c->n, 256), 256, 0, s>>>(c->n, (double2*)p.tw_n);
    twiddle_kernel<double2><<<nblk(p.n1, 256), 256, 0, s>>>(p.n1, (double2*)p.tw1);
    twiddle_kernel<double2><<<nblk(p.n2, 256), 256, 0, s>>>(p.n2, (double2*)p.tw2);
  } else {
    twiddle_kernel<float2><<<nblk(c->n, 256), 256, 0, s>>>(c->n, (float2*)p.tw_n);
    twiddle_kernel<float2><<<nblk(p.n1, 256), 256, 0, s>>>(p.n1, (float2*)p.tw1);
    twiddle_kernel<float2><<<nblk(p.n2, 256), 256, 0, s>>>(p.n2, (float2*)p.tw2);
  }
  return cudaGetLastError();
}

cudaError_t launch_data_copy(const lisa_td_ctx* c, const double* aet, cudaStream_t s) {
  int64_t m = 3 * c->n;
  data_copy_kernel<<<nblk(m, 256), 256, 0, s>>>(m, aet, c->data64, c->data32);
  return cudaGetLastError();
}

}  // namespace lisa
