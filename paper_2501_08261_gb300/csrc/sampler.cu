// Fisher-Gaussian proposal and Metropolis-Hastings accept (include/lisa_sampler.h;
// Sec. II.C Fisher initialization, exact-likelihood acceptance).  All FP64:
// these kernels touch W x 15 numbers per step, negligible next to one
// likelihood, so they favour exactness over speed.
#include <math.h>
#include <string.h>

#include "../../include/lisa_sampler.h"
#include "internal.h"

namespace lisa {
namespace {

constexpr int kP = LISA_NPARAM;

struct SampleSpec {                 // sampled parameters, passed by value
  int32_t idx[kP];
  double eps[kP];
  double lo[kP], hi[kP];
  int32_t D;
};

__global__ void fisher_points_kernel(const double* __restrict__ theta0, SampleSpec sp, int P,
                                     double* __restrict__ pts) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double th[kP];
  for (int k = 0; k < kP; ++k) th[k] = theta0[k];
  const int D = sp.D;
  if (p >= 1 && p <= 2 * D) {
    const int a = (p - 1) / 2;
    const double s = ((p - 1) % 2 == 0) ? 1.0 : -1.0;
    th[sp.idx[a]] += s * sp.eps[a];
  } else if (p > 2 * D) {
    const int q = p - 1 - 2 * D;
    int rem = q / 4, a = 0;
    while (rem >= D - 1 - a) {
      rem -= D - 1 - a;
      ++a;
    }
    const int b = a + 1 + rem;
    const int sg = q % 4;
    const double sa = sg < 2 ? 1.0 : -1.0, sb = (sg % 2 == 0) ? 1.0 : -1.0;
    th[sp.idx[a]] += sa * sp.eps[a];
    th[sp.idx[b]] += sb * sp.eps[b];
  }
  for (int k = 0; k < kP; ++k) pts[(int64_t)p * kP + k] = th[k];
}

__global__ void fisher_assemble_kernel(const double* __restrict__ logl, SampleSpec sp,
                                       double* __restrict__ F) {
  const int D = sp.D;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= D * D) return;
  const int a = id / D, b = id % D;
  if (b < a) return;
  const double L0 = logl[0];
  if (a == b) {
    const double ea = sp.eps[a];
    F[a * D + a] = -((logl[1 + 2 * a] - 2.0 * L0) + logl[2 + 2 * a]) / (ea * ea);
    return;
  }
  const int pair = a * D - a * (a + 1) / 2 + (b - a - 1);
  const double* v = logl + 1 + 2 * D + 4 * pair;
  const double f = -(((v[0] - v[1]) - v[2]) + v[3]) / ((4.0 * sp.eps[a]) * sp.eps[b]);
  F[a * D + b] = f;
  F[b * D + a] = f;
}

__global__ void cholesky_kernel(const double* __restrict__ A, SampleSpec dg, int D,
                                double* __restrict__ L, int32_t* info) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int q = 0; q < D * D; ++q) L[q] = 0.0;
  int bad = 0;
  for (int j = 0; j < D && !bad; ++j) {
    double s = A[j * D + j] + dg.eps[j];
    for (int k = 0; k < j; ++k) s -= L[j * D + k] * L[j * D + k];
    if (!(s > 0.0)) {
      bad = j + 1;
      break;
    }
    const double ljj = sqrt(s);
    L[j * D + j] = ljj;
    for (int i = j + 1; i < D; ++i) {
      double t = A[i * D + j];
      for (int k = 0; k < j; ++k) t -= L[i * D + k] * L[j * D + k];
      L[i * D + j] = t / ljj;
    }
  }
  *info = bad;
}

__device__ double log_norm_const(const double* __restrict__ L, int D) {
  double s = 0.0;
  for (int i = 0; i < D; ++i) s += log(L[i * D + i]);
  return s - 0.5 * D * log(2.0 * 3.14159265358979323846);
}

__global__ void gauss_draw_kernel(const double* __restrict__ mu, const double* __restrict__ L,
                                  SampleSpec sp, const double* __restrict__ z, int W,
                                  double* __restrict__ x, double* __restrict__ logq) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int D = sp.D;
  double zz[kP], y[kP];
  double q2 = 0.0;
  for (int i = 0; i < D; ++i) {
    zz[i] = z[(int64_t)w * D + i];
    q2 += zz[i] * zz[i];
  }
  for (int i = D - 1; i >= 0; --i) {            // L^T y = z (back substitution)
    double t = zz[i];
    for (int k = i + 1; k < D; ++k) t -= L[k * D + i] * y[k];
    y[i] = t / L[i * D + i];
  }
  for (int k = 0; k < kP; ++k) x[(int64_t)w * kP + k] = mu[k];
  for (int i = 0; i < D; ++i) x[(int64_t)w * kP + sp.idx[i]] = mu[sp.idx[i]] + y[i];
  logq[w] = -0.5 * q2 + log_norm_const(L, D);
}

__global__ void gauss_walk_kernel(const double* __restrict__ x, const double* __restrict__ L,
                                  SampleSpec sp, const double* __restrict__ z, int W, double step,
                                  double* __restrict__ xp) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int D = sp.D;
  double y[kP];
  for (int i = D - 1; i >= 0; --i) {            // L^T y = z
    double t = z[(int64_t)w * D + i];
    for (int k = i + 1; k < D; ++k) t -= L[k * D + i] * y[k];
    y[i] = t / L[i * D + i];
  }
  for (int k = 0; k < kP; ++k) xp[(int64_t)w * kP + k] = x[(int64_t)w * kP + k];
  for (int i = 0; i < D; ++i) xp[(int64_t)w * kP + sp.idx[i]] += step * y[i];
}

__global__ void gauss_logq_kernel(const double* __restrict__ mu, const double* __restrict__ L,
                                  SampleSpec sp, const double* __restrict__ x, int W,
                                  double* __restrict__ logq) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int D = sp.D;
  double dx[kP];
  for (int i = 0; i < D; ++i) dx[i] = x[(int64_t)w * kP + sp.idx[i]] - mu[sp.idx[i]];
  double q2 = 0.0;
  for (int i = 0; i < D; ++i) {                 // z = L^T dx
    double t = 0.0;
    for (int k = i; k < D; ++k) t += L[k * D + i] * dx[k];
    q2 += t * t;
  }
  logq[w] = -0.5 * q2 + log_norm_const(L, D);
}

__global__ void mh_accept_kernel(int W, const double* __restrict__ xp,
                                 const double* __restrict__ loglp, const double* __restrict__ logqp,
                                 const double* __restrict__ u, const double* __restrict__ beta,
                                 SampleSpec sp, double* __restrict__ x,
                                 double* __restrict__ logl, double* __restrict__ logq,
                                 int32_t* __restrict__ accepted) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  bool ok = loglp[w] > -INFINITY;
  for (int k = 0; k < kP && ok; ++k) {
    const double v = xp[(int64_t)w * kP + k];
    ok = (v >= sp.lo[k]) && (v <= sp.hi[k]);
  }
  const double b = beta ? beta[w] : 1.0;            // target pi^b (tempered chains)
  if (ok) ok = log(u[w]) < (b * loglp[w] - logqp[w]) - (b * logl[w] - logq[w]);
  if (ok) {
    for (int k = 0; k < kP; ++k) x[(int64_t)w * kP + k] = xp[(int64_t)w * kP + k];
    logl[w] = loglp[w];
    logq[w] = logqp[w];
  }
  if (accepted) accepted[w] = ok ? 1 : 0;
}

// replica exchange: thread per walker column w, pairs (k, k+1) from the
// hottest down; states [T][W] temperature-major
__global__ void pt_swap_kernel(int T, int W, SampleSpec bt, const double* __restrict__ u,
                               double* __restrict__ x, double* __restrict__ logl,
                               double* __restrict__ logq, int32_t* __restrict__ swapped) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  for (int k = T - 2; k >= 0; --k) {
    const int64_t a = (int64_t)k * W + w, b = (int64_t)(k + 1) * W + w;
    const double acc = (bt.eps[k] - bt.eps[k + 1]) * (logl[b] - logl[a]);
    const bool s = log(u[(int64_t)k * W + w]) < acc;
    if (s) {
      for (int q = 0; q < kP; ++q) {
        const double t = x[a * kP + q];
        x[a * kP + q] = x[b * kP + q];
        x[b * kP + q] = t;
      }
      double t = logl[a];
      logl[a] = logl[b];
      logl[b] = t;
      t = logq[a];
      logq[a] = logq[b];
      logq[b] = t;
    }
    if (swapped) swapped[(int64_t)k * W + w] = s ? 1 : 0;
  }
}

int spec_from(const int32_t* idx, const double* eps, int D, SampleSpec* sp) {
  if (D < 1 || D > kP) return report_error(LISA_TD_EINVAL, "D=%d must be in 1..15", D);
  memset(sp, 0, sizeof(*sp));
  sp->D = D;
  if (idx) {
    for (int i = 0; i < D; ++i) {
      if (idx[i] < 0 || idx[i] >= kP) return report_error(LISA_TD_EINVAL, "idx[%d]=%d out of 0..14", i, idx[i]);
      for (int k = 0; k < i; ++k)
        if (idx[k] == idx[i]) return report_error(LISA_TD_EINVAL, "idx has %d twice", idx[i]);
      sp->idx[i] = idx[i];
    }
  }
  if (eps) {
    for (int i = 0; i < D; ++i) {
      if (!(eps[i] > 0.0) || !isfinite(eps[i])) return report_error(LISA_TD_EINVAL, "eps[%d] must be > 0", i);
      sp->eps[i] = eps[i];
    }
  }
  return LISA_TD_OK;
}

int launched(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return LISA_TD_OK;
}

inline unsigned nb(int64_t m, int b) { return (unsigned)((m + b - 1) / b); }

}  // namespace
}  // namespace lisa

using namespace lisa;

extern "C" {

int lisa_fisher_npoints(int32_t D) { return 1 + 2 * D + 2 * D * (D - 1); }

int lisa_fisher_points(const double* theta0_dev, const int32_t* idx_host, const double* eps_host,
                       int32_t D, double* points_dev, void* stream) {
  if (!theta0_dev || !idx_host || !eps_host || !points_dev) return report_error(LISA_TD_EINVAL, "NULL argument");
  SampleSpec sp;
  int rc = spec_from(idx_host, eps_host, D, &sp);
  if (rc) return rc;
  const int P = lisa_fisher_npoints(D);
  fisher_points_kernel<<<nb(P, 128), 128, 0, (cudaStream_t)stream>>>(theta0_dev, sp, P, points_dev);
  return launched("lisa_fisher_points");
}

int lisa_fisher_assemble(const double* logl_dev, const double* eps_host, int32_t D,
                         double* fisher_dev, void* stream) {
  if (!logl_dev || !eps_host || !fisher_dev) return report_error(LISA_TD_EINVAL, "NULL argument");
  SampleSpec sp;
  int rc = spec_from(nullptr, eps_host, D, &sp);
  if (rc) return rc;
  fisher_assemble_kernel<<<nb(D * D, 128), 128, 0, (cudaStream_t)stream>>>(logl_dev, sp, fisher_dev);
  return launched("lisa_fisher_assemble");
}

int lisa_cholesky(const double* a_dev, const double* diag_host, int32_t D, double* l_dev,
                  int32_t* info_dev, void* stream) {
  if (!a_dev || !l_dev || !info_dev) return report_error(LISA_TD_EINVAL, "NULL argument");
  if (D < 1 || D > kP) return report_error(LISA_TD_EINVAL, "D=%d must be in 1..15", D);
  SampleSpec dg;
  memset(&dg, 0, sizeof(dg));
  if (diag_host)
    for (int j = 0; j < D; ++j) {
      if (!(diag_host[j] >= 0.0) || !isfinite(diag_host[j])) return report_error(LISA_TD_EINVAL, "diag[%d] must be >= 0", j);
      dg.eps[j] = diag_host[j];
    }
  cholesky_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(a_dev, dg, D, l_dev, info_dev);
  return launched("lisa_cholesky");
}

int lisa_gauss_draw(const double* mu_dev, const double* l_dev, const int32_t* idx_host, int32_t D,
                    const double* z_dev, int32_t W, double* x_dev, double* logq_dev, void* stream) {
  if (!mu_dev || !l_dev || !idx_host || !z_dev || !x_dev || !logq_dev)
    return report_error(LISA_TD_EINVAL, "NULL argument");
  if (W < 1) return report_error(LISA_TD_EINVAL, "W must be >= 1");
  SampleSpec sp;
  int rc = spec_from(idx_host, nullptr, D, &sp);
  if (rc) return rc;
  gauss_draw_kernel<<<nb(W, 128), 128, 0, (cudaStream_t)stream>>>(mu_dev, l_dev, sp, z_dev, W,
                                                                  x_dev, logq_dev);
  return launched("lisa_gauss_draw");
}

int lisa_gauss_walk(const double* x_dev, const double* l_dev, const int32_t* idx_host, int32_t D,
                    const double* z_dev, int32_t W, double step, double* x_prop_dev, void* stream) {
  if (!x_dev || !l_dev || !idx_host || !z_dev || !x_prop_dev)
    return report_error(LISA_TD_EINVAL, "NULL argument");
  if (W < 1) return report_error(LISA_TD_EINVAL, "W must be >= 1");
  if (!(step > 0.0)) return report_error(LISA_TD_EINVAL, "step must be > 0");
  SampleSpec sp;
  int rc = spec_from(idx_host, nullptr, D, &sp);
  if (rc) return rc;
  gauss_walk_kernel<<<nb(W, 128), 128, 0, (cudaStream_t)stream>>>(x_dev, l_dev, sp, z_dev, W, step,
                                                                  x_prop_dev);
  return launched("lisa_gauss_walk");
}

int lisa_gauss_logq(const double* mu_dev, const double* l_dev, const int32_t* idx_host, int32_t D,
                    const double* x_dev, int32_t W, double* logq_dev, void* stream) {
  if (!mu_dev || !l_dev || !idx_host || !x_dev || !logq_dev)
    return report_error(LISA_TD_EINVAL, "NULL argument");
  if (W < 1) return report_error(LISA_TD_EINVAL, "W must be >= 1");
  SampleSpec sp;
  int rc = spec_from(idx_host, nullptr, D, &sp);
  if (rc) return rc;
  gauss_logq_kernel<<<nb(W, 128), 128, 0, (cudaStream_t)stream>>>(mu_dev, l_dev, sp, x_dev, W,
                                                                  logq_dev);
  return launched("lisa_gauss_logq");
}

int lisa_mh_accept(int32_t W, const double* x_prop_dev, const double* logl_prop_dev,
                   const double* logq_prop_dev, const double* u_dev, const double* beta_dev,
                   const double* lo_host, const double* hi_host, double* x_dev, double* logl_dev,
                   double* logq_dev, int32_t* accepted_dev, void* stream) {
  if (!x_prop_dev || !logl_prop_dev || !logq_prop_dev || !u_dev || !lo_host || !hi_host ||
      !x_dev || !logl_dev || !logq_dev)
    return report_error(LISA_TD_EINVAL, "NULL argument");
  if (W < 1) return report_error(LISA_TD_EINVAL, "W must be >= 1");
  SampleSpec sp;
  memset(&sp, 0, sizeof(sp));
  for (int k = 0; k < kP; ++k) {
    sp.lo[k] = lo_host[k];
    sp.hi[k] = hi_host[k];
  }
  mh_accept_kernel<<<nb(W, 128), 128, 0, (cudaStream_t)stream>>>(
      W, x_prop_dev, logl_prop_dev, logq_prop_dev, u_dev, beta_dev, sp, x_dev, logl_dev, logq_dev,
      accepted_dev);
  return launched("lisa_mh_accept");
}

int lisa_pt_swap(int32_t T, int32_t W, const double* betas_host, const double* u_dev,
                 double* x_dev, double* logl_dev, double* logq_dev, int32_t* swapped_dev,
                 void* stream) {
  if (!betas_host || !u_dev || !x_dev || !logl_dev || !logq_dev)
    return report_error(LISA_TD_EINVAL, "NULL argument");
  if (T < 2 || T > kP) return report_error(LISA_TD_EINVAL, "T=%d must be in 2..15", T);
  if (W < 1) return report_error(LISA_TD_EINVAL, "W must be >= 1");
  SampleSpec bt;
  memset(&bt, 0, sizeof(bt));
  for (int k = 0; k < T; ++k) {
    if (!(betas_host[k] > 0.0) || betas_host[k] > 1.0) return report_error(LISA_TD_EINVAL, "betas must be in (0, 1]");
    bt.eps[k] = betas_host[k];
  }
  pt_swap_kernel<<<nb(W, 128), 128, 0, (cudaStream_t)stream>>>(T, W, bt, u_dev, x_dev, logl_dev,
                                                               logq_dev, swapped_dev);
  return launched("lisa_pt_swap");
}

}  // extern "C"
