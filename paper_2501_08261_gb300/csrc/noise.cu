// lisa_td_noise: coloured Gaussian noise for the A, E, T channels (data =
// signal + noise instead of a zero-noise injection).  Per band bin k the
// noise's DFT is N_k = (x_k + i y_k) / sqrt(w_k), w_k = dt^2 4 df / S_c(f_k)
// the PSD weight of the likelihood (so E|N_k|^2 = n S / (2 dt)), and the series
// is its real inverse DFT n_j = (2/n) sum_band Re(N_k e^{2 pi i j k / n}).
// A one-off set-up step: one thread per output sample sums the band in FP64
// with a rotation recurrence re-anchored exactly every 512 bins.
#include <math.h>

#include "internal.h"

namespace lisa {
namespace {

__global__ void noise_kernel(const double* __restrict__ z, const double* __restrict__ psdw,
                             int64_t n, int64_t klo, int64_t khi, double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (j >= n) return;
  const int64_t nb = n / 2 + 1;
  const double* w = psdw + (c == 2 ? nb : 0);
  const double* zx = z + ((int64_t)c * 2 + 0) * nb;
  const double* zy = z + ((int64_t)c * 2 + 1) * nb;
  double ss, cs;
  sincospi(2.0 * (double)j / (double)n, &ss, &cs);             // step e^{2 pi i j / n}
  double er = 0.0, ei = 0.0, acc = 0.0;
  for (int64_t k = klo; k <= khi; ++k) {
    if (((k - klo) & 511) == 0) {                               // exact anchor
      const int64_t m = (j * k) % n;
      sincospi(2.0 * (double)m / (double)n, &ei, &er);
    }
    const double wk = w[k];
    if (wk > 0.0) {
      const double a = 1.0 / sqrt(wk);
      acc += a * (zx[k] * er - zy[k] * ei);
    }
    const double t = er * cs - ei * ss;
    ei = er * ss + ei * cs;
    er = t;
  }
  out[(int64_t)c * n + j] = 2.0 * acc / (double)n;
}

}  // namespace
}  // namespace lisa

using namespace lisa;

extern "C" int lisa_td_noise(lisa_td_ctx* c, const double* z_dev, double* noise_dev, void* stream) {
  if (!c || !z_dev || !noise_dev) return report_error(LISA_TD_EINVAL, "NULL argument");
  const double df = 1.0 / ((double)c->n * c->cfg.dt);
  int64_t klo = (int64_t)ceil(c->cfg.f_lo / df), khi = (int64_t)floor(c->cfg.f_hi / df);
  if (klo < 1) klo = 1;
  if (khi > c->n / 2 - 1) khi = c->n / 2 - 1;
  if (khi < klo) return report_error(LISA_TD_EINVAL, "no frequency bin inside the band");
  dim3 grid((unsigned)((c->n + 127) / 128), 3);
  noise_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(z_dev, c->psdw, c->n, klo, khi, noise_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LISA_TD_OK : report_error(LISA_TD_ECUDA, "lisa_td_noise: %s", cudaGetErrorString(e));
}
