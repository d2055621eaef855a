// lisa_td_residual_loglike_noalloc: the DFT + PSD-weighted norm stages of the
// likelihood run on residual series the caller supplies, with every scratch
// buffer (twiddles, PSD weights, the four-step FFT intermediate, the partial
// sums) carved from one static device array instead of cudaMalloc.
//
// It exists for callers that must not allocate device memory: code whose
// device memory is owned by a framework's caching pool (a cudaMalloc of the
// library's own can then fail although the pool holds free blocks), and
// sampler loops that cannot afford the device-wide synchronisation cudaFree
// implies.  It launches the same kernels as lisa_td_loglike_batch's FFT and
// norm stages; only where their scratch lives differs.
#include <string.h>

#include <mutex>

#include "internal.h"

namespace lisa {
namespace {

// 32 MiB, held on every GPU that loads the library, until the process exits.
constexpr size_t kNoallocBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];      // device address of the array, per device
std::mutex g_scratch_mu;

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// channel list and zeroed walker records (the norm stages read only the
// status word, which must be 0 for every walker)
__global__ void noalloc_setup_kernel(int mask, int* chans, int* walker_words, int64_t nwords) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id == 0) {
    int k = 0;
    for (int q = 0; q < 3; ++q)
      if ((mask >> q) & 1) chans[k++] = q;
    for (; k < 3; ++k) chans[k] = 0;
  }
  for (int64_t q = id; q < nwords; q += (int64_t)gridDim.x * blockDim.x) walker_words[q] = 0;
}

int check(const lisa_td_config* g, const void* r, int32_t W, const double* out) {
  if (!g || !r || !out) return report_error(LISA_TD_EINVAL, "noalloc: NULL argument");
  if (!(g->dt > 0.0) || !isfinite(g->dt))
    return report_error(LISA_TD_EINVAL, "noalloc: dt must be finite and > 0");
  if (g->n < 64 || g->n > (int64_t(1) << 24)) return report_error(LISA_TD_ERANGE, "noalloc: n out of [64, 2^24]");
  if (!(g->f_lo >= 0.0) || !(g->f_hi > g->f_lo))
    return report_error(LISA_TD_EINVAL, "noalloc: band must satisfy 0 <= f_lo < f_hi");
  if (g->tdi_gen != 15 && g->tdi_gen != 20) return report_error(LISA_TD_EINVAL, "noalloc: tdi_gen must be 15 or 20");
  if (g->channel_mask < 1 || g->channel_mask > 7)
    return report_error(LISA_TD_EINVAL, "noalloc: channel_mask must be in 1..7");
  if (g->precision != 0 && g->precision != 1) return report_error(LISA_TD_EINVAL, "noalloc: precision must be 0 or 1");
  if (W < 2 || (W & 1))
    return report_error(LISA_TD_EINVAL,
                        "noalloc: W=%d must be even and >= 2 (series are transformed in pairs; "
                        "pad with a zero series)", W);
  const size_t align = g->precision == 0 ? 16 : 8;
  if ((uintptr_t)r % align) return report_error(LISA_TD_EINVAL, "noalloc: r_dev must be %zu-byte aligned", align);
  if ((uintptr_t)out % 8) return report_error(LISA_TD_EINVAL, "noalloc: logl_dev must be 8-byte aligned");
  return LISA_TD_OK;
}

}  // namespace
}  // namespace lisa

extern "C" int lisa_td_residual_loglike_noalloc(const lisa_td_config* cfg, const void* r_dev,
                                                int32_t W, double* logl_dev, void* stream) {
  using namespace lisa;
  int rc = check(cfg, r_dev, W, logl_dev);
  if (rc) return rc;
  lisa_td_ctx c;
  memset(&c, 0, sizeof(c));
  c.cfg = *cfg;
  c.cfg.max_walkers = W;
  c.n = cfg->n;
  c.wmax_pad = W;
  c.esize = cfg->precision == 0 ? 8 : 4;
  if (plan_fft(c.n, &c.plan) != 0) return report_error(LISA_TD_EINVAL, "noalloc: n must be 2^a 3^b 5^c 7^d times at most one prime in [11, 127]");
  const int64_t n = c.n;
  const size_t cs = 2 * (size_t)c.esize;
  // scratch layout, each region 256-byte aligned
  size_t off[8], at = 0;
  const size_t bytes[8] = {cs * n, cs * c.plan.n1, cs * c.plan.n2, psd_bytes(n),
                           sizeof(int) * 4, sizeof(WalkerRec) * (size_t)W,
                           (size_t)c.esize * 3 * n * W,
                           sizeof(double) * 3 * (c.plan.n1 / 2 + 1) * (size_t)W};
  for (int q = 0; q < 8; ++q) {
    off[q] = at;
    at += up256(bytes[q]);
  }
  if (at > kNoallocBytes)
    return report_error(LISA_TD_ERANGE,
                        "noalloc: n=%lld, W=%d need %zu bytes of scratch, above the fixed %zu "
                        "(about 3 n W x %d bytes are needed)", (long long)n, W, at, kNoallocBytes,
                        c.esize);
  // per-device set-up: the host-side name of the array is not a device address
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report_error(LISA_TD_ERANGE, "noalloc: device %d above %d", dev, kMaxDevices);
  // Outside stream capture the address is looked up on every call, so a
  // device reset (after which the module and its array are loaded again) never
  // leaves a stale pointer; during capture the address of the last call made
  // outside capture is used.
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "noalloc: cudaStreamIsCapturing: %s", cudaGetErrorString(e));
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return report_error(LISA_TD_ECUDA, "noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    } else if (!g_scratch_addr[dev]) {
      return report_error(LISA_TD_EINVAL,
                          "noalloc: the first call on a device must come before stream capture");
    }
    base = (unsigned char*)g_scratch_addr[dev];
  }
  c.plan.tw_n = base + off[0];
  c.plan.tw1 = base + off[1];
  c.plan.tw2 = base + off[2];
  c.psdw = (double*)(base + off[3]);
  c.chan_list = (int*)(base + off[4]);
  c.walkers = (WalkerRec*)(base + off[5]);
  c.fy = base + off[6];
  c.partial = (double*)(base + off[7]);
  const int64_t nwords = (int64_t)(sizeof(WalkerRec) * (size_t)W / sizeof(int));
  noalloc_setup_kernel<<<(unsigned)((nwords + 255) / 256 > 0 ? (nwords + 255) / 256 : 1), 256, 0, s>>>(
      cfg->channel_mask, c.chan_list, (int*)c.walkers, nwords);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_twiddles(&c, s);
  if (e == cudaSuccess) e = launch_psd_weights(&c, s);
  if (e == cudaSuccess) e = launch_fft_pass1(&c, W, r_dev, s);
  if (e == cudaSuccess) e = launch_fft_pass2(&c, W, s);
  if (e == cudaSuccess) e = launch_reduce(&c, W, W, logl_dev, nullptr, s);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "noalloc: %s", cudaGetErrorString(e));
  return LISA_TD_OK;
}
