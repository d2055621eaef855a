// lisa_td_fp32_fma_rate: the FP32 FMA rate this GPU sustains, measured in the
// caller's process and on its clocks, as the denominator of the mixed path's
// roofline (measurement support; the paper has no counterpart).
//
// Every thread of a grid that fills each SM (4 CTAs of 512 threads) runs 16
// independent FMA chains; each chain's recurrence a = a * b + c converges to
// c / (1 - b) and never overflows.  One result per thread is stored only if it
// is not finite (never), so the compiler cannot drop the chains.
#include <math.h>

#include "internal.h"

namespace lisa {
namespace {

constexpr int kChains = 16;
constexpr int kIters = 16384;
constexpr int kThreads = 512;
constexpr int kCtasPerSm = 4;

__global__ void __launch_bounds__(kThreads) fma_rate_kernel(float b, float c, float* sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (!isfinite(s)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace lisa

extern "C" int lisa_td_fp32_fma_rate(double* tflops_host, void* stream) {
  using namespace lisa;
  if (!tflops_host) return report_error(LISA_TD_EINVAL, "fp32_fma_rate: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "fp32_fma_rate: %s", cudaGetErrorString(e));
  const int blocks = sms * kCtasPerSm;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  float best = 0.0f;
  // the sink is never written (every chain stays finite): a null pointer
  // would do, but a valid one keeps the store well-defined if it ever ran
  float* sink = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&sink, sizeof(float) * blocks * kThreads, s);
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) {
      fma_rate_kernel<<<blocks, kThreads, 0, s>>>(0.999f, 1e-3f, sink);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;   // rep 0 warms up
  }
  if (sink) cudaFreeAsync(sink, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "fp32_fma_rate: %s", cudaGetErrorString(e));
  const double flops = 2.0 * kChains * (double)kIters * kThreads * (double)blocks;
  *tflops_host = flops / (best * 1e-3) / 1e12;
  return LISA_TD_OK;
}
