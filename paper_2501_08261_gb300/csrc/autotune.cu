// lisa_td_autotune: measured choice of the launch shapes that are free
// parameters of the path -- the projection's tile length (samples per CTA)
// and warps per CTA, and the columns and threads per block of the two FFT
// passes (for the whole grid and, for ragged batches, for each window length).  Every
// candidate computes the same result up to rounding (the projection's FP32
// tile anchors move with the tile length); the Lagrange order is not a
// candidate, since it changes the interpolation and therefore the result.
#include <float.h>

#include <map>
#include <vector>

#include "internal.h"

namespace lisa {
namespace {

constexpr int kReps = 5;

// mean milliseconds of `reps` runs of f on stream s (after one untimed run);
// FLT_MAX if a launch fails (an invalid candidate)
template <typename F>
float time_it(F f, cudaStream_t s) {
  if (f() != cudaSuccess) {
    cudaGetLastError();
    return FLT_MAX;
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, s);
  bool ok = true;
  for (int q = 0; q < kReps && ok; ++q) ok = f() == cudaSuccess;
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  float ms = FLT_MAX;
  if (ok) {
    cudaEventElapsedTime(&ms, a, b);
    ms /= kReps;
  } else {
    cudaGetLastError();
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

// pass 1 / pass 2 columns per block and threads per block for context (or
// view) v and Wp columns
void tune_fft(lisa_td_ctx* v, int Wp, const void* r, cudaStream_t s) {
  const int cand[] = {1, 2, 4, 8, 16};
  const int bsz[] = {256, 512};
  float best = FLT_MAX;
  int pick = 0, pbs = 512;
  for (int bs : bsz) {
    for (int pb : cand) {
      if (!fft_pb_valid(v, Wp, 1, pb)) continue;
      v->tune_pb1 = pb;
      v->tune_bs1 = bs;
      float ms = time_it([&] { return launch_fft_pass1(v, Wp, r, s); }, s);
      if (ms < best) { best = ms; pick = pb; pbs = bs; }
    }
  }
  v->tune_pb1 = pick;
  v->tune_bs1 = pbs;
  launch_fft_pass1(v, Wp, r, s);
  best = FLT_MAX;
  pick = 0;
  pbs = 512;
  for (int bs : bsz) {
    for (int pb : cand) {
      if (!fft_pb_valid(v, Wp, 2, pb)) continue;
      v->tune_pb2 = pb;
      v->tune_bs2 = bs;
      float ms = time_it([&] { return launch_fft_pass2(v, Wp, s); }, s);
      if (ms < best) { best = ms; pick = pb; pbs = bs; }
    }
  }
  v->tune_pb2 = pick;
  v->tune_bs2 = pbs;
}

}  // namespace
}  // namespace lisa

using namespace lisa;

extern "C" int lisa_td_autotune(lisa_td_ctx* c, const double* params_dev, int32_t W,
                                const int64_t* n_host, int32_t* choice_host, void* stream) {
  if (!c || !params_dev) return report_error(LISA_TD_EINVAL, "NULL argument");
  if (W < 1 || W > c->cfg.max_walkers) return report_error(LISA_TD_ERANGE, "W=%d out of [1, max_walkers]", W);
  cudaStream_t s = (cudaStream_t)stream;
  const int Wp = (W + 31) / 32 * 32;
  cudaError_t e = launch_prep(c, params_dev, W, Wp, s);
  if (e == cudaSuccess) e = launch_waveform(c, Wp, c->h, s);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "autotune: %s", cudaGetErrorString(e));
  // projection: tile length x warps per CTA (the FP64 kernel keeps 4 warps)
  const int tiles[] = {64, 128, 256};
  const int warps_mixed[] = {4, 8};
  float best = FLT_MAX;
  int bt = 0, bw = 0;
  for (int t : tiles) {
    for (int wq : warps_mixed) {
      if (c->cfg.precision == 0 && wq != 4) continue;
      c->tune_tile = t;
      c->tune_warps = c->cfg.precision == 0 ? 0 : wq;
      float ms = time_it([&] { return launch_project(c, Wp, Wp, c->h, c->y, s); }, s);
      if (ms < best) { best = ms; bt = t; bw = c->tune_warps; }
    }
  }
  c->tune_tile = bt;
  c->tune_warps = bw;
  e = launch_project(c, Wp, Wp, c->h, c->y, s);
  if (e == cudaSuccess) e = launch_tdi(c, Wp, Wp, c->y, c->r, 1, s);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "autotune: %s", cudaGetErrorString(e));
  tune_fft(c, Wp, c->r, s);
  if (n_host) {
    // each window length of a ragged batch: its FFT passes on its column count
    std::map<int64_t, int> counts;
    for (int w = 0; w < W; ++w) counts[n_host[w]] += 1;
    for (auto& kv : counts) {
      FftPlan p;
      if (kv.first < 128 || kv.first > c->n || kv.first % kTdiTile || plan_fft(kv.first, &p) != 0)
        return report_error(LISA_TD_EINVAL, "autotune: window length %lld not valid", (long long)kv.first);
      lisa_td_ctx* v = nullptr;
      e = ragged_view(c, kv.first, s, &v);
      if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "autotune: %s", cudaGetErrorString(e));
      lisa_td_ctx f = *v;
      f.fy = c->fy;
      tune_fft(&f, kv.second + (kv.second & 1), c->r, s);
      v->tune_pb1 = f.tune_pb1;
      v->tune_pb2 = f.tune_pb2;
      v->tune_bs1 = f.tune_bs1;
      v->tune_bs2 = f.tune_bs2;
    }
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "autotune: %s", cudaGetErrorString(e));
  if (choice_host) {
    choice_host[0] = c->tune_tile;
    choice_host[1] = c->tune_warps;
    choice_host[2] = c->tune_pb1;
    choice_host[3] = c->tune_pb2;
    choice_host[4] = c->tune_bs1;
    choice_host[5] = c->tune_bs2;
  }
  return LISA_TD_OK;
}
