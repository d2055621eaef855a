// Ragged batches (lisa_td_loglike_ragged): walkers whose analysis windows have
// different lengths.  Walker w is evaluated on the last n_w samples of the
// context's grid -- its own likelihood on that window, with its own DFT
// length and frequency resolution 1 / (n_w dt).
//
// Design: walkers are grouped by window length ("length classes").  When the
// workspace has room for one extra column per class, the classes run as one
// batch on the common grid ("tiled"): walkers sorted by window length
// (longest first) form the columns, each walker carries the row where its
// window starts (woff), and the waveform, projection and TDI kernels skip
// tiles before a walker group's windows begin and read rows outside a
// walker's window as zero; only the DFT and norm run per class, on the
// class's block of rows and columns of the residual, with the class's own
// FFT plan and PSD weights (a window view).  A class with an odd number of
// walkers gets one padding column (walkers are transformed in pairs).
// Otherwise each class runs the seven stages on its own window view, one
// class after another ("per class").  Views are created on first use of a
// length and kept.  With graph capture enabled the whole launch sequence is
// captured once per (class histogram, pointers) and replayed.
#include <math.h>
#include <string.h>

#include <functional>
#include <map>
#include <vector>

#include "internal.h"
#include "trace.h"

namespace lisa {
namespace {

struct View {
  lisa_td_ctx v;              // shallow copy of the context with window fields replaced
  int64_t off;
  int data_version;
};

struct Ragged {
  std::map<int64_t, View*> views;
  int cap;                    // columns the buffers below hold
  // column maps, packed [perm int32 cap][dst int32 cap][woff int64 cap]: the
  // walker behind each column, where its result goes (-1: padding column),
  // and the row its window starts at
  unsigned char* perm_ring[2];  // pinned, two used in turn, each reused only
  cudaEvent_t perm_ev[2];       // after its previous upload completed
  int ring;
  unsigned char* perm_host;   // the ring entry of the current call
  unsigned char* maps_dev;
  int32_t* perm_dev;
  int32_t* dst_dev;
  int64_t* woff_dev;
  double* params_ws;          // [cap][15]
  double* logl_ws;            // [cap]
  int32_t* status_ws;         // [cap]
  int graph_on;
  std::vector<int64_t> key;   // class histogram + pointers of the captured graph
  cudaGraphExec_t exec;
};

__global__ void view_data_kernel(const double* __restrict__ d64, int64_t n, int64_t off,
                                 int64_t nv, double* __restrict__ o64, float* __restrict__ o32) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= 3 * nv) return;
  const int64_t c = id / nv, i = id % nv;
  const double v = d64[c * n + off + i];
  o64[id] = v;
  o32[id] = (float)v;
}

__global__ void gather_kernel(const double* __restrict__ params, const int32_t* __restrict__ perm,
                              int start, int Wc, double* __restrict__ out) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= Wc * 15) return;
  const int k = id / 15, j = id % 15;
  out[id] = params[(int64_t)perm[start + k] * 15 + j];
}

__global__ void scatter_cols_kernel(const double* __restrict__ logl_ws,
                                    const int32_t* __restrict__ st_ws,
                                    const int32_t* __restrict__ dst, int ncol,
                                    double* __restrict__ logl, int32_t* __restrict__ status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ncol) return;
  const int w = dst[k];
  if (w < 0) return;                               // padding column
  logl[w] = logl_ws[k];
  if (status) status[w] = st_ws[k];
}

__global__ void scatter_kernel(const double* __restrict__ logl_ws, const int32_t* __restrict__ st_ws,
                               const int32_t* __restrict__ perm, int start, int Wc,
                               double* __restrict__ logl, int32_t* __restrict__ status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Wc) return;
  const int w = perm[start + k];
  logl[w] = logl_ws[k];
  if (status) status[w] = st_ws[k];
}

void free_view(View* vw) {
  if (!vw) return;
  void* ptrs[] = {vw->v.plan.tw_n, vw->v.plan.tw1, vw->v.plan.tw2, vw->v.psdw, vw->v.data64,
                  vw->v.data32, vw->v.partial};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete vw;
}

Ragged* state(lisa_td_ctx* c) {
  if (!c->ragged) {
    Ragged* r = new Ragged();
    r->cap = 0;
    r->perm_ring[0] = r->perm_ring[1] = nullptr;
    r->perm_ev[0] = r->perm_ev[1] = nullptr;
    r->ring = 0;
    r->perm_host = nullptr;
    r->maps_dev = nullptr;
    r->perm_dev = nullptr;
    r->dst_dev = nullptr;
    r->woff_dev = nullptr;
    r->params_ws = nullptr;
    r->logl_ws = nullptr;
    r->status_ws = nullptr;
    r->graph_on = 0;
    r->exec = nullptr;
    c->ragged = r;
  }
  return (Ragged*)c->ragged;
}

void release_buffers(Ragged* r) {
  for (int q = 0; q < 2; ++q) {
    if (r->perm_ev[q]) {
      cudaEventSynchronize(r->perm_ev[q]);
      cudaEventDestroy(r->perm_ev[q]);
    }
    if (r->perm_ring[q]) cudaFreeHost(r->perm_ring[q]);
    r->perm_ring[q] = nullptr;
    r->perm_ev[q] = nullptr;
  }
  void* ptrs[] = {r->maps_dev, r->params_ws, r->logl_ws, r->status_ws};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  r->perm_host = nullptr;
  r->maps_dev = nullptr;
  r->perm_dev = nullptr;
  r->dst_dev = nullptr;
  r->woff_dev = nullptr;
  r->params_ws = nullptr;
  r->logl_ws = nullptr;
  r->status_ws = nullptr;
  r->cap = 0;
}

cudaError_t ensure_buffers(Ragged* r, int W) {
  if (r->cap >= W) return cudaSuccess;
  release_buffers(r);
  cudaError_t e = cudaSuccess;
  const size_t mb = (size_t)W * (4 + 4 + 8);
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
    e = cudaMallocHost((void**)&r->perm_ring[q], mb);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->perm_ev[q], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->maps_dev, mb);
  if (e == cudaSuccess) {
    r->perm_dev = (int32_t*)r->maps_dev;
    r->dst_dev = (int32_t*)(r->maps_dev + (size_t)W * 4);
    r->woff_dev = (int64_t*)(r->maps_dev + (size_t)W * 8);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->params_ws, sizeof(double) * 15 * W);
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->logl_ws, sizeof(double) * W);
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->status_ws, sizeof(int32_t) * W);
  if (e == cudaSuccess) r->cap = W;
  return e;
}

// the view of the last nv samples (created on first use)
cudaError_t get_view(lisa_td_ctx* c, Ragged* r, int64_t nv, cudaStream_t s, View** out) {
  auto it = r->views.find(nv);
  View* vw = it == r->views.end() ? nullptr : it->second;
  if (!vw) {
    vw = new View();
    vw->v = *c;
    vw->off = c->n - nv;
    vw->data_version = -1;
    lisa_td_ctx& v = vw->v;
    v.n = nv;
    v.cfg.n = nv;
    v.cfg.t0 = c->cfg.t0 + (double)vw->off * c->cfg.dt;
    v.orb64 = c->orb64 + vw->off;
    v.orb32 = c->orb32 + vw->off;
    v.tdi_tiles = c->tdi_tiles + (vw->off / kTdiTile) * c->n_dterms;
    v.tdi_pairs = c->tdi_pairs + (vw->off / kTdiTile) * kTdiPairs;
    v.prof_ev = nullptr;
    v.prof_on = 0;
    v.ragged = nullptr;
    v.plan.tw_n = v.plan.tw1 = v.plan.tw2 = nullptr;
    v.psdw = nullptr;
    v.data64 = nullptr;
    v.data32 = nullptr;
    v.partial = nullptr;
    plan_fft(nv, &v.plan);
    const size_t cs = 2 * (size_t)c->esize;
    cudaError_t e = cudaMalloc(&v.plan.tw_n, cs * nv);
    if (e == cudaSuccess) e = cudaMalloc(&v.plan.tw1, cs * v.plan.n1);
    if (e == cudaSuccess) e = cudaMalloc(&v.plan.tw2, cs * v.plan.n2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&v.psdw, psd_bytes(nv));
    if (e == cudaSuccess) e = cudaMalloc((void**)&v.data64, sizeof(double) * 3 * nv);
    if (e == cudaSuccess) e = cudaMalloc((void**)&v.data32, sizeof(float) * 3 * nv);
    if (e == cudaSuccess)
      e = cudaMalloc((void**)&v.partial, sizeof(double) * 3 * (v.plan.n1 / 2 + 1) * c->wmax_pad);
    if (e == cudaSuccess) e = launch_twiddles(&v, s);
    if (e == cudaSuccess) e = launch_psd_weights(&v, s);
    if (e != cudaSuccess) {
      free_view(vw);
      return e;
    }
    r->views[nv] = vw;
  }
  if (vw->data_version != c->data_version) {
    const int64_t m = 3 * nv;
    view_data_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(c->data64, c->n, vw->off, nv,
                                                                vw->v.data64, vw->v.data32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    vw->data_version = c->data_version;
    vw->v.has_data = 1;
  }
  *out = vw;
  return cudaSuccess;
}

}  // namespace

cudaError_t ragged_view(lisa_td_ctx* c, int64_t nv, cudaStream_t s, lisa_td_ctx** out) {
  View* vw = nullptr;
  cudaError_t e = get_view(c, state(c), nv, s, &vw);
  if (e == cudaSuccess) *out = &vw->v;
  return e;
}

void free_ragged(lisa_td_ctx* c) {
  Ragged* r = (Ragged*)c->ragged;
  if (!r) return;
  for (auto& kv : r->views) free_view(kv.second);
  if (r->exec) cudaGraphExecDestroy(r->exec);
  release_buffers(r);
  delete r;
  c->ragged = nullptr;
}

}  // namespace lisa

using namespace lisa;

extern "C" {

int lisa_td_ragged_graph(lisa_td_ctx* c, int32_t enable) {
  if (!c) return report_error(LISA_TD_EINVAL, "NULL context");
  Ragged* r = state(c);
  r->graph_on = enable ? 1 : 0;
  return LISA_TD_OK;
}

int lisa_td_loglike_ragged(lisa_td_ctx* c, const double* params_dev, int32_t W,
                           const int64_t* n_host, double* logl_dev, int32_t* status_dev,
                           void* stream) {
  if (!c || !params_dev || !n_host || !logl_dev) return report_error(LISA_TD_EINVAL, "NULL argument");
  if (W < 1) return report_error(LISA_TD_EINVAL, "W must be >= 1");
  if (W > c->cfg.max_walkers) return report_error(LISA_TD_ERANGE, "W=%d above max_walkers=%d", W, c->cfg.max_walkers);
  if (!c->has_data) return report_error(LISA_TD_EINVAL, "lisa_td_set_data has not been called");
  if (c->n % kTdiTile) return report_error(LISA_TD_EINVAL, "ragged batches need n to be a multiple of %d", kTdiTile);
  // classes: window length (longest first) -> walkers (in input order)
  std::map<int64_t, std::vector<int32_t>, std::greater<int64_t>> cls;
  for (int w = 0; w < W; ++w) {
    const int64_t nv = n_host[w];
    FftPlan p;
    if (nv < 2 * kTdiTile || nv > c->n || nv % kTdiTile || plan_fft(nv, &p) != 0)
      return report_error(LISA_TD_EINVAL,
                          "n[%d]=%lld: window lengths must be multiples of %d, 2^a 3^b 5^c 7^d (times at most one prime in [11, 127]), "
                          "in [%d, n]", w, (long long)nv, kTdiTile, 2 * kTdiTile);
    cls[nv].push_back(w);
  }
  cudaStream_t s = (cudaStream_t)stream;
  Ragged* r = state(c);
  cudaError_t e = ensure_buffers(r, c->wmax_pad + 64);
  if (e != cudaSuccess) return report_error(LISA_TD_ENOMEM, "ragged buffers: %s", cudaGetErrorString(e));
  // tiled when every class plus its padding column fits the workspace
  int ncol = 0;
  for (auto& kv : cls) ncol += (int)kv.second.size() + ((int)kv.second.size() & 1);
  const int Wtp = (ncol + 31) / 32 * 32;
  const bool tiled = Wtp <= c->wmax_pad;
  // the ring entry's previous upload must have completed before it is rewritten
  r->ring ^= 1;
  r->perm_host = r->perm_ring[r->ring];
  e = cudaEventSynchronize(r->perm_ev[r->ring]);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "ragged: %s", cudaGetErrorString(e));
  const int cap = r->cap;
  int32_t* perm = (int32_t*)r->perm_host;
  int32_t* dst = (int32_t*)(r->perm_host + (size_t)cap * 4);
  int64_t* wo = (int64_t*)(r->perm_host + (size_t)cap * 8);
  struct Cls { View* vw; int64_t nv; int col0, wc, wp; };
  std::vector<Cls> cl;
  std::vector<int64_t> key;
  key.push_back(tiled ? 1 : 0);
  int col = 0;
  for (auto& kv : cls) {
    View* vw = nullptr;
    e = get_view(c, r, kv.first, s, &vw);
    if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "ragged view n=%lld: %s", (long long)kv.first, cudaGetErrorString(e));
    const int wc = (int)kv.second.size();
    const int wp = tiled ? wc + (wc & 1) : wc;
    cl.push_back({vw, kv.first, col, wc, wp});
    for (int32_t w : kv.second) {
      perm[col] = w;
      dst[col] = w;
      wo[col] = c->n - kv.first;
      ++col;
    }
    if (wp > wc) {                                 // padding column: a copy of the last walker
      perm[col] = kv.second.back();
      dst[col] = -1;
      wo[col] = c->n - kv.first;
      ++col;
    }
    key.push_back(kv.first);
    key.push_back(wc);
  }
  for (int k = col; k < cap; ++k) {                // beyond the columns: inactive everywhere
    perm[k] = perm[0];
    dst[k] = -1;
    wo[k] = c->n;
  }
  key.push_back((int64_t)(uintptr_t)params_dev);
  key.push_back((int64_t)(uintptr_t)logl_dev);
  key.push_back((int64_t)(uintptr_t)status_dev);
  e = cudaMemcpyAsync(r->maps_dev, r->perm_host, (size_t)cap * 16, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(r->perm_ev[r->ring], s);
  if (e != cudaSuccess) return report_error(LISA_TD_ECUDA, "ragged: %s", cudaGetErrorString(e));

  auto enqueue_tiled = [&]() -> cudaError_t {
    gather_kernel<<<(unsigned)((Wtp * 15 + 255) / 256), 256, 0, s>>>(params_dev, r->perm_dev, 0,
                                                                    Wtp, r->params_ws);
    cudaError_t er = cudaGetLastError();
    if (er != cudaSuccess) return er;
    lisa_td_ctx g = *c;                            // the common grid, window starts per column
    g.woff = r->woff_dev;
    g.prof_ev = nullptr;
    if ((er = launch_prep(&g, r->params_ws, Wtp, Wtp, s)) != cudaSuccess) return er;
    if ((er = launch_waveform(&g, Wtp, c->h, s)) != cudaSuccess) return er;
    if ((er = launch_project(&g, Wtp, Wtp, c->h, c->y, s)) != cudaSuccess) return er;
    if ((er = launch_tdi(&g, Wtp, Wtp, c->y, c->r, 1, s)) != cudaSuccess) return er;
    for (const Cls& k : cl) {                      // DFT + norm per class, on its block
      lisa_td_ctx f = k.vw->v;
      f.fy = c->fy;
      f.walkers = c->walkers + k.col0;
      f.woff = nullptr;
      f.fft_roff = c->n - k.nv;
      f.fft_col0 = k.col0;
      f.fft_ldr = Wtp;
      f.fft_cstride = c->n * (int64_t)Wtp;
      if ((er = launch_fft_pass1(&f, k.wp, c->r, s)) != cudaSuccess) return er;
      if ((er = launch_fft_pass2(&f, k.wp, s)) != cudaSuccess) return er;
      if ((er = launch_reduce(&f, k.wp, k.wp, r->logl_ws + k.col0, r->status_ws + k.col0, s)) != cudaSuccess)
        return er;
    }
    scatter_cols_kernel<<<(unsigned)((col + 127) / 128), 128, 0, s>>>(r->logl_ws, r->status_ws,
                                                                     r->dst_dev, col, logl_dev,
                                                                     status_dev);
    return cudaGetLastError();
  };

  auto enqueue_per_class = [&]() -> cudaError_t {
    for (const Cls& k : cl) {
      gather_kernel<<<(unsigned)((k.wc * 15 + 255) / 256), 256, 0, s>>>(params_dev, r->perm_dev,
                                                                       k.col0, k.wc, r->params_ws);
      cudaError_t er = cudaGetLastError();
      if (er != cudaSuccess) return er;
      er = run_loglike_stages(&k.vw->v, r->params_ws, k.wc, r->logl_ws, r->status_ws, s, nullptr);
      if (er != cudaSuccess) return er;
      scatter_kernel<<<(unsigned)((k.wc + 127) / 128), 128, 0, s>>>(r->logl_ws, r->status_ws,
                                                                    r->perm_dev, k.col0, k.wc,
                                                                    logl_dev, status_dev);
      er = cudaGetLastError();
      if (er != cudaSuccess) return er;
    }
    return cudaSuccess;
  };
  auto enqueue = [&]() -> cudaError_t { return tiled ? enqueue_tiled() : enqueue_per_class(); };

  if (!r->graph_on || s == nullptr) {
    e = enqueue();
    return e == cudaSuccess ? LISA_TD_OK : report_error(LISA_TD_ECUDA, "ragged: %s", cudaGetErrorString(e));
  }
  if (!r->exec || key != r->key) {
    if (r->exec) {
      cudaGraphExecDestroy(r->exec);
      r->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t eq = enqueue();
      e = cudaStreamEndCapture(s, &g);
      if (eq != cudaSuccess) e = eq;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&r->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      r->exec = nullptr;
      return report_error(LISA_TD_ECUDA, "ragged graph capture: %s", cudaGetErrorString(e));
    }
    r->key = key;
  }
  lisa::TraceRange range_("lisa_td/ragged_graph");
  e = cudaGraphLaunch(r->exec, s);
  return e == cudaSuccess ? LISA_TD_OK : report_error(LISA_TD_ECUDA, "ragged graph launch: %s", cudaGetErrorString(e));
}

}  // extern "C"
