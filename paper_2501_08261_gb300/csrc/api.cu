// C-ABI entry points of include/lisa_td.h: argument checks, context and
// workspace ownership, and the launch sequence of each call.  No compute
// happens on the host; every step of the likelihood runs in the kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "internal.h"
#include "trace.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(LISA_TD_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
  return fail(LISA_TD_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(expr, where)                          \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

void free_ctx(lisa_td_ctx* c) {
  if (!c) return;
  lisa::free_ragged(c);
  lisa::free_het(c);
  if (c->prof_ev) {
    for (int q = 0; q < LISA_TD_PROF_CALLS * (LISA_TD_NSTAGE + 1); ++q)
      if (c->prof_ev[q]) cudaEventDestroy(c->prof_ev[q]);
    free(c->prof_ev);
  }
  void* ptrs[] = {c->orb64, c->orb32, c->psdw, c->plan.tw_n, c->plan.tw1, c->plan.tw2,
                  c->tdi_tab, c->chan_list, c->data64, c->data32, c->walkers, c->h, c->y,
                  c->r, c->fy, c->partial, c->status, c->tdi_tiles, c->tdi_pairs,
                  c->tdi_flag, c->orb_table};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free(c);
}

int check_cfg(const lisa_td_config* g) {
  if (!(g->dt > 0.0) || !isfinite(g->dt)) return fail(LISA_TD_EINVAL, "dt must be > 0");
  if (g->n < 64 || g->n > (int64_t(1) << 24)) return fail(LISA_TD_ERANGE, "n out of [64, 2^24]");
  if (!isfinite(g->t0)) return fail(LISA_TD_EINVAL, "t0 must be finite");
  if (!(g->f_lo >= 0.0) || !(g->f_hi > g->f_lo)) return fail(LISA_TD_EINVAL, "band must satisfy 0 <= f_lo < f_hi");
  if (g->tdi_gen != 15 && g->tdi_gen != 20) return fail(LISA_TD_EINVAL, "tdi_gen must be 15 or 20");
  if (g->channel_mask < 1 || g->channel_mask > 7) return fail(LISA_TD_EINVAL, "channel_mask must be in 1..7");
  int p = g->lagrange_order;
  if (!(p == 1 || p == 3 || p == 5 || p == 7 || p == 15 || p == 31))
    return fail(LISA_TD_EINVAL, "lagrange_order must be one of 1, 3, 5, 7, 15, 31");
  if (g->orbit_kind < 0 || g->orbit_kind > 2) return fail(LISA_TD_EINVAL, "orbit_kind must be 0, 1 or 2");
  if (g->mode_mask < 1 || g->mode_mask > 31) return fail(LISA_TD_EINVAL, "mode_mask must be in 1..31");
  if (g->precessing != 0 && g->precessing != 1) return fail(LISA_TD_EINVAL, "precessing must be 0 or 1");
  if (g->precision != 0 && g->precision != 1) return fail(LISA_TD_EINVAL, "precision must be 0 or 1");
  if (g->max_walkers < 1 || g->max_walkers > 65536) return fail(LISA_TD_ERANGE, "max_walkers out of [1, 65536]");
  if (g->tdi_nested != 0 && g->tdi_nested != 1) return fail(LISA_TD_EINVAL, "tdi_nested must be 0 or 1");
  return LISA_TD_OK;
}

int check_w(const lisa_td_ctx* c, int W) {
  if (W < 1) return fail(LISA_TD_EINVAL, "W must be >= 1");
  if (W > c->cfg.max_walkers) return fail(LISA_TD_ERANGE, "W=%d above max_walkers=%d", W, c->cfg.max_walkers);
  return LISA_TD_OK;
}

inline int pad32(int w) { return (w + 31) / 32 * 32; }

// The caller's orbit table (orbit_kind 2): coverage of the grid, finite
// positions, arms near the nominal 2.5e9 m (the TDI and projection halos are
// sized for them), and the guiding centre's phase and largest offset.
int check_orbit_table(const lisa_td_config* g, const lisa_td_orbit_table* T, double* phase,
                      double* dev) {
  if (!T || !T->pos_host) return fail(LISA_TD_EINVAL, "orbit table is NULL");
  if (T->rows < 8) return fail(LISA_TD_EINVAL, "orbit table needs at least 8 rows");
  if (!(T->dt > 0.0) || !isfinite(T->dt) || !isfinite(T->t0))
    return fail(LISA_TD_EINVAL, "orbit table: t0 must be finite and dt finite and > 0");
  const double last = g->t0 + (double)(g->n - 1) * g->dt;
  if (T->t0 > g->t0 - 120.0 || T->t0 + (double)(T->rows - 1) * T->dt < last)
    return fail(LISA_TD_EINVAL,
                "orbit table covers [%.6g, %.6g] s; it must start 120 s before the grid "
                "(%.6g s) and reach its last sample (%.6g s)", T->t0,
                T->t0 + (double)(T->rows - 1) * T->dt, g->t0, last);
  const double arm = 2.5e9;
  const double omega = lisa::kOmegaOrb;            // the guiding centre's rate
  const double au = lisa::kAUSec * lisa::kC;
  const int64_t mid = T->rows / 2;
  double bx = 0.0, by = 0.0;
  for (int k = 0; k < 3; ++k) {
    bx += T->pos_host[(mid * 3 + k) * 3 + 0] / 3.0;
    by += T->pos_host[(mid * 3 + k) * 3 + 1] / 3.0;
  }
  *phase = atan2(by, bx) - omega * (T->t0 + (double)mid * T->dt);
  double worst = 0.0;
  for (int64_t j = 0; j < T->rows; ++j) {
    const double* r = T->pos_host + j * 9;
    for (int q = 0; q < 9; ++q)
      if (!isfinite(r[q])) return fail(LISA_TD_EINVAL, "orbit table row %lld is not finite", (long long)j);
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3;
      const double dx = r[a * 3] - r[b * 3], dy = r[a * 3 + 1] - r[b * 3 + 1], dz = r[a * 3 + 2] - r[b * 3 + 2];
      const double len = sqrt(dx * dx + dy * dy + dz * dz);
      if (!(len >= 0.9 * arm && len <= 1.08 * arm))
        return fail(LISA_TD_EINVAL, "orbit table row %lld: arm %d-%d is %.6g m, outside [0.9, 1.08] x 2.5e9 m",
                    (long long)j, a + 1, b + 1, len);
    }
    const double a = omega * (T->t0 + (double)j * T->dt) + *phase;
    double off2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double gd = d == 0 ? au * cos(a) : (d == 1 ? au * sin(a) : 0.0);
      const double bd = (r[d] + r[3 + d] + r[6 + d]) / 3.0 - gd;
      off2 += bd * bd;
    }
    worst = fmax(worst, sqrt(off2));
  }
  *dev = worst / lisa::kC;
  if (g->precision == 1 && worst > 0.1 * au)
    return fail(LISA_TD_ERANGE,
                "orbit table: the constellation's barycentre leaves the 1 AU guiding circle by "
                "%.3g AU (the mixed path allows 0.1 AU)", worst / au);
  return LISA_TD_OK;
}

}  // namespace

namespace lisa {

const char* const kStageRange[7] = {"lisa_td/prep", "lisa_td/waveform", "lisa_td/project",
                                    "lisa_td/tdi", "lisa_td/fft_pass1", "lisa_td/fft_pass2_norm",
                                    "lisa_td/reduce"};

cudaError_t run_loglike_stages(const lisa_td_ctx* c, const double* params, int W, double* logl,
                               int32_t* status, cudaStream_t s, cudaEvent_t* ev) {
  const int Wp = pad32(W);
  cudaError_t e = cudaSuccess;
#define STAGE(k, call)                                   \
  do {                                                   \
    TraceRange range_(kStageRange[k]);                   \
    if (ev && (e = cudaEventRecord(ev[k], s)) != cudaSuccess) return e; \
    if ((e = (call)) != cudaSuccess) return e;           \
  } while (0)
  STAGE(0, launch_prep(c, params, W, Wp, s));
  STAGE(1, launch_waveform(c, Wp, c->h, s));
  STAGE(2, launch_project(c, Wp, Wp, c->h, c->y, s));
  STAGE(3, launch_tdi(c, Wp, Wp, c->y, c->r, 1, s));
  STAGE(4, launch_fft_pass1(c, Wp, c->r, s));
  STAGE(5, launch_fft_pass2(c, Wp, s));
  STAGE(6, launch_reduce(c, W, Wp, logl, status, s));
#undef STAGE
  if (ev) e = cudaEventRecord(ev[LISA_TD_NSTAGE], s);
  return e;
}

int report_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}
}  // namespace lisa

extern "C" {

const char* lisa_td_last_error(void) { return g_err; }

static int create_ctx(lisa_td_ctx** out, const lisa_td_config* cfg,
                      const lisa_td_orbit_table* orbits, void* stream) {
  g_err[0] = 0;
  if (!out) return fail(LISA_TD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(LISA_TD_EINVAL, "cfg is NULL");
  int rc = check_cfg(cfg);
  if (rc) return rc;
  if (cfg->orbit_kind == 2 && !orbits)
    return fail(LISA_TD_EINVAL, "orbit_kind 2 takes the caller's table: use lisa_td_create_orbits");
  if (cfg->orbit_kind != 2 && orbits)
    return fail(LISA_TD_EINVAL, "an orbit table needs orbit_kind 2");
  double phase = 0.0, dev = 0.0;
  if (orbits && (rc = check_orbit_table(cfg, orbits, &phase, &dev)) != 0) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  lisa_td_ctx* c = (lisa_td_ctx*)calloc(1, sizeof(lisa_td_ctx));
  if (!c) return fail(LISA_TD_ENOMEM, "host allocation failed");
  c->cfg = *cfg;
  c->orb_phase = phase;
  c->orb_dev = dev;
  if (orbits) {
    c->orb_rows = orbits->rows;
    c->orb_t0 = orbits->t0;
    c->orb_dt = orbits->dt;
    const size_t bytes = sizeof(double) * 9 * (size_t)orbits->rows;
    double* host = (double*)malloc(bytes);
    if (!host) {
      free_ctx(c);
      return fail(LISA_TD_ENOMEM, "host allocation failed");
    }
    for (size_t q = 0; q < 9 * (size_t)orbits->rows; ++q) host[q] = orbits->pos_host[q] / lisa::kC;
    cudaError_t e = cudaMalloc((void**)&c->orb_table, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(c->orb_table, host, bytes, cudaMemcpyHostToDevice);
    free(host);
    if (e != cudaSuccess) {
      if (e == cudaErrorMemoryAllocation) c->orb_table = nullptr;
      free_ctx(c);
      cudaGetLastError();
      return cuda_fail(e, "lisa_td_create_orbits: orbit table");
    }
  }
  c->n = cfg->n;
  c->wmax_pad = pad32(cfg->max_walkers);
  c->esize = cfg->precision == 0 ? 8 : 4;
  if (lisa::plan_fft(c->n, &c->plan) != 0) {
    free_ctx(c);
    return fail(LISA_TD_EINVAL, "n must be 2^a 3^b 5^c 7^d times at most one prime in [11, 127]");
  }
  const int64_t n = c->n;
  const size_t W = (size_t)c->wmax_pad;
  const size_t cs = 2 * (size_t)c->esize;          // complex element
  struct { void** p; size_t bytes; } allocs[] = {
      {(void**)&c->orb64, sizeof(lisa::OrbitRec64) * n},
      {(void**)&c->orb32, sizeof(lisa::OrbitRec32) * n},
      {(void**)&c->psdw, lisa::psd_bytes(n)},
      {(void**)&c->plan.tw_n, cs * n},
      {(void**)&c->plan.tw1, cs * c->plan.n1},
      {(void**)&c->plan.tw2, cs * c->plan.n2},
      {(void**)&c->tdi_tab, sizeof(lisa::TdiTable)},
      {(void**)&c->chan_list, sizeof(int) * 3},
      {(void**)&c->data64, sizeof(double) * 3 * n},
      {(void**)&c->data32, sizeof(float) * 3 * n},
      {(void**)&c->walkers, sizeof(lisa::WalkerRec) * W},
      {(void**)&c->h, cs * n * W},
      {(void**)&c->y, (size_t)c->esize * 6 * n * W},
      {(void**)&c->r, (size_t)c->esize * 3 * n * W},
      {(void**)&c->fy, (size_t)c->esize * 3 * n * W},
      {(void**)&c->partial, sizeof(double) * 3 * (c->plan.n1 / 2 + 1) * W},
      {(void**)&c->status, sizeof(int32_t) * W},
      {(void**)&c->tdi_tiles, sizeof(lisa::TdiTileTerm) * ((n + lisa::kTdiTile - 1) / lisa::kTdiTile) * 42},
      {(void**)&c->tdi_pairs, sizeof(lisa::TdiTilePair) * ((n + lisa::kTdiTile - 1) / lisa::kTdiTile) * lisa::kTdiPairs},
      {(void**)&c->tdi_flag, sizeof(int)},
  };
  // host-side fault injection: LISA_TD_FAIL_ALLOC=k makes the k-th workspace
  // allocation (0-based) fail as if the device were out of memory, so that the
  // clean-up path and the LISA_TD_ENOMEM report can be tested without a fault
  const char* inject = getenv("LISA_TD_FAIL_ALLOC");
  const long fail_at = inject ? strtol(inject, nullptr, 10) : -1;
  long at = 0;
  for (auto& a : allocs) {
    cudaError_t e = at++ == fail_at ? cudaErrorMemoryAllocation : cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      *a.p = nullptr;
      free_ctx(c);
      cudaGetLastError();
      return cuda_fail(e, "lisa_td_create: cudaMalloc");
    }
  }
  lisa::TdiTable tab = lisa::build_tdi_table(cfg->tdi_gen);
  c->tdi_nd = tab.max_links_in_delay;
  c->n_dterms = tab.n_dterms;
  int chans[3] = {0, 0, 0}, nch = 0;
  for (int q = 0; q < 3; ++q)
    if ((cfg->channel_mask >> q) & 1) chans[nch++] = q;
  cudaError_t e = cudaMemcpyAsync(c->tdi_tab, &tab, sizeof(tab), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->chan_list, chans, sizeof(chans), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->data64, 0, sizeof(double) * 3 * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->data32, 0, sizeof(float) * 3 * n, s);
  if (e == cudaSuccess) e = lisa::launch_orbit_tables(c, s);
  if (e == cudaSuccess) e = lisa::launch_psd_weights(c, s);
  if (e == cudaSuccess) e = lisa::launch_twiddles(c, s);
  if (e == cudaSuccess) e = lisa::launch_tdi_tiles(c, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->tdi_flag, 0, sizeof(int), s);
  if (e == cudaSuccess) e = lisa::launch_tdi_pairs(c, s);
  int wide = 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&wide, c->tdi_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(e, "lisa_td_create");
  }
  // the combined-FIR TDI kernel runs when every pair fits (grids of a few
  // seconds' spacing); finer grids keep one FIR per term
  c->tdi_comb = wide ? 0 : 1;
  if (c->orb_table) {                              // only the orbit tables read it
    cudaFree(c->orb_table);
    c->orb_table = nullptr;
  }
  *out = c;
  return LISA_TD_OK;
}

int lisa_td_create(lisa_td_ctx** out, const lisa_td_config* cfg, void* stream) {
  return create_ctx(out, cfg, nullptr, stream);
}

int lisa_td_create_orbits(lisa_td_ctx** out, const lisa_td_config* cfg,
                          const lisa_td_orbit_table* orbits, void* stream) {
  if (!orbits) {
    g_err[0] = 0;
    if (out) *out = nullptr;
    return fail(LISA_TD_EINVAL, "orbit table is NULL");
  }
  if (cfg && cfg->orbit_kind != 2) {
    g_err[0] = 0;
    if (out) *out = nullptr;
    return fail(LISA_TD_EINVAL, "lisa_td_create_orbits needs orbit_kind 2");
  }
  return create_ctx(out, cfg, orbits, stream);
}

int lisa_td_set_data(lisa_td_ctx* c, const double* aet_dev, void* stream) {
  g_err[0] = 0;
  if (!c || !aet_dev) return fail(LISA_TD_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(lisa::launch_data_copy(c, aet_dev, s), "lisa_td_set_data");
  CK(cudaStreamSynchronize(s), "lisa_td_set_data");
  c->has_data = 1;
  c->data_version += 1;
  return LISA_TD_OK;
}

int lisa_td_waveform(lisa_td_ctx* c, const double* params_dev, int32_t W, void* h_dev,
                     void* stream) {
  g_err[0] = 0;
  if (!c || !params_dev || !h_dev) return fail(LISA_TD_EINVAL, "NULL argument");
  int rc = check_w(c, W);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CK(lisa::launch_prep(c, params_dev, W, pad32(W), s), "lisa_td_waveform: prep");
  CK(lisa::launch_waveform(c, W, h_dev, s), "lisa_td_waveform");
  return LISA_TD_OK;
}

int lisa_td_project(lisa_td_ctx* c, const double* params_dev, int32_t W, void* y_dev,
                    void* stream) {
  g_err[0] = 0;
  if (!c || !params_dev || !y_dev) return fail(LISA_TD_EINVAL, "NULL argument");
  int rc = check_w(c, W);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int Wp = pad32(W);
  CK(lisa::launch_prep(c, params_dev, W, Wp, s), "lisa_td_project: prep");
  CK(lisa::launch_waveform(c, Wp, c->h, s), "lisa_td_project: waveform");
  CK(lisa::launch_project(c, W, W, c->h, y_dev, s), "lisa_td_project");
  return LISA_TD_OK;
}

int lisa_td_tdi(lisa_td_ctx* c, const void* y_dev, int32_t W, void* aet_dev, void* stream) {
  g_err[0] = 0;
  if (!c || !y_dev || !aet_dev) return fail(LISA_TD_EINVAL, "NULL argument");
  int rc = check_w(c, W);
  if (rc) return rc;
  CK(lisa::launch_tdi(c, W, W, y_dev, aet_dev, 0, (cudaStream_t)stream), "lisa_td_tdi");
  return LISA_TD_OK;
}

int lisa_td_loglike_batch(lisa_td_ctx* c, const double* params_dev, int32_t W, double* logl_dev,
                          int32_t* status_dev, void* stream) {
  g_err[0] = 0;
  if (!c || !params_dev || !logl_dev) return fail(LISA_TD_EINVAL, "NULL argument");
  int rc = check_w(c, W);
  if (rc) return rc;
  if (!c->has_data) return fail(LISA_TD_EINVAL, "lisa_td_set_data has not been called");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t* ev = nullptr;
  if (c->prof_on && c->prof_calls < LISA_TD_PROF_CALLS)
    ev = c->prof_ev + (size_t)(c->prof_calls++) * (LISA_TD_NSTAGE + 1);
  CK(lisa::run_loglike_stages(c, params_dev, W, logl_dev, status_dev, s, ev), "lisa_td_loglike_batch");
  return LISA_TD_OK;
}

int lisa_td_profile(lisa_td_ctx* c, int32_t enable) {
  g_err[0] = 0;
  if (!c) return fail(LISA_TD_EINVAL, "NULL context");
  if (enable && !c->prof_ev) {
    const int m = LISA_TD_PROF_CALLS * (LISA_TD_NSTAGE + 1);
    c->prof_ev = (cudaEvent_t*)calloc(m, sizeof(cudaEvent_t));
    if (!c->prof_ev) return fail(LISA_TD_ENOMEM, "host allocation failed");
    for (int q = 0; q < m; ++q) CK(cudaEventCreate(&c->prof_ev[q]), "lisa_td_profile");
  }
  c->prof_on = enable ? 1 : 0;
  c->prof_calls = 0;
  return LISA_TD_OK;
}

int lisa_td_profile_read(lisa_td_ctx* c, double* stage_ms, int64_t* calls) {
  g_err[0] = 0;
  if (!c || !stage_ms || !calls) return fail(LISA_TD_EINVAL, "NULL argument");
  for (int k = 0; k < LISA_TD_NSTAGE; ++k) stage_ms[k] = 0.0;
  *calls = c->prof_calls;
  for (int q = 0; q < c->prof_calls; ++q) {
    cudaEvent_t* ev = c->prof_ev + (size_t)q * (LISA_TD_NSTAGE + 1);
    CK(cudaEventSynchronize(ev[LISA_TD_NSTAGE]), "lisa_td_profile_read");
    for (int k = 0; k < LISA_TD_NSTAGE; ++k) {
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]), "lisa_td_profile_read");
      stage_ms[k] += ms;
    }
  }
  c->prof_calls = 0;
  return LISA_TD_OK;
}

void lisa_td_destroy(lisa_td_ctx* c) { free_ctx(c); }

}  // extern "C"
