// Host-side internals: the context object and the kernel launchers that the
// C-ABI entry points in api.cu sequence.  Not part of the public header.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lisa_td.h"
#include "common.cuh"

namespace lisa {

constexpr int kMaxRadix = 16;

struct FftPlan {
  int n1, n2;                      // n = n1 * n2 (n2 contiguous in pass 1's input)
  int r1[kMaxRadix], nr1;          // radix sequence of the n1-point transforms
  int r2[kMaxRadix], nr2;          // radix sequence of the n2-point transforms
  void* tw_n;                      // W_n^j, j < n          (double2 / float2)
  void* tw1;                       // W_n1^j, j < n1
  void* tw2;                       // W_n2^j, j < n2
};

}  // namespace lisa

struct lisa_td_ctx {
  lisa_td_config cfg;
  int64_t n;
  int wmax_pad;                    // max walkers rounded up to 32
  int esize;                       // 8 (FP64) or 4 (mixed)
  lisa::OrbitRec64* orb64;
  lisa::OrbitRec32* orb32;
  // orbit_kind 2: the caller's positions [rows][3][3] in light-seconds on the
  // device, their time grid, and the phase of the guiding centre
  // g(t) = AU (cos(Omega t + orb_phase), sin(Omega t + orb_phase), 0)
  double* orb_table;
  int64_t orb_rows;
  double orb_t0, orb_dt;
  double orb_phase;                // 0 for the built-in models
  double orb_dev;                  // largest |barycentre - g(t)| of the table [light-s]
  double* psdw;                    // [2][n/2+1]: dt^2 * 4 df / S (AE, T) in band, else 0,
                                   // followed by the same as float x 2^-160 (psd_bytes)
  lisa::FftPlan plan;
  lisa::TdiTable* tdi_tab;         // device copy of the TDI term table
  int tdi_nd;                      // most light times in one delay
  int* chan_list;                  // device [3]: indices of the channels in the mask
  lisa::TdiTileTerm* tdi_tiles;    // mixed path: [n / 64 tiles][delayed terms]
  int n_dterms;                    // delayed terms (18 for TDI 1.5, 42 for TDI 2)
  lisa::TdiTilePair* tdi_pairs;    // mixed path: [n / 64 tiles][kTdiPairs] combined FIRs
  int tdi_comb;                    // 1: every pair's FIR fits kGMax taps (tdi_comb_kernel)
  int* tdi_flag;                   // device word: set when a pair is wider than kGMax
  double* data64;                  // [3][n]
  float* data32;                   // [3][n]
  int has_data;
  // workspace
  lisa::WalkerRec* walkers;        // [wmax_pad]
  void* h;                         // [wmax_pad][n][2]
  void* y;                         // [6][n][wmax_pad]
  void* r;                         // [3][n][wmax_pad]
  void* fy;                        // [3][n1][n2][wmax_pad/2] complex
  double* partial;                 // [3][n1/2+1][wmax_pad]
  int32_t* status;                 // [wmax_pad]
  // stage timing (lisa_td_profile)
  int prof_on;
  int prof_calls;
  cudaEvent_t* prof_ev;            // [LISA_TD_PROF_CALLS][LISA_TD_NSTAGE + 1]
  // ragged batches (ragged.cu): window views and their workspace; data version
  // bumped by lisa_td_set_data so that the views refresh their data windows
  void* ragged;
  int data_version;
  // ragged batches on the common grid: woff[w] = first row of walker w's
  // window (rows before it are outside the window: the waveform is not
  // evaluated there and every stage reads them as zero); nullptr = row 0
  const int64_t* woff;
  // FFT input block of one length class: row offset, column offset and row
  // stride (reals) inside the residual buffer, channel stride (reals);
  // fft_ldr == 0 selects the whole buffer [3][n][Wpad]
  int64_t fft_roff;
  int fft_col0;
  int fft_ldr;
  int64_t fft_cstride;
  // launch shapes chosen by lisa_td_autotune (0 = built-in default): tile of
  // the projection (samples per CTA) and its warps per CTA; columns per block
  // of FFT pass 1 and pass 2
  int tune_tile, tune_warps, tune_pb1, tune_pb2;
  int tune_bs1, tune_bs2;          // FFT threads per block (0: 512)
  // heterodyned likelihood (heterodyne.cu): fiducial tables and node workspace
  void* het;
};

namespace lisa {

// prep.cu
cudaError_t launch_prep(const lisa_td_ctx* c, const double* params, int W, int Wpad,
                        cudaStream_t s);
// orbit.cu (create-time tables)
cudaError_t launch_orbit_tables(const lisa_td_ctx* c, cudaStream_t s);
cudaError_t launch_psd_weights(const lisa_td_ctx* c, cudaStream_t s);
// bytes of the psdw block for n samples: FP64 weights, then their FP32 copies
// scaled by 2^-160 (the mixed pass 2 reads those, with no FP64 arithmetic)
inline size_t psd_bytes(int64_t n) { return (sizeof(double) + sizeof(float)) * 2 * (size_t)(n / 2 + 1); }
cudaError_t launch_twiddles(const lisa_td_ctx* c, cudaStream_t s);
cudaError_t launch_data_copy(const lisa_td_ctx* c, const double* aet, cudaStream_t s);
// waveform.cu: h[w][i][2] for w < W (row stride n)
cudaError_t launch_waveform(const lisa_td_ctx* c, int W, void* h, cudaStream_t s);
// project.cu: y[l][i][ldw] for w < W, from the walker-major h with Wpad rows
cudaError_t launch_project(const lisa_td_ctx* c, int W, int ldw, const void* h, void* y,
                           cudaStream_t s);
// tdi.cu: out[c][i][ldw] = AET (resid = 0) or AET - data (resid = 1)
cudaError_t launch_tdi(const lisa_td_ctx* c, int W, int ldw, const void* y, void* out,
                       int resid, cudaStream_t s);
// fft.cu: residual r[3][n][Wpad] -> (pass 1) -> (pass 2 + weighted norm) partial sums
cudaError_t launch_fft_pass1(const lisa_td_ctx* c, int Wpad, const void* r, cudaStream_t s);
cudaError_t launch_fft_pass2(const lisa_td_ctx* c, int Wpad, cudaStream_t s);
cudaError_t launch_reduce(const lisa_td_ctx* c, int W, int Wpad, double* logl,
                          int32_t* status, cudaStream_t s);
int plan_fft(int64_t n, FftPlan* p);
// api.cu: set the thread's lisa_td_last_error() text, return `code`
int report_error(int code, const char* fmt, ...);
// ragged.cu: release the window views of a context; the view of the last nv
// samples (created on first use)
void free_ragged(lisa_td_ctx* c);
cudaError_t ragged_view(lisa_td_ctx* c, int64_t nv, cudaStream_t s, lisa_td_ctx** out);
// fft.cu: whether Pb columns per block is a valid choice for pass 1 / pass 2
bool fft_pb_valid(const lisa_td_ctx* c, int Wpad, int pass, int pb);
// the seven stages of one likelihood evaluation on context (or view) c
cudaError_t run_loglike_stages(const lisa_td_ctx* c, const double* params, int W, double* logl,
                               int32_t* status, cudaStream_t s, cudaEvent_t* ev);
TdiTable build_tdi_table(int gen);
cudaError_t launch_tdi_tiles(const lisa_td_ctx* c, cudaStream_t s);
// combined per-(channel, link) FIR weights of the mixed TDI; sets *c->tdi_flag
// when a pair needs more than kGMax taps
cudaError_t launch_tdi_pairs(const lisa_td_ctx* c, cudaStream_t s);
// heterodyne.cu: release the heterodyned likelihood's tables of a context
void free_het(lisa_td_ctx* c);

}  // namespace lisa
