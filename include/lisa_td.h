/*
 * lisa_td.h -- C ABI of the GB300 batched time-domain LISA log-likelihood.
 *
 * The library evaluates, for a batch of W walkers (parameter vectors), the
 * full time-domain LISA likelihood of arXiv:2501.08261 (Sec. II):
 *   waveform modes (Sec. II.A) -> polarisations h+, hx -> link responses y_slr
 *   (Sec. II.B, Eq. yslr) -> TDI X, Y, Z (Sec. II.B, X_1.5 / X_2 equations and
 *   cyclic permutation) -> A, E, T -> DFT -> PSD-weighted residual norm
 *   logL = -1/2 sum_c (h_c - d_c | h_c - d_c) (Sec. II.B, inner product and
 *   footnote on the complete log-likelihood).
 *
 * Conventions shared by every entry point
 *   - All functions are extern "C", return int status: LISA_TD_OK (0) or a
 *     negative LISA_TD_E* code; lisa_td_last_error() then describes the
 *     failure (thread-local string, valid until the next call on the thread).
 *   - Pointers named *_dev are CUDA device pointers; *_host are host pointers.
 *     The caller owns every input and output buffer; the library owns only the
 *     context and the workspace it allocates in lisa_td_create().
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls only enqueue work on it and return; no host
 *     synchronisation happens except in lisa_td_create / lisa_td_set_data
 *     (which wait for their own set-up kernels).
 *   - Parameter vectors: params_dev is FP64 [W][15], row-major, in the order
 *       m1, m2 [Msun], a1 (chi1z if aligned), theta1, phi1, a2 (chi2z), theta2,
 *       phi2, D [Gpc], iota, phi_ref, beta (ecliptic latitude), lambda
 *       (ecliptic longitude), psi, t_c [s]   (angles in radians).
 *     Table I of the paper lists the first fourteen; t_c is the time
 *     parameter of the inspiral closed form.
 *   - Sample index i <-> time t_i = t0 + i*dt, 0 <= i < n.
 *   - Element type of h / y / aet buffers: double when precision == 0 (FP64
 *     path), float when precision == 1 (mixed path: FP64 only for per-block
 *     phase/time anchors, FP32 elsewhere).
 */
#ifndef LISA_TD_H
#define LISA_TD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LISA_TD_OK        0
#define LISA_TD_EINVAL   -1   /* bad argument (NULL pointer, size, option)       */
#define LISA_TD_ENOMEM   -2   /* device allocation failed                        */
#define LISA_TD_ECUDA    -3   /* a CUDA runtime call or kernel launch failed     */
#define LISA_TD_ETIMEOUT -4   /* a bounded device-side wait gave up              */
#define LISA_TD_ERANGE   -5   /* W above the context's max_walkers, n too large  */

typedef struct lisa_td_ctx lisa_td_ctx;   /* opaque */

typedef struct {
  double  dt;              /* sample spacing [s] (Sec. II.C: 5 s)                 */
  int64_t n;               /* samples per series, 64..2^24: 2^a 3^b 5^c 7^d times
                            * at most one prime in [11, 127] (61 days at 5 s:
                            * 2^7 3^3 5 61)                                      */
  double  t0;              /* time of sample 0 [s]                               */
  double  f_lo, f_hi;      /* inner-product band [Hz] (Sec. II.C)                */
  int32_t tdi_gen;         /* 15 (X_1.5) or 20 (X_2)                             */
  int32_t channel_mask;    /* bit0 A, bit1 E, bit2 T (Sec. III.D: A, AE, AET)   */
  int32_t lagrange_order;  /* odd p in {1, 3, 5, ..., 31}; 1 = linear (Sec. II.B) */
  int32_t orbit_kind;      /* 0 rigid equal-arm, 1 Keplerian unequal-arm, 2 the
                            * caller's table of spacecraft positions
                            * (lisa_td_create_orbits)                            */
  int32_t mode_mask;       /* bits (2,2),(2,1),(3,3),(3,2),(4,4) (Sec. II.A)     */
  int32_t precessing;      /* 0 aligned spins, 1 precessing twist-up             */
  int32_t precision;       /* 0 FP64, 1 mixed                                    */
  int32_t max_walkers;     /* workspace is sized for this many walkers (>= 1)    */
  int32_t tdi_nested;      /* 0: every TDI delay is the printed sum of light times
                            * at the output time (Sec. II.B); 1: each delay is the
                            * product of one-link operators D_l f(t) = f(t - L_l(t)),
                            * applied from the output time backwards (the ordering
                            * of the standard factorised X_1.5 / X_2).  Equal for
                            * rigid orbits.                                        */
} lisa_td_config;

/* Create a context: validates cfg, builds the orbit tables (one kernel, FP64),
 * the PSD weights of the band bins and the FFT plan, and allocates the
 * workspace for cfg->max_walkers walkers.  Sec. II.B: the orbit quantities
 * are computed once, not per likelihood call.  On error *out is set to NULL
 * and everything allocated so far is freed; LISA_TD_ENOMEM when a device
 * allocation fails.  With the environment variable LISA_TD_FAIL_ALLOC=k the
 * k-th workspace allocation (0-based) fails that way on purpose (host-side
 * fault injection for testing the clean-up path). */
int lisa_td_create(lisa_td_ctx** out, const lisa_td_config* cfg, void* stream);

/* Spacecraft positions supplied by the caller, e.g. a mission orbit file such
 * as the one the paper's unequal-arm runs use (Sec. II.B, orbits; Sec. III.C).
 * Row j holds the three spacecraft's positions at time t0 + j dt:
 * pos_host[(j * 3 + k) * 3 + d] = coordinate d (x, y, z) of spacecraft k + 1,
 * in metres, in the solar-system-barycentric ecliptic frame.  The table must
 * cover the grid and the light times before it: t0 <= grid t0 - 120 s and
 * t0 + (rows - 1) dt >= last grid time; rows >= 8.  The library resamples it
 * with the centred 8-point Lagrange interpolant in the row index (nodes
 * j - 3 .. j + 4 around floor((t - t0) / dt), shifted inwards at the table's
 * ends), solves each light time from |r_r(t) - r_s(t - L)| = c L by
 * fixed-point iteration, and takes emission positions at t - L, as for the
 * built-in orbit models.  The mixed path stores positions as FP32 offsets
 * from a guiding centre on the 1 AU circle turning at the sidereal rate, with
 * its phase fitted to the table; tables whose barycentre leaves that circle
 * by more than 0.1 AU are refused (LISA_TD_ERANGE) for precision 1. */
typedef struct {
  double t0;               /* time of row 0 [s]                                  */
  double dt;               /* row spacing [s], > 0                               */
  int64_t rows;            /* rows in the table                                  */
  const double* pos_host;  /* [rows][3][3] positions [m]; copied, not kept       */
} lisa_td_orbit_table;

/* lisa_td_create for cfg->orbit_kind == 2: the orbit tables are built from
 * the caller's positions (lisa_td_orbit_table).  LISA_TD_EINVAL when
 * orbit_kind is not 2, the table is NULL, too short or does not cover the
 * grid. */
int lisa_td_create_orbits(lisa_td_ctx** out, const lisa_td_config* cfg,
                          const lisa_td_orbit_table* orbits, void* stream);

/* Store the data d (A, E, T time series; FP64 device [3][n], row c = A,E,T).
 * Sec. II.C: zero-noise injections, so d is normally an injected template.
 * The library keeps its own copy; the call synchronises `stream`. */
int lisa_td_set_data(lisa_td_ctx* ctx, const double* aet_dev, void* stream);

/* Polarisations h+, hx (after the polarisation-angle rotation, Sec. III.A) on
 * the grid for W walkers.  h_dev: [W][n][2] (h+, hx interleaved), element type
 * per cfg.precision.  Sec. II.A (aligned modes; precessing: Eq. newtwistup). */
int lisa_td_waveform(lisa_td_ctx* ctx, const double* params_dev, int32_t W,
                     void* h_dev, void* stream);

/* Link responses y_slr (Eq. yslr) on the grid.  y_dev: [6][n][W] (link-major,
 * then sample, walker fastest), link order l = 1, 2, 3, -1, -2, -3 where link
 * l joins the two spacecraft other than |l| and (s, r) = (3,2), (1,3), (2,1),
 * (2,3), (3,1), (1,2). */
int lisa_td_project(lisa_td_ctx* ctx, const double* params_dev, int32_t W,
                    void* y_dev, void* stream);

/* TDI X, Y, Z of generation cfg.tdi_gen from y (layout of lisa_td_project),
 * then A, E, T (Sec. II.B).  aet_dev: [3][n][W], element type per precision. */
int lisa_td_tdi(lisa_td_ctx* ctx, const void* y_dev, int32_t W, void* aet_dev,
                void* stream);

/* The hot path: logL[w] = -1/2 sum_{c in mask} (h_c - d_c | h_c - d_c) for
 * W walkers.  logl_dev: FP64 [W].  status_dev: int32 [W] or NULL; a walker
 * with non-finite or non-physical parameters gets status 1 and logL = -inf
 * without failing the call.  Requires lisa_td_set_data first. */
int lisa_td_loglike_batch(lisa_td_ctx* ctx, const double* params_dev, int32_t W,
                          double* logl_dev, int32_t* status_dev, void* stream);

/* Coloured Gaussian noise with the likelihood's PSDs (data = signal + noise
 * instead of the zero-noise injections of Sec. II.C; the paper's stated next
 * step): per band bin k the noise's DFT is N_k = sqrt(n S_c(f_k) / (2 dt))
 * (x_k + i y_k) / sqrt(2) (S_AE for A and E, S_T for T), zero outside the
 * band, and noise_dev [3][n] (FP64) is its real inverse DFT, so that the
 * likelihood's (n|n) equals the sum of x_k^2 + y_k^2 over the band.
 * z_dev [3][2][n/2 + 1] FP64: the standard normals x, y of each channel and
 * bin (the caller's random numbers; entries outside the band are unused).
 * A set-up step (O(n x band bins) FP64 work), not part of the hot path. */
int lisa_td_noise(lisa_td_ctx* ctx, const double* z_dev, double* noise_dev, void* stream);

/* Ragged batch (walkers of uneven signal length): walker w is evaluated on
 * its own analysis window, the last n_host[w] samples of the grid (times
 * t0 + (n - n_w + j) dt, j < n_w), with the data restricted to that window
 * and its own DFT of length n_w (frequency resolution 1 / (n_w dt)); the
 * result is what lisa_td_loglike_batch gives on a context whose grid is that
 * window.  n_host [W] (host): multiples of 64, FFT lengths as for n, in [128, n];
 * cfg.n must be a multiple of 64.  Walkers are grouped by window length; the
 * first call with a new length allocates that length's FFT plan, PSD weights
 * and data window (kept until lisa_td_destroy).  Rewriting the order of
 * walkers needs the previous call's upload of it to have completed, which
 * the call waits for. */
int lisa_td_loglike_ragged(lisa_td_ctx* ctx, const double* params_dev, int32_t W,
                           const int64_t* n_host, double* logl_dev, int32_t* status_dev,
                           void* stream);

/* With enable = 1, lisa_td_loglike_ragged captures its whole launch sequence
 * (all length classes) in a CUDA graph on first use of a given class
 * histogram and pointer set, and replays it while they repeat (needs a
 * non-default stream; on the legacy stream it runs uncaptured). */
int lisa_td_ragged_graph(lisa_td_ctx* ctx, int32_t enable);

/* Autotuner (measurement support, no paper counterpart): times the launch
 * shapes that are free parameters of the path on the caller's walkers
 * params_dev [W][15] -- the projection's tile length (64, 128, 256 samples
 * per CTA) and warps per CTA (4, 8; mixed path), and the columns per block
 * (1..16) and threads per block (256, 512) of the two FFT passes -- and keeps
 * the fastest in the context; with n_host [W] (window lengths as for
 * lisa_td_loglike_ragged, may be NULL) also the FFT shapes of each window
 * length.  Results are unchanged up to rounding (the projection's FP32 tile
 * anchors move with the tile length); the Lagrange order is not tuned (it
 * changes the result).  choice_host [6] (may be NULL): tile, warps, pass-1 and
 * pass-2 columns per block, pass-1 and pass-2 threads per block.
 * Uses the context's workspace and synchronises `stream`; call it before
 * timing or capturing. */
int lisa_td_autotune(lisa_td_ctx* ctx, const double* params_dev, int32_t W,
                     const int64_t* n_host, int32_t* choice_host, void* stream);

/* Stage timing of lisa_td_loglike_batch (measurement support, no paper
 * counterpart).  lisa_td_profile(ctx, 1) makes the following loglike calls
 * record a CUDA event on their stream before each stage and after the last
 * (at most LISA_TD_PROF_CALLS calls are recorded; later calls run untimed).
 * lisa_td_profile_read waits for the recorded events, writes the summed
 * milliseconds of each stage to stage_ms[LISA_TD_NSTAGE] and the number of
 * timed calls to *calls, and clears the record.  Stages: 0 prep, 1 waveform,
 * 2 link projection, 3 TDI + A,E,T residual, 4 FFT pass 1, 5 FFT pass 2 +
 * weighted norm, 6 final reduction. */
#define LISA_TD_NSTAGE 7
#define LISA_TD_PROF_CALLS 256
int lisa_td_profile(lisa_td_ctx* ctx, int32_t enable);
int lisa_td_profile_read(lisa_td_ctx* ctx, double* stage_ms, int64_t* calls);

/* FP32 FMA rate of the current device (measurement support, no paper
 * counterpart): the denominator of the mixed path's roofline, measured in the
 * caller's process and on its clocks.  Runs a grid of 4 CTAs x 512 threads per
 * SM, each thread 16 independent FMA chains of 16384 steps, four times on
 * `stream` (the first untimed), and writes the best rate in TFLOP/s (2 flops
 * per FMA) to *tflops_host.  Synchronises `stream`; allocates (and frees) a
 * small stream-ordered buffer.  LISA_TD_EINVAL for a NULL pointer,
 * LISA_TD_ECUDA when a CUDA call fails. */
int lisa_td_fp32_fma_rate(double* tflops_host, void* stream);

/* No-allocation variant of the DFT + PSD-weighted norm stages.  The paper has
 * no counterpart: this is a service for callers that must not allocate device
 * memory -- processes whose device memory a framework's caching pool already
 * holds (a cudaMalloc of the library's own can fail although the pool has free
 * blocks), or sampler loops that cannot take the device-wide synchronisation
 * that cudaFree implies.  It needs no context and calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *   logl_dev[w] = -1/2 sum_{c in cfg->channel_mask} (r_c | r_c),   w < W,
 * for residual series r = h - d the caller supplies: r_dev is [3][n][W]
 * (channel A, E, T, then sample, walker fastest), double when
 * cfg->precision == 0 and float when 1, 16- (double) or 8-byte (float)
 * aligned.  Fields of cfg used: dt, n, f_lo, f_hi, tdi_gen (PSD), channel_mask,
 * precision; the others are ignored.  W must be even (series are transformed
 * in pairs; pad with a zero series).  With r = AET(theta) - d it returns what
 * lisa_td_loglike_batch returns for theta.
 * Limit: all scratch lives in one static 32 MiB device array, held on every
 * GPU that loads the library until the process exits; about 3 n W x 8 (FP64)
 * or x 4 (mixed) bytes are needed, and larger (n, W) fail with LISA_TD_ERANGE
 * (n = 17280 allows W <= 78 in FP64, W <= 156 mixed).  dt must be finite and
 * > 0.  Each call made outside stream capture looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it; a call on a capturing stream
 * uses the address kept by the last uncaptured call on that device, so make
 * one call before any stream capture, and one more after a cudaDeviceReset
 * before capturing again.  Every call shares the array: calls that can
 * overlap on the GPU (different streams, or several host threads) race and
 * give wrong results; order them on one stream. */
int lisa_td_residual_loglike_noalloc(const lisa_td_config* cfg, const void* r_dev, int32_t W,
                                     double* logl_dev, void* stream);

/* Heterodyned time-domain likelihood.  The paper names heterodyning and
 * relative binning as the route to cheaper likelihoods (Sec. I, Sec. IV) and
 * gives no time-domain form; this is the library's:
 *   - every mode pair j = (l, +-m) is written as an analytic signal whose real
 *     part is the pair's h+ (hx) and whose phase is the mode's own
 *     e^{-i Phi_lm}; its TDI channel c in continuous time (waveform at the
 *     exact emission and reception times of Eq. yslr, delays as in the TDI
 *     equations, link geometry at the delayed times) is X_jc(t; theta);
 *   - with a fiducial theta0, carriers C_j(t) = e^{-i Phi_lm(t; theta0)} and
 *     nodes 0 = i_0 < ... < i_{B-1} = n - 1, the node differences are
 *     dZ_jc,b = conj(C_j(t_b)) (X_jc(t_b; theta) - X_jc(t_b; theta0));
 *   - the model on the grid is X0_c(t_i) + Re sum_j C_j(t_i) P_jc(i), P_jc the
 *     cubic Lagrange polynomial through the node differences of the nodes
 *     a .. a + 3 around sample i (a = min(max(b - 1, 0), B - 4), b the node
 *     interval holding i),
 *     X0 = Re sum_j X_jc(t_i; theta0) (computed once in FP64), and logL is the
 *     full likelihood's DFT + PSD-weighted norm of model - data.
 * At theta0 the model is X0 exactly; with a node at every sample it is the
 * continuous-time response of theta.  Only the B nodes pay for the waveform and
 * response (96 waveform evaluations per node for TDI 2); the grid pays a
 * complex multiply-add per mode and channel.
 *
 * lisa_td_het_setup: fiducial theta0_host [15] (host), nodes_host [B] (host,
 * int64 sample indices rising strictly from 0 to n - 1, B >= 4).  Computes
 * the fiducial's carriers, X0 and node values; replaces an earlier set-up.
 * Allocates n (76 + 24 nmodes) + 96 x 48 x max(B, 16384) + 48 nmodes B
 * + 3 nmodes B (16 or 8) Wmax bytes, Wmax = max_walkers rounded up to a
 * multiple of 32 (48 = the TDI-2 terms of X, Y, Z,
 * 24 for TDI 1.5; the last term is the node differences, 16 B per complex
 * value in FP64 contexts, 8 in mixed ones); synchronises `stream`.  The node
 * sums are FP64 in both precisions (FP32 terms would leave rounding that the
 * TDI combinations do not cancel); a mixed context rounds each node
 * difference to FP32 and expands and transforms in FP32.  LISA_TD_EINVAL for NULL
 * pointers, bad nodes or an invalid fiducial (the prep checks of
 * lisa_td_loglike_batch), LISA_TD_ENOMEM, LISA_TD_ECUDA.  Every orbit kind,
 * TDI generation and delay form of the context is supported; ragged batches
 * are not.
 *
 * lisa_td_het_loglike: as lisa_td_loglike_batch (same arguments, data and
 * status semantics) with the heterodyned model; LISA_TD_EINVAL before
 * lisa_td_het_setup or lisa_td_set_data.  Stage profiling (lisa_td_profile)
 * records: 0 prep, 1 node differences, 2 expansion to the grid + residual,
 * 3 (empty), 4 FFT pass 1, 5 FFT pass 2 + norm, 6 reduction.
 *
 * lisa_td_het_deltas: the node differences dZ of W walkers, written to
 * dz_dev [B][nmodes][3][W] complex (double2 for precision 0, float2 for 1),
 * modes in mask order, channels A, E, T.
 * lisa_td_het_aet: the heterodyned model A, E, T of W walkers, written to
 * aet_dev [3][n][W] (double / float).
 * Both need lisa_td_het_setup; neither needs data. */
int lisa_td_het_setup(lisa_td_ctx* ctx, const double* theta0_host, const int64_t* nodes_host,
                      int64_t B, void* stream);
int lisa_td_het_loglike(lisa_td_ctx* ctx, const double* params_dev, int32_t W, double* logl_dev,
                        int32_t* status_dev, void* stream);
int lisa_td_het_deltas(lisa_td_ctx* ctx, const double* params_dev, int32_t W, void* dz_dev,
                       void* stream);
int lisa_td_het_aet(lisa_td_ctx* ctx, const double* params_dev, int32_t W, void* aet_dev,
                    void* stream);

void lisa_td_destroy(lisa_td_ctx* ctx);
const char* lisa_td_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LISA_TD_H */
