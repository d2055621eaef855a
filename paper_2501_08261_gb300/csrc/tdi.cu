// TDI Michelson X (generation 1.5 or 2.0), Y and Z by cyclic permutation, and
// A, E, T (Sec. II.B).  Every delayed term y_l(t - D(t)) takes D(t) as the plain
// sum of the link light times at the output time t (the printed form) or, with
// tdi_nested, as the product of one-link delay operators applied from t
// backwards, and interpolates y with the centred Lagrange stencil; undelayed
// terms read y_l(t) directly.
//
// Layout: one CTA = 32 walkers (lanes) x a tile of output samples.  The kernel
// stages one link's y window at a time in shared memory and adds that link's
// terms (4 for TDI 1.5, 8 for TDI 2) into per-thread X, Y, Z accumulators.
#include <math.h>
#include <string.h>

#include "internal.h"
#include "delay.cuh"
#include "lagrange.cuh"

namespace lisa {

namespace {

// X as printed (Sec. II.B): (link l, sign, links of the delay), y_{1-32} = link
// -3, y_{231} = 3, y_{123} = 2, y_{3-21} = -2.  TDI 2: the third y_123 term is
// read with delay 2L-2 + L2 + 2L3 + 2L-3.  The printed sums fix only how often
// each light time enters a delay; the links are listed here in the operator
// order of the factorised combinations (D_12 = link 3, D_21 = -3, D_13 = -2,
// D_31 = 2; D_121 = D_12 D_21, ...)
//   X_1.5 = (1 - D_121)(y_{3-21} + D_13 y_123) - (1 - D_131)(y_231 + D_12 y_{1-32}),
//   X_2   = (1 - D_121 - D_12131 + D_1312121)(y_{3-21} + D_13 y_123)
//         - (1 - D_131 - D_13121 + D_1213131)(y_231 + D_12 y_{1-32}),
// of which every printed term is exactly one product; the nested form uses
// that order, the summed form only the counts.
struct HostTerm { int l, sign, nd, d[8]; };
const HostTerm kX15[8] = {
    {-3, +1, 3, {-2, 2, 3}}, {-3, -1, 1, {3}}, {3, +1, 2, {-2, 2}}, {3, -1, 0, {}},
    {2, +1, 1, {-2}}, {2, -1, 3, {3, -3, -2}}, {-2, +1, 0, {}}, {-2, -1, 2, {3, -3}}};
const HostTerm kX20[16] = {
    {-3, +1, 3, {-2, 2, 3}}, {-3, -1, 1, {3}},
    {-3, +1, 5, {-2, 2, 3, -3, 3}}, {-3, -1, 7, {3, -3, -2, 2, -2, 2, 3}},
    {3, +1, 2, {-2, 2}}, {3, -1, 0, {}},
    {3, +1, 4, {-2, 2, 3, -3}}, {3, -1, 6, {3, -3, -2, 2, -2, 2}},
    {2, +1, 1, {-2}}, {2, -1, 3, {3, -3, -2}},
    {2, +1, 7, {-2, 2, 3, -3, 3, -3, -2}}, {2, -1, 5, {3, -3, -2, 2, -2}},
    {-2, +1, 0, {}}, {-2, -1, 2, {3, -3}},
    {-2, +1, 6, {-2, 2, 3, -3, 3, -3}}, {-2, -1, 4, {3, -3, -2, 2}}};

inline int link_index(int l) { return l > 0 ? l - 1 : 2 - l; }
inline int cyc(int l, int times) {
  int a = l > 0 ? l : -l;
  for (int t = 0; t < times; ++t) a = a % 3 + 1;
  return l > 0 ? a : -a;
}

}  // namespace

TdiTable build_tdi_table(int gen) {
  TdiTable T;
  memset(&T, 0, sizeof(T));
  const HostTerm* X = gen == 15 ? kX15 : kX20;
  int nx = gen == 15 ? 8 : 16;
  T.max_links_in_delay = 0;
  for (int ch = 0; ch < 3; ++ch) {
    for (int q = 0; q < nx; ++q) {
      int j = link_index(cyc(X[q].l, ch));
      TdiTerm& t = T.term[j][T.nterm[j]++];
      t.chan = (int8_t)ch;
      t.sign = (int8_t)X[q].sign;
      t.ndelay = (int8_t)X[q].nd;
      for (int d = 0; d < X[q].nd; ++d) {
        const int li = link_index(cyc(X[q].d[d], ch));
        t.cnt[li]++;
        T.chain[j][T.nterm[j] - 1][d] = (int8_t)li;
      }
      if (X[q].nd > T.max_links_in_delay) T.max_links_in_delay = X[q].nd;
    }
  }
  T.n_dterms = 0;
  for (int j = 0; j < kNLink; ++j)
    for (int q = 0; q < 8; ++q)
      T.dterm[j][q] = (q < T.nterm[j] && T.term[j][q].ndelay > 0) ? (int8_t)T.n_dterms++ : -1;
  return T;
}

namespace {

constexpr int kPW = 33;

// every walker of a group starts its window at or after row `end`
__device__ inline bool group_inactive(const int64_t* __restrict__ wo, int cnt, int64_t end) {
  int64_t m = wo[0];
  for (int k = 1; k < cnt; ++k) m = wo[k] < m ? wo[k] : m;
  return m >= end;
}

// one delayed term of one lane with its own weights (lanes of a warp whose
// window starts differ, in ragged batches); kept out of line so that its
// weight array does not crowd the registers of the shared-weight path
template <int K>
__device__ __noinline__ double fp64_lane_term(double eps, int64_t loc, int64_t base, int64_t lo,
                                              int rows, const double* __restrict__ ywin,
                                              const double* __restrict__ cinv,
                                              const double* __restrict__ y, int64_t row0,
                                              int64_t n, int ldw_in, int w, int W, int lane) {
  double wts[K];
  lagrange_weights<double, K>(eps, cinv, wts);
  double v = 0.0;
  if (loc >= 0 && loc + K <= rows) {
#pragma unroll
    for (int m = 0; m < K; ++m) v += wts[m] * ywin[(loc + m) * kPW + lane];
  } else {
    for (int m = 0; m < K; ++m) {
      const int64_t g = base + m;
      if (g >= lo && g >= 0 && g < n && w < W) v += wts[m] * y[(row0 + g) * ldw_in + w];
    }
  }
  return v;
}

template <int K, int SPT>
__global__ void __launch_bounds__(128) tdi_fp64_kernel(
    const TdiTable* __restrict__ tab, int W, int ldw_in, int ldw_out, int64_t n, double dt,
    const OrbitRec64* __restrict__ orb,
    const double* __restrict__ y, double* __restrict__ out, const double* __restrict__ data,
    int resid, int hl, int hr, const int64_t* __restrict__ woff, int nested) {
  constexpr int NW = 4;
  constexpr int TILE = NW * SPT;
  extern __shared__ double ywin[];              // [(TILE + hl + hr)][kPW]
  __shared__ double cinv_s[K];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * TILE;
  const int w = blockIdx.y * 32 + lane;
  const int rows = TILE + hl + hr;
  if (woff && group_inactive(woff + blockIdx.y * 32, 32, i0 + TILE)) return;
  const int64_t lo = woff ? woff[w] : 0;        // rows before lo: outside the walker's window
  // the delays depend on the sample only, so with a common window start all
  // lanes of a warp need the same Lagrange weights: lane m then evaluates
  // weight m alone and the taps take it by shuffle (a third of the FP64
  // instructions of every lane evaluating all K, on GB300's 1/64-rate pipe)
  const bool shared_w = !woff || __all_sync(0xffffffffu, lo == __shfl_sync(0xffffffffu, lo, 0));
  constexpr int H = (K - 2) / 2;
  if (warp == 0 && lane < K) cinv_s[lane] = lagrange_denom_inv<double, K>(lane);
  double ax[SPT], ay[SPT], az[SPT];      // X, Y, Z accumulators
#pragma unroll
  for (int s = 0; s < SPT; ++s) ax[s] = ay[s] = az[s] = 0.0;
  __syncthreads();

  for (int j = 0; j < kNLink; ++j) {
    __syncthreads();
    for (int r = warp; r < rows; r += NW) {
      int64_t g = i0 - hl + r;
      double v = 0.0;
      if (g >= lo && g >= 0 && g < n && w < W) v = y[((int64_t)j * n + g) * ldw_in + w];
      ywin[r * kPW + lane] = v;
    }
    __syncthreads();
    const int nt = tab->nterm[j];
    for (int q = 0; q < nt; ++q) {
      const TdiTerm T = tab->term[j][q];
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        const int ls = warp + s * NW;
        const int64_t i = i0 + ls;
        if (i >= n) continue;
        double v;
        if (T.ndelay == 0) {
          v = ywin[(ls + hl) * kPW + lane];
        } else {
          const double D = term_delay_at(T, tab->chain[j][q], orb, n, i, dt, nested);
          double tau = (double)(i - lo) - D / dt;    // relative to the window start
          double fl = floor(tau);
          const double eps = tau - fl;
          int64_t base = lo + (int64_t)fl - (K - 2) / 2;
          int64_t loc = base - (i0 - hl);
          v = 0.0;
          if (shared_w) {
            double wm = 0.0;                         // this lane's weight (lanes < K)
            if (lane < K) {
              wm = cinv_s[lane];
#pragma unroll
              for (int m = 0; m < K; ++m) wm *= m == lane ? 1.0 : eps - (double)(m - H);
            }
            if (loc >= 0 && loc + K <= rows) {       // warp-uniform: loc is common
#pragma unroll
              for (int m = 0; m < K; ++m)
                v += __shfl_sync(0xffffffffu, wm, m) * ywin[(loc + m) * kPW + lane];
            } else {
              for (int m = 0; m < K; ++m) {
                const double wk = __shfl_sync(0xffffffffu, wm, m);
                int64_t g = base + m;
                if (g >= lo && g >= 0 && g < n && w < W) v += wk * y[((int64_t)j * n + g) * ldw_in + w];
              }
            }
          } else {
            v = fp64_lane_term<K>(eps, loc, base, lo, rows, ywin, cinv_s, y, (int64_t)j * n, n,
                                  ldw_in, w, W, lane);
          }
        }
        v *= (double)T.sign;
        if (T.chan == 0) ax[s] += v;
        else if (T.chan == 1) ay[s] += v;
        else az[s] += v;
      }
    }
  }
  if (w >= W) return;
  const double r2 = 0.70710678118654752440, r6 = 0.40824829046386301637,
               r3 = 0.57735026918962576451;
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    const int64_t i = i0 + warp + s * NW;
    if (i >= n || i < lo) continue;
    double X = ax[s], Y = ay[s], Z = az[s];
    double A = (Z - X) * r2, E = (X - 2.0 * Y + Z) * r6, T = (X + Y + Z) * r3;
    if (resid) {
      A -= data[i];
      E -= data[n + i];
      T -= data[2 * n + i];
    }
    out[(0 * n + i) * ldw_out + w] = A;
    out[(1 * n + i) * ldw_out + w] = E;
    out[(2 * n + i) * ldw_out + w] = T;
  }
}

// ---------------------------------------------------------------------------
// Mixed path.
//
// TDI cancels the signal by ~(2 pi f L)^2 (X, A, E) and up to ~(2 pi f L)^4
// (T of TDI 2) at low frequency, so any *systematic* per-term error -- FP32
// rounding of Lagrange weights that stay constant while the delay drifts
// slowly, or of the fractional delay itself -- leaks through where the PSD
// weights are largest.  The delays depend only on the orbit, so their weights
// are tabulated once per context in FP64 (tdi_tiles_kernel): per 64-sample
// tile and delayed term, FP32-rounded weights at the tile anchor, the exact
// DC gain of those rounded weights, the first moment of their rounding error,
// and a quadratic for the drift of the fraction inside the tile.  The kernel
// applies the constant tile weights as an FIR plus the two one-tap corrections
// (see TdiTileTerm), so its remaining errors are FP32 rounding of the samples
// themselves, which is white and harmless.
// ---------------------------------------------------------------------------

__device__ void lagrange_weights_f64(double eps, int K, double* w) {
  const int H = (K - 2) / 2;
  for (int j = 0; j < K; ++j) {
    double num = 1.0, den = 1.0;
    for (int m = 0; m < K; ++m) {
      if (m == j) continue;
      num *= eps - (double)(m - H);
      den *= (double)(j - m);
    }
    w[j] = num / den;
  }
}

// Tile record of delayed term (jl, q) for the tile starting at sample
// tile * kTdiTile; cs[0 .. K-2] receives the signed FP64 difference weights
// (the centre one without the linear part eps_a, which the kernels add
// exactly), whose FP32 roundings are R.C.
__device__ void build_tile_term(const TdiTable* __restrict__ tab,
                                const OrbitRec64* __restrict__ orb, int64_t n, double dt, int K,
                                int tile, int jl, int q, int nested, TdiTileTerm& R, double* cs) {
  const TdiTerm T = tab->term[jl][q];
  const int64_t ia = (int64_t)tile * kTdiTile;
  auto tau_rel = [&](int j) -> double {          // tau(i) - i at i = ia + j
    int64_t i = ia + j < n ? ia + j : n - 1;
    return -term_delay_at(T, tab->chain[jl][q], orb, n, i, dt, nested) / dt;
  };
  const double ta = tau_rel(0);
  const double fl = floor(ta);
  const double eps = ta - fl;
  R.bo = (int)fl;
  R.eps_a = (float)eps;
  // quadratic drift through j = 0, 32, 63
  const double d32 = tau_rel(32) - ta, d63 = tau_rel(63) - ta;
  const double a2 = (d63 / 63.0 - d32 / 32.0) / (63.0 - 32.0);
  const double a1 = d32 / 32.0 - a2 * 32.0;
  R.a1 = (float)a1;
  R.a2 = (float)a2;
  int split = 0;
  for (int j = 0; j < kTdiTile; ++j) {
    double e = eps + (tau_rel(j) - ta);
    if (e < 0.0 || e >= 1.0) split = 1;
  }
  R.split = split;
  double w[32];
  lagrange_weights_f64(eps, K, w);
  const int H = (K - 2) / 2;                       // node offsets o_k = k - H, k = 0..K-1
  const double sgd = (double)T.sign;
  double mom = 0.0;
  for (int q2 = 0; q2 < 32; ++q2) R.C[q2] = 0.0f;
  for (int mi = 0; mi < K - 1; ++mi) {             // m = mi - H, from -H to H
    const int m = mi - H;
    double c = 0.0;
    for (int k = 0; k < K; ++k) {
      const int o = k - H;
      if (m >= 0 && o > m) c += w[k];
      if (m < 0 && o <= m) c -= w[k];
    }
    if (m == 0) {
      // the linear-interpolation part eps_a dy_c goes to the compensated main
      // accumulator in the kernel; the table keeps the remainder
      const double rem = c - (double)R.eps_a;
      const float cf = (float)rem;
      R.C[mi] = cf;
      cs[mi] = sgd * rem;
      mom += ((double)R.eps_a + (double)cf) - c;
    } else {
      const float cf = (float)c;
      R.C[mi] = cf;
      cs[mi] = sgd * c;
      mom += (double)cf - c;
    }
  }
  // the term's sign, exact on every field that the kernel only adds
  const float sg = (float)T.sign;
  for (int q2 = 0; q2 < 32; ++q2) R.C[q2] *= sg;
  R.m1 = sg * (float)mom;
  R.sa1 = sg * R.a1;
  R.sa2 = sg * R.a2;
  R.se = sg * R.eps_a;
  R.pad[0] = R.pad[1] = R.pad[2] = 0;
}

__global__ void tdi_tiles_kernel(const TdiTable* __restrict__ tab,
                                 const OrbitRec64* __restrict__ orb, int64_t n, double dt, int K,
                                 int ntiles, int nested, TdiTileTerm* __restrict__ out) {
  const int nd = tab->n_dterms;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)ntiles * nd) return;
  const int tile = (int)(id / nd), d = (int)(id % nd);
  int jl = 0, q = 0;
  for (int j = 0; j < kNLink; ++j)
    for (int qq = 0; qq < tab->nterm[j]; ++qq)
      if (tab->dterm[j][qq] == d) { jl = j; q = qq; }
  TdiTileTerm R;
  double cs[32];
  build_tile_term(tab, orb, n, dt, K, tile, jl, q, nested, R, cs);
  out[id] = R;
}

// channel of pair (link j, k-th channel reading link j in term order), or -1
__host__ __device__ inline int pair_channel(const TdiTable* tab, int j, int k) {
  int seen[3] = {-1, -1, -1}, ns = 0;
  for (int q = 0; q < tab->nterm[j]; ++q) {
    const int ch = tab->term[j][q].chan;
    bool dup = false;
    for (int u = 0; u < ns; ++u) dup = dup || seen[u] == ch;
    if (!dup && ns < 3) seen[ns++] = ch;
  }
  return k < ns ? seen[k] : -1;
}

// One thread per (tile, pair): the pair's terms and their combined FIR.
__global__ void tdi_pairs_kernel(const TdiTable* __restrict__ tab,
                                 const OrbitRec64* __restrict__ orb, int64_t n, double dt, int K,
                                 int ntiles, int nested, TdiTilePair* __restrict__ out,
                                 int* __restrict__ too_wide) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)ntiles * kTdiPairs) return;
  const int tile = (int)(id / kTdiPairs), pj = (int)(id % kTdiPairs);
  const int j = pj / 2, ch = pair_channel(tab, j, pj % 2);
  const int H = (K - 2) / 2;
  TdiTilePair P;
  memset(&P, 0, sizeof(P));
  P.chan = ch < 0 ? 0 : ch;
  double g[kGMax];
  for (int k = 0; k < kGMax; ++k) g[k] = 0.0;
  double cs[4][32];
  int first = -1, bmin = 0, bmax = 0, cmin = 0, cmax = 0;
  for (int q = 0; q < tab->nterm[j] && ch >= 0; ++q) {
    const TdiTerm T = tab->term[j][q];
    if (T.chan != ch || P.nterm >= 4) continue;
    TdiTermLite& L = P.t[P.nterm];
    L.sg = (float)T.sign;
    if (T.ndelay == 0) {
      L.kind = 0;
      L.bo = 0;
    } else {
      TdiTileTerm R;
      build_tile_term(tab, orb, n, dt, K, tile, j, q, nested, R, cs[P.nterm]);
      L.bo = R.bo;
      L.kind = R.split ? 2 : 1;
      L.se = R.se;
      L.sa1 = R.sa1;
      L.sa2 = R.sa2;
      L.eps_a = R.eps_a;
      L.a1 = R.a1;
      L.a2 = R.a2;
      if (!R.split) {
        const int b = R.bo - H;
        if (first < 0) {
          first = P.nterm;
          bmin = bmax = b;
          cmin = cmax = R.bo;
        }
        bmin = b < bmin ? b : bmin;
        bmax = b > bmax ? b : bmax;
        cmin = R.bo < cmin ? R.bo : cmin;
        cmax = R.bo > cmax ? R.bo : cmax;
      }
    }
    P.nterm++;
  }
  if (first >= 0) {
    const int ntap = bmax - bmin + K - 1;
    if (ntap > kGMax) {
      atomicOr(too_wide, 1);
    } else {
      for (int u = 0; u < P.nterm; ++u) {
        if (P.t[u].kind != 1) continue;
        const int o = P.t[u].bo - H - bmin;
        for (int m = 0; m < K - 1; ++m) g[o + m] += cs[u][m];
      }
      // zeroth and first moments (rows relative to the output row) of the
      // rounding error, cancelled by taps at the outermost centre rows
      double s0 = 0.0, s1 = 0.0;
      for (int k = 0; k < kGMax; ++k) {
        P.G[k] = (float)g[k];
        const double e = (double)P.G[k] - g[k];
        s0 += e;
        s1 += e * (double)(bmin + k);
      }
      const int ka = cmin, kb = cmax > cmin ? cmax : cmin + 1;
      const double wb = (s0 * (double)ka - s1) / (double)(kb - ka);
      P.wa = (float)(-s0 - wb);
      P.wb = (float)wb;
      P.ma = ka;
      P.mb = kb;
      P.boff = bmin;
      P.ntap4 = (ntap + 3) & ~3;
    }
  }
  out[id] = P;
}

constexpr int kMixTile = kTdiTile;
constexpr int kMixSpt = 4;                  // samples per thread (16 warps x 4 = 64)
constexpr int kMixWarps = kMixTile / kMixSpt;
constexpr int kPW2 = 33;                    // padded walker pairs per row

struct f2 { float x, y; };                  // two walkers of one lane

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ f2 ld2(const float2* p) { float2 v = *p; return {v.x, v.y}; }

// compensated (Knuth two-sum) accumulation of the |y|-sized centre samples:
// hi + lo keeps their sum exact to ~2^-48, so that the TDI cancellation in X,
// Y, Z (and further in T) is not limited by FP32 rounding of these sums; the
// lo parts go to the small accumulator
__device__ __forceinline__ void acc2(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}

template <int SPT>
__device__ __forceinline__ void add_rows(f2 (&hi)[SPT], f2 (&lo)[SPT], const float2* __restrict__ yw,
                                         int row0, float sg, int lane) {
#pragma unroll
  for (int r = 0; r < SPT; ++r) {
    const f2 v = ld2(&yw[(row0 + r) * kPW2 + lane]);
    acc2(hi[r].x, lo[r].x, sg * v.x);
    acc2(hi[r].y, lo[r].y, sg * v.y);
  }
}

// small[r] += sum_{m'} c[m'] dy[b0 + r + m'] + dr_r dy[b0 + r + H], c and dr carrying the
// sign (stored signed in the tile table); the linear-interpolation part sg eps_a
// dy[b0 + r + H] is added to the main accumulator exactly (FMA two-product,
// two-sum), since its rounding in the small accumulator is noise of size
// ulp(|dy|) that TDI 2's T channel no longer suppresses
template <int K, int SPT>
__device__ __forceinline__ void apply_tile_term(f2 (&main)[SPT], f2 (&acc)[SPT],
                                                const float2* __restrict__ dyw,
                                                const TdiTileTerm& P, int s0, int b0, int lane) {
  constexpr int H = (K - 2) / 2;
  constexpr int NT = K - 1;                       // taps on the differences
  float c[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) c[k] = P.C[k];
  const float m1 = P.m1, a1 = P.sa1, a2 = P.sa2, se = P.se;
  f2 win[SPT];
#pragma unroll
  for (int r = 0; r < SPT; ++r) win[r] = ld2(&dyw[(b0 + r) * kPW2 + lane]);
#pragma unroll
  for (int m = 0; m < NT; ++m) {
#pragma unroll
    for (int r = 0; r < SPT; ++r) {
      acc[r].x = fmaf(c[m], win[r].x, acc[r].x);
      acc[r].y = fmaf(c[m], win[r].y, acc[r].y);
    }
    if (m == H) {                                 // win[r] = dy at the centre
#pragma unroll
      for (int r = 0; r < SPT; ++r) {
        const float jj = (float)(s0 + r);
        const float dr = jj * fmaf(jj, a2, a1) - m1;
        acc[r].x = fmaf(dr, win[r].x, acc[r].x);
        acc[r].y = fmaf(dr, win[r].y, acc[r].y);
        const float px = se * win[r].x, py = se * win[r].y;
        const float ex = fmaf(se, win[r].x, -px), ey = fmaf(se, win[r].y, -py);
        acc2(main[r].x, acc[r].x, px);
        acc2(main[r].y, acc[r].y, py);
        acc[r].x += ex;
        acc[r].y += ey;
      }
    }
    if (m + 1 < NT) {
#pragma unroll
      for (int r = 0; r < SPT - 1; ++r) win[r] = win[r + 1];
      win[SPT - 1] = ld2(&dyw[(b0 + SPT + m) * kPW2 + lane]);
    }
  }
}

// tiles whose fraction wraps inside the tile (rare): per-sample FP32 weights,
// still as y_c' + sum w_k (y_k - y_c') so that their DC error meets only differences
template <int K, typename Rec>
__device__ __noinline__ float4 split_one(const float2* __restrict__ yw, const Rec* P,
                                         int s, int hl, int rows, int lane) {
  const int H = (K - 2) / 2;
  const float jj = (float)s;
  float e = P->eps_a + jj * fmaf(jj, P->a2, P->a1);
  float fl = floorf(e);
  float eps = e - fl;
  const int c = s + hl + P->bo + (int)fl;
  const float2 yc = (c >= 0 && c < rows) ? yw[c * kPW2 + lane] : make_float2(0.0f, 0.0f);
  float ax = 0.0f, ay = 0.0f;
  for (int k = 0; k < K; ++k) {
    float num = 1.0f, den = 1.0f;
    for (int m = 0; m < K; ++m) {
      if (m == k) continue;
      num *= eps - (float)(m - H);
      den *= (float)(k - m);
    }
    const float wk = num / den;
    const int row = c + k - H;
    float2 v = (row >= 0 && row < rows) ? yw[row * kPW2 + lane] : make_float2(0.0f, 0.0f);
    ax = fmaf(wk, v.x - yc.x, ax);
    ay = fmaf(wk, v.y - yc.y, ay);
  }
  return make_float4(yc.x, yc.y, ax, ay);
}

// One CTA = 64 walkers (two per lane) x 64 output samples (16 warps x 4).
// Accumulators: `m*` hold the |y|-sized centre samples of every term
// (compensated), `s*` the difference FIRs, corrections and compensation terms;
// A, E, T are formed from the m parts error-free before the s parts are added.
template <int K>
__global__ void __launch_bounds__(32 * kMixWarps, 1) tdi_mixed_kernel(
    const TdiTable* __restrict__ tab, const TdiTileTerm* __restrict__ tiles, int W, int ldw,
    int64_t n, const float* __restrict__ y, float* __restrict__ out,
    const float* __restrict__ data, int resid, int hl, int hr,
    const int64_t* __restrict__ woff) {
  constexpr int SPT = kMixSpt;
  extern __shared__ float2 smem2[];
  const int rows = kMixTile + hl + hr;
  float2* ybuf0 = smem2;                           // [rows][kPW2], links 0, 2, 4
  float2* ybuf1 = smem2 + rows * kPW2;             // links 1, 3, 5
  float2* dyw = smem2 + 2 * rows * kPW2;           // dy_r = y_{r+1} - y_r of the current link
  __shared__ TdiTileTerm tts[42];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int tid = warp * 32 + lane;
  const int64_t i0 = (int64_t)blockIdx.x * kMixTile;
  const int wa = blockIdx.y * 64 + 2 * lane;       // walkers wa, wa + 1
  const int s0 = warp * SPT;
  const int nd = tab->n_dterms;
  if (woff && group_inactive(woff + blockIdx.y * 64, 64, i0 + kMixTile)) return;
  // rows before lo_a / lo_b are outside the windows of walkers wa / wa + 1
  const int64_t lo_a = woff ? woff[wa] : 0, lo_b = woff ? woff[wa + 1] : 0;
  {
    const int* src = reinterpret_cast<const int*>(tiles + (int64_t)blockIdx.x * nd);
    int* dst = reinterpret_cast<int*>(tts);
    const int words = nd * (int)(sizeof(TdiTileTerm) / sizeof(int));
    for (int q = tid; q < words; q += 32 * kMixWarps) dst[q] = src[q];
  }
  f2 mx[SPT], my[SPT], mz[SPT], sx[SPT], sy[SPT], sz[SPT];
#pragma unroll
  for (int r = 0; r < SPT; ++r)
    mx[r] = my[r] = mz[r] = sx[r] = sy[r] = sz[r] = f2{0.0f, 0.0f};

  // y rows of link j -> dst by asynchronous copies (zeros outside the grid and
  // for walkers >= W), so that the next link's loads overlap this link's FIRs
  auto stage = [&](int j, float2* dst) {
    for (int r = warp; r < rows; r += kMixWarps) {
      const int64_t g = i0 - hl + r;
      float* d = reinterpret_cast<float*>(dst + r * kPW2 + lane);
      const bool in = g >= 0 && g < n;
      const float* src = in ? y + ((int64_t)j * n + g) * ldw + wa : y;
      if (in && g >= lo_a && wa < W) cp_async4(d, src); else d[0] = 0.0f;
      if (in && g >= lo_b && wa + 1 < W) cp_async4(d + 1, src + 1); else d[1] = 0.0f;
    }
    cp_async_commit();
  };
  stage(0, ybuf0);
  for (int j = 0; j < kNLink; ++j) {
    float2* yw = (j & 1) ? ybuf1 : ybuf0;
    if (j + 1 < kNLink) {
      stage(j + 1, (j & 1) ? ybuf0 : ybuf1);      // its buffer was last read by link j - 1
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    for (int r = warp; r < rows; r += kMixWarps) {
      float2 a = yw[r * kPW2 + lane];
      float2 b = r + 1 < rows ? yw[(r + 1) * kPW2 + lane] : a;
      dyw[r * kPW2 + lane] = make_float2(b.x - a.x, b.y - a.y);
    }
    __syncthreads();
    const int nt = tab->nterm[j];
    for (int q = 0; q < nt; ++q) {
      const TdiTerm T = tab->term[j][q];
      const float sg = (float)T.sign;
      if (T.ndelay == 0) {
        if (T.chan == 0) add_rows<SPT>(mx, sx, yw, s0 + hl, sg, lane);
        else if (T.chan == 1) add_rows<SPT>(my, sy, yw, s0 + hl, sg, lane);
        else add_rows<SPT>(mz, sz, yw, s0 + hl, sg, lane);
        continue;
      }
      const TdiTileTerm& P = tts[tab->dterm[j][q]];
      if (!P.split) {
        const int c0 = s0 + hl + P.bo;             // centre row of sample s0
        const int b0 = c0 - (K - 2) / 2;
        if (T.chan == 0) {
          add_rows<SPT>(mx, sx, yw, c0, sg, lane);
          apply_tile_term<K, SPT>(mx, sx, dyw, P, s0, b0, lane);
        } else if (T.chan == 1) {
          add_rows<SPT>(my, sy, yw, c0, sg, lane);
          apply_tile_term<K, SPT>(my, sy, dyw, P, s0, b0, lane);
        } else {
          add_rows<SPT>(mz, sz, yw, c0, sg, lane);
          apply_tile_term<K, SPT>(mz, sz, dyw, P, s0, b0, lane);
        }
      } else {
#pragma unroll
        for (int r = 0; r < SPT; ++r) {
          const float4 v = split_one<K>(yw, &P, s0 + r, hl, rows, lane);
          if (T.chan == 0) {
            acc2(mx[r].x, sx[r].x, sg * v.x); acc2(mx[r].y, sx[r].y, sg * v.y);
            sx[r].x = fmaf(sg, v.z, sx[r].x); sx[r].y = fmaf(sg, v.w, sx[r].y);
          } else if (T.chan == 1) {
            acc2(my[r].x, sy[r].x, sg * v.x); acc2(my[r].y, sy[r].y, sg * v.y);
            sy[r].x = fmaf(sg, v.z, sy[r].x); sy[r].y = fmaf(sg, v.w, sy[r].y);
          } else {
            acc2(mz[r].x, sz[r].x, sg * v.x); acc2(mz[r].y, sz[r].y, sg * v.y);
            sz[r].x = fmaf(sg, v.z, sz[r].x); sz[r].y = fmaf(sg, v.w, sz[r].y);
          }
        }
      }
    }
    __syncthreads();                               // link j's buffers are free again
  }
  const float r2 = 0.70710678118654752f, r6 = 0.40824829046386302f, r3 = 0.57735026918962576f;
#pragma unroll
  for (int r = 0; r < SPT; ++r) {
    const int64_t i = i0 + s0 + r;
    if (i >= n) continue;
    float dA = 0.0f, dE = 0.0f, dT = 0.0f;
    if (resid) {
      dA = data[i];
      dE = data[n + i];
      dT = data[2 * n + i];
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int w = wa + e;
      if (w >= W || i < (e ? lo_b : lo_a)) continue;
      const float Mx = e ? mx[r].y : mx[r].x, My = e ? my[r].y : my[r].x, Mz = e ? mz[r].y : mz[r].x;
      const float Sx = e ? sx[r].y : sx[r].x, Sy = e ? sy[r].y : sy[r].x, Sz = e ? sz[r].y : sz[r].x;
      // A, E, T from the main parts combined error-free first, the small parts after
      df32 zx = two_sum(Mz, -Mx);
      df32 xy = two_sum(Mx, -2.0f * My);
      df32 xyz = two_sum(xy.hi, Mz);
      df32 xy3 = two_sum(Mx, My);
      df32 t3 = two_sum(xy3.hi, Mz);
      const float A = zx.hi + (zx.lo + (Sz - Sx));
      const float E = xyz.hi + ((xy.lo + xyz.lo) + (Sx - 2.0f * Sy + Sz));
      const float Tt = t3.hi + ((xy3.lo + t3.lo) + (Sx + Sy + Sz));
      out[(0 * n + i) * ldw + w] = A * r2 - dA;
      out[(1 * n + i) * ldw + w] = E * r6 - dE;
      out[(2 * n + i) * ldw + w] = Tt * r3 - dT;
    }
  }
}

// The terms of one (channel, link) pair (TdiTilePair): per term its centre
// sample (compensated), its linear-interpolation part (exact product,
// compensated) and the drift of its fraction; then the pair's combined FIR on
// the differences and its two moment corrections.
template <int K, int SPT>
__device__ __forceinline__ void apply_pair(f2 (&main)[SPT], f2 (&acc)[SPT],
                                           const float2* __restrict__ yw,
                                           const float2* __restrict__ dyw, const TdiTilePair& P,
                                           int s0, int hl, int rows, int lane) {
  const int base = s0 + hl;
  for (int q = 0; q < P.nterm; ++q) {
    const TdiTermLite& T = P.t[q];
    if (T.kind == 0) {
      add_rows<SPT>(main, acc, yw, base, T.sg, lane);
      continue;
    }
    if (T.kind == 2) {
#pragma unroll
      for (int r = 0; r < SPT; ++r) {
        const float4 v = split_one<K>(yw, &T, s0 + r, hl, rows, lane);
        acc2(main[r].x, acc[r].x, T.sg * v.x);
        acc2(main[r].y, acc[r].y, T.sg * v.y);
        acc[r].x = fmaf(T.sg, v.z, acc[r].x);
        acc[r].y = fmaf(T.sg, v.w, acc[r].y);
      }
      continue;
    }
    const int c0 = base + T.bo;
    add_rows<SPT>(main, acc, yw, c0, T.sg, lane);
    const float se = T.se, a1 = T.sa1, a2 = T.sa2;
#pragma unroll
    for (int r = 0; r < SPT; ++r) {
      const f2 d = ld2(&dyw[(c0 + r) * kPW2 + lane]);
      const float jj = (float)(s0 + r);
      const float dr = jj * fmaf(jj, a2, a1);
      acc[r].x = fmaf(dr, d.x, acc[r].x);
      acc[r].y = fmaf(dr, d.y, acc[r].y);
      const float px = se * d.x, py = se * d.y;
      const float ex = fmaf(se, d.x, -px), ey = fmaf(se, d.y, -py);
      acc2(main[r].x, acc[r].x, px);
      acc2(main[r].y, acc[r].y, py);
      acc[r].x += ex;
      acc[r].y += ey;
    }
  }
  const int nt4 = P.ntap4;
  if (nt4 == 0) return;
  {
    const int ca = base + P.ma, cb = base + P.mb;
    const float wa = P.wa, wb = P.wb;
#pragma unroll
    for (int r = 0; r < SPT; ++r) {
      const f2 da = ld2(&dyw[(ca + r) * kPW2 + lane]);
      const f2 db = ld2(&dyw[(cb + r) * kPW2 + lane]);
      acc[r].x = fmaf(wa, da.x, fmaf(wb, db.x, acc[r].x));
      acc[r].y = fmaf(wa, da.y, fmaf(wb, db.y, acc[r].y));
    }
  }
  const int b0 = base + P.boff;
  f2 win[SPT];
#pragma unroll
  for (int r = 0; r < SPT; ++r) win[r] = ld2(&dyw[(b0 + r) * kPW2 + lane]);
  const float4* G4 = reinterpret_cast<const float4*>(P.G);
#pragma unroll 1
  for (int k = 0; k < nt4; k += 4) {
    const float4 g = G4[k >> 2];
    const float gk[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int r = 0; r < SPT; ++r) {
        acc[r].x = fmaf(gk[u], win[r].x, acc[r].x);
        acc[r].y = fmaf(gk[u], win[r].y, acc[r].y);
      }
#pragma unroll
      for (int r = 0; r < SPT - 1; ++r) win[r] = win[r + 1];
      win[SPT - 1] = ld2(&dyw[(b0 + SPT + k + u) * kPW2 + lane]);
    }
  }
}

// Mixed TDI with one combined FIR per (channel, link) pair: the CTA shape,
// staging, accumulators and A, E, T epilogue of tdi_mixed_kernel.
template <int K>
__global__ void __launch_bounds__(32 * kMixWarps, 1) tdi_comb_kernel(
    const TdiTilePair* __restrict__ pairs, int W, int ldw, int64_t n, const float* __restrict__ y,
    float* __restrict__ out, const float* __restrict__ data, int resid, int hl, int hr,
    const int64_t* __restrict__ woff) {
  constexpr int SPT = kMixSpt;
  extern __shared__ float2 smem2[];
  const int rows = kMixTile + hl + hr;
  float2* ybuf0 = smem2;                           // [rows][kPW2], links 0, 2, 4
  float2* ybuf1 = smem2 + rows * kPW2;             // links 1, 3, 5
  float2* dyw = smem2 + 2 * rows * kPW2;           // dy_r = y_{r+1} - y_r of the current link
  __shared__ TdiTilePair pp[kTdiPairs];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int tid = warp * 32 + lane;
  const int64_t i0 = (int64_t)blockIdx.x * kMixTile;
  const int wa = blockIdx.y * 64 + 2 * lane;       // walkers wa, wa + 1
  const int s0 = warp * SPT;
  if (woff && group_inactive(woff + blockIdx.y * 64, 64, i0 + kMixTile)) return;
  const int64_t lo_a = woff ? woff[wa] : 0, lo_b = woff ? woff[wa + 1] : 0;
  {
    const int4* src = reinterpret_cast<const int4*>(pairs + (int64_t)blockIdx.x * kTdiPairs);
    int4* dst = reinterpret_cast<int4*>(pp);
    const int words = kTdiPairs * (int)(sizeof(TdiTilePair) / sizeof(int4));
    for (int q = tid; q < words; q += 32 * kMixWarps) dst[q] = src[q];
  }
  f2 mx[SPT], my[SPT], mz[SPT], sx[SPT], sy[SPT], sz[SPT];
#pragma unroll
  for (int r = 0; r < SPT; ++r)
    mx[r] = my[r] = mz[r] = sx[r] = sy[r] = sz[r] = f2{0.0f, 0.0f};

  auto stage = [&](int j, float2* dst) {
    for (int r = warp; r < rows; r += kMixWarps) {
      const int64_t g = i0 - hl + r;
      float* d = reinterpret_cast<float*>(dst + r * kPW2 + lane);
      const bool in = g >= 0 && g < n;
      const float* src = in ? y + ((int64_t)j * n + g) * ldw + wa : y;
      if (in && g >= lo_a && wa < W) cp_async4(d, src); else d[0] = 0.0f;
      if (in && g >= lo_b && wa + 1 < W) cp_async4(d + 1, src + 1); else d[1] = 0.0f;
    }
    cp_async_commit();
  };
  stage(0, ybuf0);
  for (int j = 0; j < kNLink; ++j) {
    float2* yw = (j & 1) ? ybuf1 : ybuf0;
    if (j + 1 < kNLink) {
      stage(j + 1, (j & 1) ? ybuf0 : ybuf1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    for (int r = warp; r < rows; r += kMixWarps) {
      float2 a = yw[r * kPW2 + lane];
      float2 b = r + 1 < rows ? yw[(r + 1) * kPW2 + lane] : a;
      dyw[r * kPW2 + lane] = make_float2(b.x - a.x, b.y - a.y);
    }
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {
      const TdiTilePair& P = pp[2 * j + k];
      if (P.nterm == 0) continue;
      if (P.chan == 0) apply_pair<K, SPT>(mx, sx, yw, dyw, P, s0, hl, rows, lane);
      else if (P.chan == 1) apply_pair<K, SPT>(my, sy, yw, dyw, P, s0, hl, rows, lane);
      else apply_pair<K, SPT>(mz, sz, yw, dyw, P, s0, hl, rows, lane);
    }
    __syncthreads();                               // link j's buffers are free again
  }
  const float r2 = 0.70710678118654752f, r6 = 0.40824829046386302f, r3 = 0.57735026918962576f;
#pragma unroll
  for (int r = 0; r < SPT; ++r) {
    const int64_t i = i0 + s0 + r;
    if (i >= n) continue;
    float dA = 0.0f, dE = 0.0f, dT = 0.0f;
    if (resid) {
      dA = data[i];
      dE = data[n + i];
      dT = data[2 * n + i];
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int w = wa + e;
      if (w >= W || i < (e ? lo_b : lo_a)) continue;
      const float Mx = e ? mx[r].y : mx[r].x, My = e ? my[r].y : my[r].x, Mz = e ? mz[r].y : mz[r].x;
      const float Sx = e ? sx[r].y : sx[r].x, Sy = e ? sy[r].y : sy[r].x, Sz = e ? sz[r].y : sz[r].x;
      df32 zx = two_sum(Mz, -Mx);
      df32 xy = two_sum(Mx, -2.0f * My);
      df32 xyz = two_sum(xy.hi, Mz);
      df32 xy3 = two_sum(Mx, My);
      df32 t3 = two_sum(xy3.hi, Mz);
      const float A = zx.hi + (zx.lo + (Sz - Sx));
      const float E = xyz.hi + ((xy.lo + xyz.lo) + (Sx - 2.0f * Sy + Sz));
      const float Tt = t3.hi + ((xy3.lo + t3.lo) + (Sx + Sy + Sz));
      out[(0 * n + i) * ldw + w] = A * r2 - dA;
      out[(1 * n + i) * ldw + w] = E * r6 - dE;
      out[(2 * n + i) * ldw + w] = Tt * r3 - dT;
    }
  }
}

template <int K>
cudaError_t launch_k(const lisa_td_ctx* c, int W, int ldw, const void* y, void* out, int resid,
                     cudaStream_t s, int nd) {
  constexpr int SPT = 16;
  constexpr int TILE = 4 * SPT;
  const double dt = c->cfg.dt;
  int hl = (int)ceil(nd * 1.1 * kArmSec / dt) + K / 2 + 2;
  int hr = K / 2 + 2;
  int groups = (W + 31) / 32;
  dim3 grid((unsigned)((c->n + TILE - 1) / TILE), (unsigned)groups);
  dim3 block(32, 4);
  if (c->cfg.precision == 0) {
    size_t smem = (size_t)(TILE + hl + hr) * kPW * sizeof(double);
    cudaFuncSetAttribute(tdi_fp64_kernel<K, SPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    tdi_fp64_kernel<K, SPT><<<grid, block, smem, s>>>(
        c->tdi_tab, W, ldw, ldw, c->n, dt, c->orb64, (const double*)y, (double*)out, c->data64,
        resid, hl, hr, c->woff, c->cfg.tdi_nested);
  } else {
    int hlm = (int)ceil(nd * 1.1 * kArmSec / dt) + K / 2 + 3;
    int hrm = K / 2 + 2;
    size_t smem = (size_t)3 * (kMixTile + hlm + hrm) * kPW2 * sizeof(float2);
    dim3 gridm((unsigned)((c->n + kMixTile - 1) / kMixTile), (unsigned)((W + 63) / 64));
    cudaFuncSetAttribute(tdi_mixed_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    dim3 blockm(32, kMixTile / kMixSpt);
    if (c->tdi_comb) {
      // the combined FIR reads up to 3 zero-weight taps past a pair's window
      const int hrc = hrm + 4;
      const size_t smc = (size_t)3 * (kMixTile + hlm + hrc) * kPW2 * sizeof(float2);
      cudaFuncSetAttribute(tdi_comb_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smc);
      tdi_comb_kernel<K><<<gridm, blockm, smc, s>>>(c->tdi_pairs, W, ldw, c->n,
                                                   (const float*)y, (float*)out, c->data32,
                                                   resid, hlm, hrc, c->woff);
    } else {
      tdi_mixed_kernel<K><<<gridm, blockm, smem, s>>>(c->tdi_tab, c->tdi_tiles, W, ldw, c->n,
                                                     (const float*)y, (float*)out, c->data32,
                                                     resid, hlm, hrm, c->woff);
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tdi_tiles(const lisa_td_ctx* c, cudaStream_t s) {
  const int ntiles = (int)((c->n + kTdiTile - 1) / kTdiTile);
  const int64_t m = (int64_t)ntiles * c->n_dterms;
  tdi_tiles_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(
      c->tdi_tab, c->orb64, c->n, c->cfg.dt, c->cfg.lagrange_order + 1, ntiles,
      c->cfg.tdi_nested, c->tdi_tiles);
  return cudaGetLastError();
}

cudaError_t launch_tdi_pairs(const lisa_td_ctx* c, cudaStream_t s) {
  const int ntiles = (int)((c->n + kTdiTile - 1) / kTdiTile);
  const int64_t m = (int64_t)ntiles * kTdiPairs;
  tdi_pairs_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(
      c->tdi_tab, c->orb64, c->n, c->cfg.dt, c->cfg.lagrange_order + 1, ntiles,
      c->cfg.tdi_nested, c->tdi_pairs, c->tdi_flag);
  return cudaGetLastError();
}

cudaError_t launch_tdi(const lisa_td_ctx* c, int W, int ldw, const void* y, void* out, int resid,
                       cudaStream_t s) {
  int nd = c->tdi_nd;
  switch (c->cfg.lagrange_order) {
    case 1: return launch_k<2>(c, W, ldw, y, out, resid, s, nd);
    case 3: return launch_k<4>(c, W, ldw, y, out, resid, s, nd);
    case 5: return launch_k<6>(c, W, ldw, y, out, resid, s, nd);
    case 7: return launch_k<8>(c, W, ldw, y, out, resid, s, nd);
    case 15: return launch_k<16>(c, W, ldw, y, out, resid, s, nd);
    case 31: return launch_k<32>(c, W, ldw, y, out, resid, s, nd);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lisa
