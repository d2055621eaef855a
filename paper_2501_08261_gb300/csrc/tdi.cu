// TDI Michelson X (generation 1.5 or 2.0), Y and Z by cyclic permutation, and
// A, E, T (Sec. II.B).  Every delayed term y_l(t - D(t)) takes D(t) as the plain
// sum of the link light times at the output time t and interpolates y with the
// centred Lagrange stencil; undelayed terms read y_l(t) directly.
//
// Layout: one CTA = 32 walkers (lanes) x a tile of output samples.  The kernel
// stages one link's y window at a time in shared memory and adds that link's
// terms (4 for TDI 1.5, 8 for TDI 2) into per-thread X, Y, Z accumulators.
#include <math.h>
#include <string.h>

#include "internal.h"
#include "lagrange.cuh"

namespace lisa {

namespace {

// X as printed (Sec. II.B): (link l, sign, links of the delay), y_{1-32} = link
// -3, y_{231} = 3, y_{123} = 2, y_{3-21} = -2.  TDI 2: the third y_123 term is
// read with delay 2L-2 + L2 + 2L3 + 2L-3.
struct HostTerm { int l, sign, nd, d[8]; };
const HostTerm kX15[8] = {
    {-3, +1, 3, {3, 2, -2}}, {-3, -1, 1, {3}}, {3, +1, 2, {2, -2}}, {3, -1, 0, {}},
    {2, +1, 1, {-2}}, {2, -1, 3, {-2, -3, 3}}, {-2, +1, 0, {}}, {-2, -1, 2, {-3, 3}}};
const HostTerm kX20[16] = {
    {-3, +1, 3, {3, 2, -2}}, {-3, -1, 1, {3}},
    {-3, +1, 5, {-2, 2, 3, 3, -3}}, {-3, -1, 7, {3, 3, -3, -2, -2, 2, 2}},
    {3, +1, 2, {2, -2}}, {3, -1, 0, {}},
    {3, +1, 4, {-2, 2, 3, -3}}, {3, -1, 6, {3, -3, -2, -2, 2, 2}},
    {2, +1, 1, {-2}}, {2, -1, 3, {-2, -3, 3}},
    {2, +1, 7, {-2, -2, 2, 3, 3, -3, -3}}, {2, -1, 5, {3, -3, -2, -2, 2}},
    {-2, +1, 0, {}}, {-2, -1, 2, {-3, 3}},
    {-2, +1, 6, {-2, 2, 3, 3, -3, -3}}, {-2, -1, 4, {3, -3, -2, 2}}};

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
      for (int d = 0; d < X[q].nd; ++d) t.cnt[link_index(cyc(X[q].d[d], ch))]++;
      if (X[q].nd > T.max_links_in_delay) T.max_links_in_delay = X[q].nd;
    }
  }
  return T;
}

namespace {

constexpr int kPW = 33;

template <int K, int SPT>
__global__ void __launch_bounds__(128) tdi_fp64_kernel(
    const TdiTable* __restrict__ tab, int W, int ldw_in, int ldw_out, int64_t n, double dt,
    const OrbitRec64* __restrict__ orb,
    const double* __restrict__ y, double* __restrict__ out, const double* __restrict__ data,
    int resid, int hl, int hr) {
  constexpr int NW = 4;
  constexpr int TILE = NW * SPT;
  extern __shared__ double ywin[];              // [(TILE + hl + hr)][kPW]
  __shared__ double cinv_s[K];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * TILE;
  const int w = blockIdx.y * 32 + lane;
  const int rows = TILE + hl + hr;
  if (warp == 0 && lane < K) cinv_s[lane] = lagrange_denom_inv<double, K>(lane);
  double ax[SPT], ay[SPT], az[SPT];      // X, Y, Z accumulators
#pragma unroll
  for (int s = 0; s < SPT; ++s) ax[s] = ay[s] = az[s] = 0.0;
  __syncthreads();
  double cinv[K];
#pragma unroll
  for (int j = 0; j < K; ++j) cinv[j] = cinv_s[j];

  for (int j = 0; j < kNLink; ++j) {
    __syncthreads();
    for (int r = warp; r < rows; r += NW) {
      int64_t g = i0 - hl + r;
      double v = 0.0;
      if (g >= 0 && g < n && w < W) v = y[((int64_t)j * n + g) * ldw_in + w];
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
          const double* L = orb[i].L;
          double D = 0.0;
#pragma unroll
          for (int l = 0; l < kNLink; ++l) D += (double)T.cnt[l] * L[l];
          double tau = (double)i - D / dt;
          double fl = floor(tau);
          double wts[K];
          lagrange_weights<double, K>(tau - fl, cinv, wts);
          int64_t base = (int64_t)fl - (K - 2) / 2;
          int64_t loc = base - (i0 - hl);
          v = 0.0;
          if (loc >= 0 && loc + K <= rows) {
#pragma unroll
            for (int m = 0; m < K; ++m) v += wts[m] * ywin[(loc + m) * kPW + lane];
          } else {
            for (int m = 0; m < K; ++m) {
              int64_t g = base + m;
              if (g >= 0 && g < n && w < W) v += wts[m] * y[((int64_t)j * n + g) * ldw_in + w];
            }
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
    if (i >= n) continue;
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

// Mixed path.  One CTA = 64 walkers (each lane holds walkers 2l, 2l+1) x 64
// output samples (4 warps x 16 consecutive samples).  Per link the y window is
// staged in shared memory; per term the CTA computes the walker-independent
// Lagrange weights of its 64 samples once (delay D = n_L L0 + sum cnt dL(t),
// the n_L L0 / dt part split exactly into integer + fraction), and each thread
// applies them to its 16 samples x 2 walkers with a 16-row sliding register
// window (one new shared-memory row per tap).
constexpr int kMixTile = 64;
constexpr int kMixSpt = 16;
constexpr int kPW2 = 33;                 // padded walker pairs per row

// acc[r] += sum_m wts[m][s0 + r] * y[row(r) + m] for the thread's 16 samples
template <int K>
__device__ __forceinline__ void apply_term(float2 (&acc)[kMixSpt], const float2* __restrict__ yw,
                                           const float* __restrict__ wts, const int* base_s,
                                           int s0, int b0, bool slide, int rows, int lane) {
  if (slide) {
    float2 win[kMixSpt];
#pragma unroll
    for (int r = 0; r < kMixSpt; ++r) win[r] = yw[(b0 + r) * kPW2 + lane];
#pragma unroll
    for (int m = 0; m < K; ++m) {
      float wk[kMixSpt];
#pragma unroll
      for (int r4 = 0; r4 < kMixSpt; r4 += 4) {
        float4 t4 = *reinterpret_cast<const float4*>(&wts[m * kMixTile + s0 + r4]);
        wk[r4] = t4.x; wk[r4 + 1] = t4.y; wk[r4 + 2] = t4.z; wk[r4 + 3] = t4.w;
      }
#pragma unroll
      for (int r = 0; r < kMixSpt; ++r) {
        acc[r].x = fmaf(wk[r], win[r].x, acc[r].x);
        acc[r].y = fmaf(wk[r], win[r].y, acc[r].y);
      }
      if (m + 1 < K) {
#pragma unroll
        for (int r = 0; r < kMixSpt - 1; ++r) win[r] = win[r + 1];
        win[kMixSpt - 1] = yw[(b0 + kMixSpt + m) * kPW2 + lane];
      }
    }
  } else {                                         // rare: a stencil jump inside the run
#pragma unroll
    for (int r = 0; r < kMixSpt; ++r) {
      const int b = base_s[s0 + r];
      for (int m = 0; m < K; ++m) {
        int row = b + m;
        float2 v = (row >= 0 && row < rows) ? yw[row * kPW2 + lane] : make_float2(0.0f, 0.0f);
        float wv = wts[m * kMixTile + s0 + r];
        acc[r].x = fmaf(wv, v.x, acc[r].x);
        acc[r].y = fmaf(wv, v.y, acc[r].y);
      }
    }
  }
}

__device__ __forceinline__ void add_scaled(float2 (&dst)[kMixSpt], const float2 (&src)[kMixSpt],
                                           float sg) {
#pragma unroll
  for (int r = 0; r < kMixSpt; ++r) {
    dst[r].x = fmaf(sg, src[r].x, dst[r].x);
    dst[r].y = fmaf(sg, src[r].y, dst[r].y);
  }
}

template <int K>
__global__ void __launch_bounds__(128) tdi_mixed_kernel(
    const TdiTable* __restrict__ tab, int W, int ldw, int64_t n, double dt,
    const OrbitRec32* __restrict__ orb, const float* __restrict__ y, float* __restrict__ out,
    const float* __restrict__ data, int resid, int hl, int hr) {
  extern __shared__ float2 yw[];                   // [(64 + hl + hr)][kPW2]
  __shared__ __align__(16) float wts_s[K][kMixTile];
  __shared__ int base_s[kMixTile];
  __shared__ float cinv_s[K];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int tid = warp * 32 + lane;
  const int64_t i0 = (int64_t)blockIdx.x * kMixTile;
  const int wa = blockIdx.y * 64 + 2 * lane;       // walkers wa, wa + 1
  const int rows = kMixTile + hl + hr;
  const int s0 = warp * kMixSpt;
  if (tid < K) cinv_s[tid] = lagrange_denom_inv<float, K>(tid);
  float2 ax[kMixSpt], ay[kMixSpt], az[kMixSpt];
#pragma unroll
  for (int r = 0; r < kMixSpt; ++r) ax[r] = ay[r] = az[r] = make_float2(0.0f, 0.0f);
  const double q0 = kArmSec / dt;

  for (int j = 0; j < kNLink; ++j) {
    __syncthreads();
    for (int r = warp; r < rows; r += 4) {
      int64_t g = i0 - hl + r;
      float2 v = make_float2(0.0f, 0.0f);
      if (g >= 0 && g < n) {
        const float* src = y + ((int64_t)j * n + g) * ldw;
        if (wa < W) v.x = src[wa];
        if (wa + 1 < W) v.y = src[wa + 1];
      }
      yw[r * kPW2 + lane] = v;
    }
    const int nt = tab->nterm[j];
    for (int q = 0; q < nt; ++q) {
      const TdiTerm T = tab->term[j][q];
      const float sg = (float)T.sign;
      if (T.ndelay > 0) {
        __syncthreads();                           // previous term done with wts_s
        if (tid < kMixTile) {
          const int64_t i = i0 + tid;
          double qd = q0 * (double)T.ndelay;
          double nd = floor(qd);
          float f = -(float)(qd - nd);
          if (i < n) {
            const float* L = orb[i].L;
            float dsum = 0.0f;
#pragma unroll
            for (int l = 0; l < kNLink; ++l) dsum = fmaf((float)T.cnt[l], L[l], dsum);
            f -= dsum * (float)(1.0 / dt);
          }
          float fl = floorf(f);
          float w[K];
          float ci[K];
#pragma unroll
          for (int m = 0; m < K; ++m) ci[m] = cinv_s[m];
          lagrange_weights<float, K>(f - fl, ci, w);
#pragma unroll
          for (int m = 0; m < K; ++m) wts_s[m][tid] = sg * w[m];
          // first staged row read by sample tid
          base_s[tid] = tid + hl - (int)nd + (int)fl - (K - 2) / 2;
        }
      }
      __syncthreads();
      if (T.ndelay == 0) {
        float2 acc0[kMixSpt];
#pragma unroll
        for (int r = 0; r < kMixSpt; ++r) acc0[r] = yw[(s0 + r + hl) * kPW2 + lane];
        if (T.chan == 0) add_scaled(ax, acc0, sg);
        else if (T.chan == 1) add_scaled(ay, acc0, sg);
        else add_scaled(az, acc0, sg);
        continue;
      }
      const int b0 = base_s[s0];
      const bool slide = (base_s[s0 + kMixSpt - 1] == b0 + kMixSpt - 1) && b0 >= 0 &&
                         b0 + kMixSpt - 1 + K <= rows;
      if (T.chan == 0) apply_term<K>(ax, yw, &wts_s[0][0], base_s, s0, b0, slide, rows, lane);
      else if (T.chan == 1) apply_term<K>(ay, yw, &wts_s[0][0], base_s, s0, b0, slide, rows, lane);
      else apply_term<K>(az, yw, &wts_s[0][0], base_s, s0, b0, slide, rows, lane);
    }
  }
  const float r2 = 0.70710678118654752f, r6 = 0.40824829046386302f, r3 = 0.57735026918962576f;
#pragma unroll
  for (int r = 0; r < kMixSpt; ++r) {
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
      if (w >= W) continue;
      float X = e ? ax[r].y : ax[r].x, Y = e ? ay[r].y : ay[r].x, Z = e ? az[r].y : az[r].x;
      out[(0 * n + i) * ldw + w] = (Z - X) * r2 - dA;
      out[(1 * n + i) * ldw + w] = (X - 2.0f * Y + Z) * r6 - dE;
      out[(2 * n + i) * ldw + w] = (X + Y + Z) * r3 - dT;
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
        resid, hl, hr);
  } else {
    int hlm = (int)ceil(nd * (kArmSec / dt + 0.02)) + K / 2 + 3;
    int hrm = K / 2 + 2;
    size_t smem = (size_t)(kMixTile + hlm + hrm) * kPW2 * sizeof(float2);
    dim3 gridm((unsigned)((c->n + kMixTile - 1) / kMixTile), (unsigned)((W + 63) / 64));
    cudaFuncSetAttribute(tdi_mixed_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    tdi_mixed_kernel<K><<<gridm, block, smem, s>>>(c->tdi_tab, W, ldw, c->n, dt, c->orb32,
                                                   (const float*)y, (float*)out, c->data32,
                                                   resid, hlm, hrm);
  }
  return cudaGetLastError();
}

}  // namespace

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
