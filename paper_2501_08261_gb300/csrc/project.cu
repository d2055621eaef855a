// Link responses y_slr on the grid (Sec. II.B, Eq. yslr):
//   n = unit(r_r(t) - r_s(t - L_l)), x+ = (u.n)^2 - (v.n)^2, xx = (u.n)(v.n),
//   t_s = t - L_l - k.r_s,  t_r = t - k.r_r,
//   y = [x+ (h+(t_s) - h+(t_r)) + 2 xx (hx(t_s) - hx(t_r))] / (2 (1 - k.n)),
// h at t_s, t_r by centred Lagrange interpolation (zero outside the grid).
//
// Layout: one CTA = 32 walkers (lanes) x a tile of samples (warps stride the
// tile).  Each walker's h window, shifted by its own barycentric delay
// k.g(t)/dt, is staged in shared memory [row][walker] (rows padded to 33) so
// that the nine stencils of every sample read conflict-free columns.
#include <math.h>

#include "internal.h"
#include "lagrange.cuh"

namespace lisa {

namespace {

constexpr int kPW = 33;                 // padded walkers per shared-memory row

// every walker of the 32-walker group starts its window at or after row `end`
// (walkers are sorted by window start, but take the minimum to be safe)
__device__ inline bool tile_inactive(const int64_t* __restrict__ woff32, int64_t end) {
  int64_t m = woff32[0];
#pragma unroll 8
  for (int k = 1; k < 32; ++k) m = woff32[k] < m ? woff32[k] : m;
  return m >= end;
}

template <int K>
__global__ void __launch_bounds__(128) project_fp64_kernel(
    const WalkerRec* __restrict__ walkers, int W, int ldw, int64_t n, double t0, double dt,
    const OrbitRec64* __restrict__ orb, const double2* __restrict__ h, double* __restrict__ y,
    int tile, int halo, const int64_t* __restrict__ woff, double phase) {
  extern __shared__ double2 win[];      // [(tile + 2 halo)][kPW]
  __shared__ int shift_s[32];
  __shared__ double cinv_s[K];
  const int lane = threadIdx.x, warp = threadIdx.y, nw = blockDim.y;
  const int tid = warp * 32 + lane;
  const int64_t i0 = (int64_t)blockIdx.x * tile;
  const int w = blockIdx.y * 32 + lane;
  const int rows = tile + 2 * halo;
  if (woff && tile_inactive(woff + blockIdx.y * 32, i0 + tile)) return;
  const int64_t lo = woff ? woff[w] : 0;        // this walker's window starts at row lo
  if (tid < K) cinv_s[tid] = lagrange_denom_inv<double, K>(tid);
  if (warp == 0) {
    const WalkerRec& R = walkers[w];
    double tc = t0 + ((double)i0 + 0.5 * tile) * dt;
    double a = kOmegaOrb * tc + phase;
    double S = kAUSec * (R.k[0] * cos(a) + R.k[1] * sin(a));
    shift_s[lane] = (int)floor(S / dt);
  }
  __syncthreads();
  // stage: warp q loads walkers q, q + nw, ... (coalesced along samples)
  for (int ww = warp; ww < 32; ww += nw) {
    const int64_t a0 = i0 - shift_s[ww] - halo;
    const double2* hw = h + (int64_t)(blockIdx.y * 32 + ww) * n;
    const int64_t lw = woff ? woff[blockIdx.y * 32 + ww] : 0;
    for (int r = lane; r < rows; r += 32) {
      int64_t g = a0 + r;
      win[r * kPW + ww] = (g >= lw && g >= 0 && g < n) ? hw[g] : make_double2(0.0, 0.0);
    }
  }
  __syncthreads();
  const WalkerRec& R = walkers[w];
  const double k0 = R.k[0], k1 = R.k[1], k2 = R.k[2];
  const int64_t a0 = i0 - shift_s[lane] - halo;
  const double2* hw = h + (int64_t)w * n;
  double cinv[K];
#pragma unroll
  for (int j = 0; j < K; ++j) cinv[j] = cinv_s[j];

  // tau is relative to the window start lo (so that the fraction rounds as
  // on a grid that starts there)
  auto interp = [&](double tau, double& hp, double& hc) {
    double fl = floor(tau);
    double eps = tau - fl;
    double wts[K];
    lagrange_weights<double, K>(eps, cinv, wts);
    int64_t base = lo + (int64_t)fl - (K - 2) / 2;
    int64_t loc = base - a0;
    double sp = 0.0, sc = 0.0;
    if (loc >= 0 && loc + K <= rows) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        double2 v = win[(loc + j) * kPW + lane];
        sp += wts[j] * v.x;
        sc += wts[j] * v.y;
      }
    } else {                                   // outside the staged window: global reads
      for (int j = 0; j < K; ++j) {
        int64_t g = base + j;
        if (g >= lo && g >= 0 && g < n) {
          double2 v = hw[g];
          sp += wts[j] * v.x;
          sc += wts[j] * v.y;
        }
      }
    }
    hp = sp;
    hc = sc;
  };

  for (int s = warp; s < tile; s += nw) {
    const int64_t i = i0 + s;
    if (i >= n) break;
    const OrbitRec64& O = orb[i];
    double hpr[3], hcr[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double kr = k0 * O.rr[q][0] + k1 * O.rr[q][1] + k2 * O.rr[q][2];
      interp((double)(i - lo) - kr / dt, hpr[q], hcr[q]);
    }
#pragma unroll
    for (int j = 0; j < kNLink; ++j) {
      const int rq = link_receiver(j);
      double ks = k0 * O.rs[j][0] + k1 * O.rs[j][1] + k2 * O.rs[j][2];
      double hps, hcs;
      interp((double)(i - lo) - (O.L[j] + ks) / dt, hps, hcs);
      double nx = O.n[j][0], ny = O.n[j][1], nz = O.n[j][2];
      double un = R.u[0] * nx + R.u[1] * ny + R.u[2] * nz;
      double vn = R.v[0] * nx + R.v[1] * ny + R.v[2] * nz;
      double kn = k0 * nx + k1 * ny + k2 * nz;
      double val = ((un * un - vn * vn) * (hps - hpr[rq]) + 2.0 * un * vn * (hcs - hcr[rq])) /
                   (2.0 * (1.0 - kn));
      if (w < W && i >= lo) y[((int64_t)j * n + i) * ldw + w] = val;
    }
  }
}

// Mixed path.  Per tile and walker one FP64 anchor S_a = k.g(t_a) (split into
// an integer sample shift and a fraction); per sample the change of k.g over
// the tile (a second-order expansion in Omega dt, error < 1e-9 s) and the
// spacecraft offsets k.rho (FP32 table relative to g) enter only as small
// FP32 numbers next to exact integers.
//
// Lagrange weights: the paired form (lagrange.cuh) for K >= 8, its per-pair
// constants passed as a kernel parameter (constant bank).  The staged window
// covers every stencil by construction (halo), so the stencils read shared
// memory without a bounds branch and can be interleaved; a stencil found
// outside the window is recomputed through the bounds-checked path.
template <int K>
__global__ void __launch_bounds__(256, 2) project_mixed_kernel(
    const WalkerRec* __restrict__ walkers, int W, int ldw, int64_t n, double t0, double dt,
    const OrbitRec32* __restrict__ orb, const float2* __restrict__ h, float* __restrict__ y,
    int tile, int halo, int nL, float rL, const int64_t* __restrict__ woff,
    const LagrangePairs pairs, double phase) {
  // shared memory: (h+, hx) pairs [rows][32] -- 256-byte rows, so that a
  // 64-bit load of lane w touches banks 2w, 2w+1 whatever row each walker's
  // stencil is on (conflict-free per half-warp) -- then the orbit records
  extern __shared__ float2 smf2[];
  const int rows = tile + 2 * halo;
  float2* hws = smf2;
  OrbitRec32* ors = reinterpret_cast<OrbitRec32*>(smf2 + rows * 32);
  __shared__ int shift_s[32];
  __shared__ float fra_s[32], p1_s[32], sa_s[32];
  __shared__ float cinv_s[K];
  const int lane = threadIdx.x, warp = threadIdx.y, nw = blockDim.y;
  const int tid = warp * 32 + lane, nth = 32 * nw;
  const int64_t i0 = (int64_t)blockIdx.x * tile;
  const int w = blockIdx.y * 32 + lane;
  if (woff && tile_inactive(woff + blockIdx.y * 32, i0 + tile)) return;
  const int64_t lo = woff ? woff[w] : 0;        // this walker's window starts at row lo
  if (tid < K) cinv_s[tid] = lagrange_denom_inv<float, K>(tid);
  if (warp == 0) {
    const WalkerRec& R = walkers[w];
    double ta = t0 + (double)i0 * dt;
    double a = kOmegaOrb * ta + phase;
    double ca = cos(a), sa = sin(a);
    double S = kAUSec * (R.k[0] * ca + R.k[1] * sa);
    double sh = floor(S / dt);
    shift_s[lane] = (int)sh;
    fra_s[lane] = (float)(S / dt - sh);
    p1_s[lane] = (float)(kAUSec * (-R.k[0] * sa + R.k[1] * ca));
    sa_s[lane] = (float)S;
  }
  {  // orbit records of the tile (coalesced words)
    const int64_t nrec = (i0 + tile <= n) ? tile : (n - i0);
    const int words = (int)nrec * (int)(sizeof(OrbitRec32) / sizeof(float));
    const float* src = reinterpret_cast<const float*>(orb + i0);
    float* dst = reinterpret_cast<float*>(ors);
    for (int q = tid; q < words; q += nth) dst[q] = src[q];
  }
  __syncthreads();
  {  // h windows: lane = walker, each warp a strided set of rows
    const int64_t a0w = i0 - shift_s[lane] - halo;
    const float2* hw = h + (int64_t)w * n;
    for (int r = warp; r < rows; r += nw) {
      int64_t g = a0w + r;
      hws[r * 32 + lane] = (g >= lo && g >= 0 && g < n) ? hw[g] : make_float2(0.0f, 0.0f);
    }
  }
  __syncthreads();
  const MixRec& X = walkers[w].mx;
  const float k0 = X.k[0], k1 = X.k[1], k2 = X.k[2];
  const float u0 = X.u[0], u1 = X.u[1], u2 = X.u[2];
  const float v0 = X.v[0], v1 = X.v[1], v2 = X.v[2];
  const int64_t a0 = i0 - shift_s[lane] - halo;
  const float fra = fra_s[lane], p1 = p1_s[lane], sa = sa_s[lane];
  const float idt = (float)(1.0 / dt);
  const float odt = (float)(kOmegaOrb * dt);
  const float2* hw = h + (int64_t)w * n;
  float cinv[K];
  if constexpr (K < 8) {
#pragma unroll
    for (int j = 0; j < K; ++j) cinv[j] = cinv_s[j];
  }
  auto weights = [&](float e, float* wts) {
    if constexpr (K >= 8) lagrange_weights_paired<K>(e, pairs, wts);
    else lagrange_weights<float, K>(e, cinv, wts);
  };

  // interpolate h at local row position `row0 + f` (row0 integer, f small),
  // reading global memory where the stencil leaves the staged window
  auto interp = [&](int row0, float f, float& hp, float& hc) {
    float fl = floorf(f);
    float wts[K];
    weights(f - fl, wts);
    int loc = row0 + (int)fl - (K - 2) / 2;
    float sp = 0.0f, sc = 0.0f;
    if (loc >= 0 && loc + K <= rows) {
      float sp1 = 0.0f, sc1 = 0.0f;                // two chains each (FMA latency)
#pragma unroll
      for (int j = 0; j < K; j += 2) {
        const float2 v = hws[(loc + j) * 32 + lane];
        const float2 u = hws[(loc + j + 1) * 32 + lane];
        sp = fmaf(wts[j], v.x, sp);
        sc = fmaf(wts[j], v.y, sc);
        sp1 = fmaf(wts[j + 1], u.x, sp1);
        sc1 = fmaf(wts[j + 1], u.y, sc1);
      }
      sp += sp1;
      sc += sc1;
    } else {
      for (int j = 0; j < K; ++j) {
        int64_t g = a0 + loc + j;
        if (g >= lo && g >= 0 && g < n) {
          float2 v = hw[g];
          sp = fmaf(wts[j], v.x, sp);
          sc = fmaf(wts[j], v.y, sc);
        }
      }
    }
    hp = sp;
    hc = sc;
  };

  // the same from the staged window only; `bad` records a stencil outside it
  auto interp_fast = [&](int row0, float f, float& hp, float& hc, bool& bad) {
    float fl = floorf(f);
    float wts[K];
    weights(f - fl, wts);
    int loc = row0 + (int)fl - (K - 2) / 2;
    const bool inr = loc >= 0 && loc + K <= rows;
    bad = bad || !inr;
    loc = inr ? loc : 0;
    float sp = 0.0f, sc = 0.0f, sp1 = 0.0f, sc1 = 0.0f;   // two chains each (FMA latency)
#pragma unroll
    for (int j = 0; j < K; j += 2) {
      const float2 v = hws[(loc + j) * 32 + lane];
      const float2 u = hws[(loc + j + 1) * 32 + lane];
      sp = fmaf(wts[j], v.x, sp);
      sc = fmaf(wts[j], v.y, sc);
      sp1 = fmaf(wts[j + 1], u.x, sp1);
      sc1 = fmaf(wts[j + 1], u.y, sc1);
    }
    hp = sp + sp1;
    hc = sc + sc1;
  };

  for (int s = warp; s < tile; s += nw) {
    const int64_t i = i0 + s;
    if (i >= n) break;
    const OrbitRec32& O = ors[s];
    const float d = odt * (float)s;
    const float dS = d * p1 - 0.5f * d * d * sa;     // k.g(t) - k.g(t_a)
    const float base_f = -fra - dS * idt;
    float hpr[3], hcr[3];
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float kr = k0 * O.rr[q][0] + k1 * O.rr[q][1] + k2 * O.rr[q][2];
      interp_fast(s + halo, base_f - kr * idt, hpr[q], hcr[q], bad);
    }
    if (bad) {
#pragma unroll 1
      for (int q = 0; q < 3; ++q) {
        float kr = k0 * O.rr[q][0] + k1 * O.rr[q][1] + k2 * O.rr[q][2];
        float a, b;
        interp(s + halo, base_f - kr * idt, a, b);
        if (q == 0) { hpr[0] = a; hcr[0] = b; }
        else if (q == 1) { hpr[1] = a; hcr[1] = b; }
        else { hpr[2] = a; hcr[2] = b; }
      }
    }
    // six senders, two per iteration: the fully unrolled nine-stencil body
    // (~36 KB of code) stalled on instruction fetch
#pragma unroll 2
    for (int j = 0; j < kNLink; ++j) {
      float ks = k0 * O.rs[j][0] + k1 * O.rs[j][1] + k2 * O.rs[j][2];
      const float fs = base_f - rL - (O.L[j] + ks) * idt;
      float hs, cs;
      bool bj = false;
      interp_fast(s + halo - nL, fs, hs, cs, bj);
      if (bj) interp(s + halo - nL, fs, hs, cs);
      const int rq = link_receiver(j);
      const float hr = rq == 0 ? hpr[0] : (rq == 1 ? hpr[1] : hpr[2]);
      const float cr = rq == 0 ? hcr[0] : (rq == 1 ? hcr[1] : hcr[2]);
      float nx = O.n[j][0], ny = O.n[j][1], nz = O.n[j][2];
      float un = u0 * nx + u1 * ny + u2 * nz;
      float vn = v0 * nx + v1 * ny + v2 * nz;
      float kn = k0 * nx + k1 * ny + k2 * nz;
      float val = ((un * un - vn * vn) * (hs - hr) + 2.0f * un * vn * (cs - cr)) /
                  (2.0f * (1.0f - kn));
      if (w < W && i >= lo) y[((int64_t)j * n + i) * ldw + w] = val;
    }
  }
}

template <int K>
cudaError_t launch_k(const lisa_td_ctx* c, int W, int ldw, const void* h, void* y,
                     cudaStream_t s) {
  const double dt = c->cfg.dt;
  const int tile = c->tune_tile > 0 ? c->tune_tile : 128;
  // stencils reach k.(r - g) + L + the drift of k.g over the tile from the
  // guiding centre's shift; orb_dev widens it for the caller's orbit tables
  int halo = (K / 2) + 2 +
             (int)ceil((1.1 * kArmSec + kArmSec + c->orb_dev +
                        kAUSec * kOmegaOrb * tile * dt) / dt);
  int groups = (W + 31) / 32;
  dim3 grid((unsigned)((c->n + tile - 1) / tile), (unsigned)groups);
  dim3 block(32, 4);
  if (c->cfg.precision == 0) {
    size_t smem = (size_t)(tile + 2 * halo) * kPW * sizeof(double2);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(project_fp64_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    project_fp64_kernel<K><<<grid, block, smem, s>>>(c->walkers, W, ldw, c->n, c->cfg.t0, dt,
                                                     c->orb64, (const double2*)h, (double*)y,
                                                     tile, halo, c->woff, c->orb_phase);
  } else {
    size_t smem = (size_t)(tile + 2 * halo) * 32 * sizeof(float2) +
                  (size_t)tile * sizeof(OrbitRec32);
    double q = kArmSec / dt;
    int nL = (int)floor(q);
    float rL = (float)(q - nL);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(project_mixed_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    dim3 blockm(32, c->tune_warps > 0 ? c->tune_warps : 8);
    project_mixed_kernel<K><<<grid, blockm, smem, s>>>(c->walkers, W, ldw, c->n, c->cfg.t0, dt,
                                                      c->orb32, (const float2*)h, (float*)y,
                                                      tile, halo, nL, rL, c->woff,
                                                      lagrange_pairs<K>(), c->orb_phase);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_project(const lisa_td_ctx* c, int W, int ldw, const void* h, void* y,
                           cudaStream_t s) {
  switch (c->cfg.lagrange_order) {
    case 1: return launch_k<2>(c, W, ldw, h, y, s);
    case 3: return launch_k<4>(c, W, ldw, h, y, s);
    case 5: return launch_k<6>(c, W, ldw, h, y, s);
    case 7: return launch_k<8>(c, W, ldw, h, y, s);
    case 15: return launch_k<16>(c, W, ldw, h, y, s);
    case 31: return launch_k<32>(c, W, ldw, h, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lisa
