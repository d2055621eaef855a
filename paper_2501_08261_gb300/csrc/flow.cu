// Affine-coupling flow of include/lisa_flow.h on the tensor cores.
//
// One CTA = 128 rows (walkers / samples) x one thread per row, 4 warps; the
// three matrix products of a coupling layer's MLP (K = 16 -> 128 -> 128 -> 16)
// run as tcgen05.mma with bf16 operands staged in shared memory in the
// K-major no-swizzle layout (tc.cuh) and fp32 accumulators in TMEM; thread r
// reads row r of each accumulator back (TMEM lane r) and applies bias, tanh
// and the coupling in fp32.  All layers run inside one launch, the layer's
// bf16 weight tiles (prepared once per parameter update by
// flow_tiles_kernel in exactly the shared-memory byte layout) copied in per
// layer.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include "../../include/lisa_flow.h"
#include "internal.h"
#include "tc.cuh"

namespace lisa {
namespace {

constexpr int kH = 128;          // hidden width (fixed: one MMA tile of N)
constexpr int kMaxD = 16;
constexpr int kMaxL = 16;
constexpr int kRows = 128;       // rows per CTA = TMEM lanes
constexpr uint32_t kWaitPolls = 1u << 22;
constexpr int kMaxTrain = 8192;  // largest training batch (per-CTA gradient partials)

// bf16 weight tiles of one layer, byte offsets (K-major no-swizzle layout)
constexpr int kT_W1 = 0;                       // [128 x 16]   W1 (h, j)
constexpr int kT_W1T = kT_W1 + 4096;           // [16 x 128]   W1^T (j, h)
constexpr int kT_W2 = kT_W1T + 4096;           // [128 x 128]  W2 (o, i)
constexpr int kT_W2T = kT_W2 + 32768;          // [128 x 128]  W2^T (i, o)
constexpr int kT_W3 = kT_W2T + 32768;          // [16 x 128]   W3 (o, h)
constexpr int kT_W3T = kT_W3 + 4096;           // [128 x 16]   W3^T (h, o)
constexpr int kTileLayer = kT_W3T + 4096;      // 81920 bytes

struct FlowArgs {
  int D, L;
  int idx[kMaxD];
  int perm[kMaxL][kMaxD];
  int da[kMaxL];
  int off[kMaxL][6];             // float offsets of W1, b1, W2, b2, W3, b3
  const uint8_t* tiles;          // [L][kTileLayer]
  const float* master;           // packed fp32 parameters
  const double* mu;              // [15]
  const double* scale;           // [D]
  uint32_t wait_polls;           // limit of a wait on tensor-core work (flow_set_wait_limit)
};

__device__ __forceinline__ float pick(const float (&v)[kMaxD], int k) {
  float r = 0.0f;
#pragma unroll
  for (int j = 0; j < kMaxD; ++j)
    if (j == k) r = v[j];
  return r;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// 8 consecutive K entries of one row as a 16-byte chunk
__device__ __forceinline__ void st8(uint8_t* base, int r, int k0, int K, const float* v) {
  uint4 q;
  q.x = pack2(v[0], v[1]);
  q.y = pack2(v[2], v[3]);
  q.z = pack2(v[4], v[5]);
  q.w = pack2(v[6], v[7]);
  *reinterpret_cast<uint4*>(base + tc::kmaj_off(r, k0, K)) = q;
}

__device__ __forceinline__ void copy16(uint8_t* dst, const uint8_t* src, int bytes, int tid,
                                       int nth) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int q = tid; q < bytes / 16; q += nth) d[q] = s[q];
}

// one tcgen05 GEMM D[128 x N] = A[128 x K] B[N x K]^T, K a multiple of 16,
// issued by thread 0; with mbar != nullptr, a commit to it follows (one
// commit covers every MMA this thread issued before it, so a group of GEMMs
// is waited for with one phase of the barrier)
__device__ __forceinline__ void gemm_issue(uint32_t d_tmem, const uint8_t* A, const uint8_t* B,
                                           int K, int N, uint64_t* mbar) {
  tc::fence_after();
  const uint32_t sbo = (uint32_t)K * 16;
  for (int ks = 0; ks < K / 16; ++ks)
    tc::mma(d_tmem, tc::sdesc(A + ks * 256, 128, sbo), tc::sdesc(B + ks * 256, 128, sbo),
            tc::idesc_bf16(128, N), ks > 0 ? 1u : 0u);
  if (mbar) tc::commit(mbar);
}

// ---------------------------------------------------------------------------
// Parameters -> bf16 tiles of every layer (after each parameter update).
// ---------------------------------------------------------------------------
__global__ void flow_tiles_kernel(FlowArgs a, uint8_t* __restrict__ tiles) {
  const int l = blockIdx.y;
  const int da = a.da[l], db = a.D - da;
  const float* W1 = a.master + a.off[l][0];
  const float* W2 = a.master + a.off[l][2];
  const float* W3 = a.master + a.off[l][4];
  uint8_t* T = tiles + (size_t)l * kTileLayer;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kH * kH; e += gridDim.x * blockDim.x) {
    const int r = e / kH, c = e % kH;
    // W2 (o = r, i = c) and W2^T (i = r, o = c)
    *reinterpret_cast<__nv_bfloat16*>(T + kT_W2 + tc::kmaj_off(r, c, kH)) =
        __float2bfloat16_rn(W2[r * kH + c]);
    *reinterpret_cast<__nv_bfloat16*>(T + kT_W2T + tc::kmaj_off(r, c, kH)) =
        __float2bfloat16_rn(W2[c * kH + r]);
    if (c < 16) {
      // W1 tile (h = r, j = c) and W1^T (j = c, h = r); W3 (o = c, h = r), W3^T (h = r, o = c)
      const float w1 = c < da ? W1[r * da + c] : 0.0f;
      *reinterpret_cast<__nv_bfloat16*>(T + kT_W1 + tc::kmaj_off(r, c, 16)) = __float2bfloat16_rn(w1);
      *reinterpret_cast<__nv_bfloat16*>(T + kT_W1T + tc::kmaj_off(c, r, kH)) = __float2bfloat16_rn(w1);
      const float w3 = c < 2 * db ? W3[c * kH + r] : 0.0f;
      *reinterpret_cast<__nv_bfloat16*>(T + kT_W3 + tc::kmaj_off(c, r, kH)) = __float2bfloat16_rn(w3);
      *reinterpret_cast<__nv_bfloat16*>(T + kT_W3T + tc::kmaj_off(r, c, 16)) = __float2bfloat16_rn(w3);
    }
  }
}

// ---------------------------------------------------------------------------
// Forward (MODE 0: x -> z, log q) or inverse (MODE 1: z -> x, log q).
// store (MODE 0, training): store[l][row][k] = input of layer l, store[L] = z.
// ---------------------------------------------------------------------------
constexpr int kFwdSmem = 4096 + 4096 + 32768 + 32768 + 4096;

template <int MODE>
__global__ void __launch_bounds__(kRows, 1) flow_fwd_kernel(FlowArgs a, const double* __restrict__ in,
                                                          int W, double* __restrict__ xout,
                                                          double* __restrict__ logq,
                                                          float* __restrict__ store, int ldstore,
                                                          int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sA1 = sm;                      // [128 x 16]  u_a
  uint8_t* sW1 = sm + 4096;               // [128 x 16]
  uint8_t* sH = sm + 8192;                // [128 x 128] h1, then h2
  uint8_t* sW2 = sm + 8192 + 32768;       // [128 x 128]
  uint8_t* sW3 = sm + 8192 + 65536;       // [16 x 128]
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = blockIdx.x * kRows + tid;
  const bool valid = row < W;
  const int D = a.D;

  if (warp == 0) tc::tmem_alloc(&tslot, 256);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tslot;
  const uint32_t tl = tbase + ((uint32_t)(warp * 32) << 16);

  float v[kMaxD];
  double zsq = 0.0, lsc = 0.0;
#pragma unroll
  for (int k = 0; k < kMaxD; ++k) v[k] = 0.0f;
  for (int k = 0; k < D; ++k) lsc += log(a.scale[k]);
  if (valid) {
#pragma unroll
    for (int k = 0; k < kMaxD; ++k) {
      if (k < D) {
        if (MODE == 0) {
          v[k] = (float)((in[(int64_t)row * 15 + a.idx[k]] - a.mu[a.idx[k]]) / a.scale[k]);
        } else {
          const double z = in[(int64_t)row * D + k];
          zsq += z * z;
          v[k] = (float)z;
        }
      }
    }
  }
  float sum_s = 0.0f;
  uint32_t phase = 0;
  bool ok = true;
  for (int step = 0; step < a.L && ok; ++step) {
    const int l = MODE == 0 ? step : a.L - 1 - step;
    const int da = a.da[l], db = D - da;
    if (MODE == 0 && store && valid) {
      for (int k = 0; k < D; ++k) store[((int64_t)l * ldstore + row) * D + k] = v[k];
    }
    {  // u_a (bf16, padded to K = 16)
      float ua[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) ua[k] = (k < da && valid) ? pick(v, a.perm[l][k]) : 0.0f;
      st8(sA1, tid, 0, 16, ua);
      st8(sA1, tid, 8, 16, ua + 8);
    }
    const uint8_t* T = a.tiles + (size_t)l * kTileLayer;
    copy16(sW1, T + kT_W1, 4096, tid, kRows);
    copy16(sW2, T + kT_W2, 32768, tid, kRows);
    copy16(sW3, T + kT_W3, 4096, tid, kRows);
    tc::fence_async_smem();
    __syncthreads();
    // GEMM 1: pre1 = u_a W1^T -> TMEM columns 0..127
    if (tid == 0) gemm_issue(tbase, sA1, sW1, 16, kH, &mbar);
    ok = tc::mbar_wait(&mbar, phase, a.wait_polls);
    phase ^= 1;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after();
    const float* b1 = a.master + a.off[l][1];
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float acc[16];
      tc::tmem_ld16(tl + c0, acc);
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = tanhf(acc[j] + __ldg(b1 + c0 + j));
      st8(sH, tid, c0, kH, acc);
      st8(sH, tid, c0 + 8, kH, acc + 8);
    }
    tc::fence_before();
    tc::fence_async_smem();
    __syncthreads();
    // GEMM 2: pre2 = h1 W2^T -> columns 128..255
    if (tid == 0) gemm_issue(tbase + 128, sH, sW2, kH, kH, &mbar);
    ok = tc::mbar_wait(&mbar, phase, a.wait_polls);
    phase ^= 1;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after();
    const float* b2 = a.master + a.off[l][3];
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float acc[16];
      tc::tmem_ld16(tl + 128 + c0, acc);
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = tanhf(acc[j] + __ldg(b2 + c0 + j));
      st8(sH, tid, c0, kH, acc);
      st8(sH, tid, c0 + 8, kH, acc + 8);
    }
    tc::fence_before();
    tc::fence_async_smem();
    __syncthreads();
    // GEMM 3: (s_raw, t) = h2 W3^T -> columns 0..15
    if (tid == 0) gemm_issue(tbase, sH, sW3, kH, 16, &mbar);
    ok = tc::mbar_wait(&mbar, phase, a.wait_polls);
    phase ^= 1;
    if (!__syncthreads_and(ok)) { ok = false; break; }
    tc::fence_after();
    float o[16];
    tc::tmem_ld16(tl, o);
    const float* b3 = a.master + a.off[l][5];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j < db) {
        float tt = 0.0f;
#pragma unroll
        for (int c = 1; c <= 8; ++c)
          if (db == c) tt = o[(c + j) & 15];
        const float s = tanhf(o[j] + __ldg(b3 + j));
        const float t = tt + __ldg(b3 + db + j);
        const int p = a.perm[l][da + j];
#pragma unroll
        for (int k = 0; k < kMaxD; ++k)
          if (k == p) v[k] = MODE == 0 ? fmaf(v[k], __expf(s), t) : (v[k] - t) * __expf(-s);
        sum_s += s;
      }
    }
    tc::fence_before();
    __syncthreads();
  }
  if (valid && ok) {
    const double lg = -0.5 * (double)D * 1.8378770664093454836;   // log(2 pi)
    if (MODE == 0) {
      double q = 0.0;
      for (int k = 0; k < D; ++k) q += (double)v[k] * (double)v[k];
      logq[row] = -0.5 * q + lg + (double)sum_s - lsc;
      if (store)
        for (int k = 0; k < D; ++k) store[((int64_t)a.L * ldstore + row) * D + k] = v[k];
    } else {
      for (int k = 0; k < 15; ++k) xout[(int64_t)row * 15 + k] = a.mu[k];
      for (int k = 0; k < D; ++k)
        xout[(int64_t)row * 15 + a.idx[k]] = a.mu[a.idx[k]] + (double)v[k] * a.scale[k];
      logq[row] = -0.5 * zsq + lg + (double)sum_s - lsc;
    }
  }
  if (!ok && tid == 0) {
    atomicExch(err, 1);
    tc::mbar_wait(&mbar, phase ^ 1, kWaitPolls);   // the phase that gave up: let a late MMA
                                                   // finish before TMEM goes
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

// ---------------------------------------------------------------------------
// Backward: gradient of -mean log q over the batch with respect to every
// parameter, all layers in one launch (last layer first).  Per layer the MLP
// forward is recomputed from the stored layer input, then
//   dOut = (ds_raw, dt)                     (fp32, from the coupling)
//   dH2  = dOut W3,   dW3^T = H2^T dOut     (tensor cores)
//   dpre2 = dH2 (1 - h2^2)
//   dH1  = dpre2 W2,  dW2 = dpre2^T H1
//   dpre1 = dH1 (1 - h1^2)
//   du_a = dpre1 W1,  dW1 = dpre1^T u_a
// Transposed operands (H1^T, H2^T, u_a^T, dOut^T, dpre^T) are written to
// shared memory beside the row-major ones so that every product reads
// K-major tiles.  Each CTA writes its partial gradient (every parameter
// once) to part[cta][nparams]; bias sums use a fixed-order reduction.
// TMEM columns: pre1 0-127, pre2 128-255, out 256-271, dW3^T 272-287,
// dH2 288-415; later dH1 288-415, dW2 128-255, du_a 256-271, dW1 272-287.
// ---------------------------------------------------------------------------
constexpr int kBwdSmem = 8 * 4096 + 6 * 32768;

__device__ __forceinline__ void warp_colsum16(const float (&v)[16], float* red_row, int lane) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    float x = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red_row[j] = x;
  }
}

// store one bf16 value at (r, k) of a K-major tile with K columns
__device__ __forceinline__ void st1(uint8_t* base, int r, int k, int K, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + tc::kmaj_off(r, k, K)) = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(kRows, 1) flow_bwd_kernel(FlowArgs a, const float* __restrict__ store,
                                                          int ldstore, int B, float invB,
                                                          int64_t nparams, float* __restrict__ part,
                                                          int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sXa = sm;                  // [128 x 16]  u_a
  uint8_t* sXaT = sm + 4096;          // [16 x 128]  u_a^T
  uint8_t* sW1 = sm + 2 * 4096;       // [128 x 16]
  uint8_t* sW1T = sm + 3 * 4096;      // [16 x 128]
  uint8_t* sW3 = sm + 4 * 4096;       // [16 x 128]
  uint8_t* sW3T = sm + 5 * 4096;      // [128 x 16]
  uint8_t* sdO = sm + 6 * 4096;       // [128 x 16]  dOut
  uint8_t* sdOT = sm + 7 * 4096;      // [16 x 128]  dOut^T
  uint8_t* Bf[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) Bf[q] = sm + 8 * 4096 + q * 32768;
  // B0: h1 -> dpre2;  B1: h1^T;  B2: W2 -> W2^T;  B3: h2 -> dpre1;  B4: h2^T -> dpre2^T;  B5: dpre1^T
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ float red[4][kH];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = blockIdx.x * kRows + tid;
  const bool valid = row < B;
  const int D = a.D;
  float* pc = part + (int64_t)blockIdx.x * nparams;

  if (warp == 0) tc::tmem_alloc(&tslot, 512);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tslot;
  const uint32_t tl = tbase + ((uint32_t)(warp * 32) << 16);

  float dv[kMaxD];
#pragma unroll
  for (int k = 0; k < kMaxD; ++k)
    dv[k] = (valid && k < D) ? store[((int64_t)a.L * ldstore + row) * D + k] * invB : 0.0f;
  uint32_t phase = 0;
  bool ok = true;
  auto wait_all = [&]() -> bool {
    bool w = tc::mbar_wait(&mbar, phase, a.wait_polls);
    phase ^= 1;
    w = __syncthreads_and(w);
    tc::fence_after();
    return w;
  };
  auto sync_for_mma = [&]() {
    tc::fence_before();
    tc::fence_async_smem();
    __syncthreads();
  };
  // fixed-order sum of red[0..3][0..n) -> dst[0..n)
  auto flush_red = [&](float* dst, int n) {
    __syncthreads();
    if (tid < n) dst[tid] = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
    __syncthreads();
  };

  for (int step = 0; step < a.L && ok; ++step) {
    const int l = a.L - 1 - step;
    const int da = a.da[l], db = D - da;
    float vin[kMaxD];
#pragma unroll
    for (int k = 0; k < kMaxD; ++k)
      vin[k] = (valid && k < D) ? store[((int64_t)l * ldstore + row) * D + k] : 0.0f;
    {
      float ua[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) ua[k] = (k < da && valid) ? pick(vin, a.perm[l][k]) : 0.0f;
      st8(sXa, tid, 0, 16, ua);
      st8(sXa, tid, 8, 16, ua + 8);
#pragma unroll
      for (int k = 0; k < 16; ++k) st1(sXaT, k, tid, kH, ua[k]);
    }
    const uint8_t* T = a.tiles + (size_t)l * kTileLayer;
    copy16(sW1, T + kT_W1, 4096, tid, kRows);
    copy16(sW1T, T + kT_W1T, 4096, tid, kRows);
    copy16(sW3, T + kT_W3, 4096, tid, kRows);
    copy16(sW3T, T + kT_W3T, 4096, tid, kRows);
    copy16(Bf[2], T + kT_W2, 32768, tid, kRows);
    sync_for_mma();
    // forward recompute: pre1, pre2, out
    if (tid == 0) gemm_issue(tbase, sXa, sW1, 16, kH, &mbar);
    if (!(ok = wait_all())) break;
    const float* b1 = a.master + a.off[l][1];
    const float* b2 = a.master + a.off[l][3];
    const float* b3 = a.master + a.off[l][5];
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float acc[16];
      tc::tmem_ld16(tl + c0, acc);
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = tanhf(acc[j] + __ldg(b1 + c0 + j));
      st8(Bf[0], tid, c0, kH, acc);
      st8(Bf[0], tid, c0 + 8, kH, acc + 8);
#pragma unroll
      for (int j = 0; j < 16; ++j) st1(Bf[1], c0 + j, tid, kH, acc[j]);
    }
    sync_for_mma();
    if (tid == 0) gemm_issue(tbase + 128, Bf[0], Bf[2], kH, kH, &mbar);
    if (!(ok = wait_all())) break;
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float acc[16];
      tc::tmem_ld16(tl + 128 + c0, acc);
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = tanhf(acc[j] + __ldg(b2 + c0 + j));
      st8(Bf[3], tid, c0, kH, acc);
      st8(Bf[3], tid, c0 + 8, kH, acc + 8);
#pragma unroll
      for (int j = 0; j < 16; ++j) st1(Bf[4], c0 + j, tid, kH, acc[j]);
    }
    sync_for_mma();
    if (tid == 0) gemm_issue(tbase + 256, Bf[3], sW3, kH, 16, &mbar);
    if (!(ok = wait_all())) break;
    // coupling backward -> dOut; gradient wrt the transformed inputs
    {
      float o[16];
      tc::tmem_ld16(tl + 256, o);
      float dO[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) dO[k] = 0.0f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (j < db) {
          const float s = tanhf(o[j] + __ldg(b3 + j));
          const float es = __expf(s);
          const int p = a.perm[l][da + j];
          const float ub = pick(vin, p), dyb = pick(dv, p);
          const float ds = valid ? fmaf(dyb * ub, es, -invB) : 0.0f;
          const float dsr = ds * (1.0f - s * s);
#pragma unroll
          for (int c = 1; c <= 8; ++c)
            if (db == c) dO[(c + j) & 15] = dyb;
          dO[j] = dsr;
#pragma unroll
          for (int k = 0; k < kMaxD; ++k)
            if (k == p) dv[k] = dyb * es;
        }
      }
      st8(sdO, tid, 0, 16, dO);
      st8(sdO, tid, 8, 16, dO + 8);
#pragma unroll
      for (int k = 0; k < 16; ++k) st1(sdOT, k, tid, kH, dO[k]);
      warp_colsum16(dO, red[warp], lane);
      flush_red(pc + a.off[l][5], 2 * db);                      // b3
    }
    copy16(Bf[2], T + kT_W2T, 32768, tid, kRows);              // W2 -> W2^T (GEMM 2 done)
    sync_for_mma();
    if (tid == 0) {
      gemm_issue(tbase + 288, sdO, sW3T, 16, kH, nullptr);     // dH2 = dOut W3
      gemm_issue(tbase + 272, Bf[4], sdOT, kH, 16, &mbar);     // dW3^T = H2^T dOut
    }
    if (!(ok = wait_all())) break;
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float g[16], pre[16];
      tc::tmem_ld16(tl + 288 + c0, g);
      tc::tmem_ld16(tl + 128 + c0, pre);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float h = tanhf(pre[j] + __ldg(b2 + c0 + j));
        g[j] = valid ? g[j] * (1.0f - h * h) : 0.0f;
      }
      st8(Bf[0], tid, c0, kH, g);
      st8(Bf[0], tid, c0 + 8, kH, g + 8);
#pragma unroll
      for (int j = 0; j < 16; ++j) st1(Bf[4], c0 + j, tid, kH, g[j]);
      warp_colsum16(g, red[warp] + c0, lane);
    }
    flush_red(pc + a.off[l][3], kH);                            // b2
    {
      float g[16];
      tc::tmem_ld16(tl + 272, g);                               // dW3^T row h = tid
      float* w3 = pc + a.off[l][4];
#pragma unroll
      for (int o = 0; o < 16; ++o)
        if (o < 2 * db) w3[o * kH + tid] = g[o];
    }
    sync_for_mma();
    if (tid == 0) {
      gemm_issue(tbase + 288, Bf[0], Bf[2], kH, kH, nullptr);   // dH1 = dpre2 W2
      gemm_issue(tbase + 128, Bf[4], Bf[1], kH, kH, &mbar);     // dW2 = dpre2^T H1
    }
    if (!(ok = wait_all())) break;
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float g[16], pre[16];
      tc::tmem_ld16(tl + 288 + c0, g);
      tc::tmem_ld16(tl + c0, pre);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float h = tanhf(pre[j] + __ldg(b1 + c0 + j));
        g[j] = valid ? g[j] * (1.0f - h * h) : 0.0f;
      }
      st8(Bf[3], tid, c0, kH, g);
      st8(Bf[3], tid, c0 + 8, kH, g + 8);
#pragma unroll
      for (int j = 0; j < 16; ++j) st1(Bf[5], c0 + j, tid, kH, g[j]);
      warp_colsum16(g, red[warp] + c0, lane);
    }
    flush_red(pc + a.off[l][1], kH);                            // b1
    {
      float* w2 = pc + a.off[l][2] + (int64_t)tid * kH;         // dW2 row o = tid
      for (int c0 = 0; c0 < kH; c0 += 16) {
        float g[16];
        tc::tmem_ld16(tl + 128 + c0, g);
#pragma unroll
        for (int j = 0; j < 16; ++j) w2[c0 + j] = g[j];
      }
    }
    sync_for_mma();
    if (tid == 0) {
      gemm_issue(tbase + 256, Bf[3], sW1T, kH, 16, nullptr);    // du_a = dpre1 W1
      gemm_issue(tbase + 272, Bf[5], sXaT, kH, 16, &mbar);      // dW1 = dpre1^T u_a
    }
    if (!(ok = wait_all())) break;
    {
      float g[16];
      tc::tmem_ld16(tl + 256, g);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j < da) {
          const int p = a.perm[l][j];
#pragma unroll
          for (int k = 0; k < kMaxD; ++k)
            if (k == p) dv[k] += valid ? g[j] : 0.0f;
        }
      }
      tc::tmem_ld16(tl + 272, g);                               // dW1 row h = tid
      float* w1 = pc + a.off[l][0] + (int64_t)tid * da;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < da) w1[j] = g[j];
    }
    tc::fence_before();
    __syncthreads();
  }
  if (!ok && tid == 0) {
    atomicExch(err, 1);
    tc::mbar_wait(&mbar, phase ^ 1, kWaitPolls);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// grad[p] = sum over CTAs of part[cta][p] (fixed order)
__global__ void flow_reduce_kernel(const float* __restrict__ part, int ncta, int64_t np,
                                   float* __restrict__ grad) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < ncta; ++c) s += part[(int64_t)c * np + p];
    grad[p] = s;
  }
}

// loss = -mean log q over B rows (one block, fixed order); acc: optional running sum
__global__ void flow_loss_kernel(const double* __restrict__ logq, int B, float* __restrict__ loss,
                                 float* __restrict__ acc, float wacc) {
  __shared__ double r[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) s += logq[i];
  r[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) r[threadIdx.x] += r[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float L = (float)(-r[0] / B);
    if (loss) *loss = L;
    if (acc) *acc += wacc * L;
  }
}

__global__ void flow_adam_kernel(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                                 const float* __restrict__ g, int64_t np, float lr, float c1,
                                 float c2) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float gp = g[p];
    const float mp = 0.9f * m[p] + 0.1f * gp;
    const float vp = 0.999f * v[p] + 0.001f * gp * gp;
    m[p] = mp;
    v[p] = vp;
    th[p] -= lr * (mp * c1) / (sqrtf(vp * c2) + 1e-8f);
  }
}

// batch gather: out[i] = samples[(a * (first + i) + c) mod S]
__global__ void flow_gather_kernel(const double* __restrict__ samples, int64_t S, int64_t first,
                                   int Bn, int64_t mul, int64_t add, double* __restrict__ out) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= (int64_t)Bn * 15) return;
  const int64_t i = id / 15, k = id % 15;
  const int64_t src = (int64_t)(((unsigned __int128)mul * (unsigned __int128)(first + i) + add) % S);
  out[id] = samples[src * 15 + k];
}

__global__ void frame_init_kernel(double* mu, double* scale, int D) {
  const int k = threadIdx.x;
  if (k < 15) mu[k] = 0.0;
  if (k < D) scale[k] = 1.0;
}

}  // namespace
}  // namespace lisa

struct flow_ctx {
  lisa::FlowArgs args;
  int max_batch;
  int64_t nparams;
  float* master;        // [nparams]
  float* adam_m;        // [nparams]
  float* adam_v;        // [nparams]
  int adam_t;
  uint8_t* tiles;       // [L][kTileLayer]
  double* mu;           // [15]
  double* scale;        // [D]
  int* err;             // device flag: a bounded wait gave up
  int* err_host;        // pinned mirror read at the next call
  // training workspace (batches up to max_train rows)
  int max_train;
  float* store;         // [L + 1][max_train][D] layer inputs and z
  double* logq_ws;      // [max_train]
  float* part;          // [max_train / 128][nparams] per-CTA partial gradients
  float* grad_ws;       // [nparams]
  double* batch_ws;     // [max_train][15]
};

namespace {

using namespace lisa;

int flow_err(int code, const char* msg) { return report_error(code, "%s", msg); }

int cuda_err(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) return report_error(LISA_TD_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
  return report_error(LISA_TD_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// a bounded wait in an earlier launch gave up: report it once
int check_timeout(flow_ctx* f) {
  if (*(volatile int*)f->err_host) {
    *(volatile int*)f->err_host = 0;
    cudaMemset(f->err, 0, sizeof(int));
    return report_error(LISA_TD_ETIMEOUT, "a flow kernel's wait on its tensor-core work gave up");
  }
  return LISA_TD_OK;
}

void free_flow(flow_ctx* f) {
  if (!f) return;
  void* ptrs[] = {f->master, f->adam_m, f->adam_v, f->tiles, f->mu, f->scale, f->err,
                  f->store, f->logq_ws, f->part, f->grad_ws, f->batch_ws};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (f->err_host) cudaFreeHost(f->err_host);
  free(f);
}

cudaError_t refresh_tiles(flow_ctx* f, cudaStream_t s) {
  dim3 grid(32, (unsigned)f->args.L);
  flow_tiles_kernel<<<grid, 256, 0, s>>>(f->args, f->tiles);
  return cudaGetLastError();
}

int run_fwd(flow_ctx* f, int mode, const double* in, int W, double* xout, double* logq,
            float* store, int ldstore, cudaStream_t s) {
  const unsigned grid = (unsigned)((W + kRows - 1) / kRows);
  cudaError_t e;
  if (mode == 0) {
    cudaFuncSetAttribute(flow_fwd_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
    flow_fwd_kernel<0><<<grid, kRows, kFwdSmem, s>>>(f->args, in, W, xout, logq, store, ldstore, f->err);
  } else {
    cudaFuncSetAttribute(flow_fwd_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
    flow_fwd_kernel<1><<<grid, kRows, kFwdSmem, s>>>(f->args, in, W, xout, logq, store, ldstore, f->err);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->err_host, f->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  return e == cudaSuccess ? LISA_TD_OK : cuda_err(e, "flow kernel");
}

int run_grad(flow_ctx* f, const double* x, int B, float* loss, float* loss_acc, float wacc,
             float* grad, cudaStream_t s) {
  const int ld = (B + kRows - 1) / kRows * kRows;
  int rc = run_fwd(f, 0, x, B, nullptr, f->logq_ws, f->store, ld, s);
  if (rc) return rc;
  flow_loss_kernel<<<1, 256, 0, s>>>(f->logq_ws, B, loss, loss_acc, wacc);
  const int ncta = ld / kRows;
  cudaFuncSetAttribute(flow_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmem);
  flow_bwd_kernel<<<ncta, kRows, kBwdSmem, s>>>(f->args, f->store, ld, B, 1.0f / (float)B,
                                                f->nparams, f->part, f->err);
  flow_reduce_kernel<<<(unsigned)((f->nparams + 255) / 256), 256, 0, s>>>(f->part, ncta,
                                                                          f->nparams, grad);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->err_host, f->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  return e == cudaSuccess ? LISA_TD_OK : cuda_err(e, "flow gradient");
}

int run_adam(flow_ctx* f, const float* grad, float lr, cudaStream_t s) {
  f->adam_t += 1;
  const float c1 = (float)(1.0 / (1.0 - pow(0.9, f->adam_t)));
  const float c2 = (float)(1.0 / (1.0 - pow(0.999, f->adam_t)));
  flow_adam_kernel<<<(unsigned)((f->nparams + 255) / 256), 256, 0, s>>>(
      f->master, f->adam_m, f->adam_v, grad, f->nparams, lr, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = refresh_tiles(f, s);
  return e == cudaSuccess ? LISA_TD_OK : cuda_err(e, "flow_adam");
}

}  // namespace

extern "C" {

int flow_create(flow_ctx** out, int32_t dim, int32_t layers, int32_t hidden, int32_t max_batch,
                const int32_t* idx_host, const int32_t* perm_host, void* stream) {
  if (!out) return flow_err(LISA_TD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!idx_host || !perm_host) return flow_err(LISA_TD_EINVAL, "NULL argument");
  if (dim < 1 || dim > 15) return report_error(LISA_TD_EINVAL, "dim=%d must be in 1..15", dim);
  if (layers < 1 || layers > kMaxL) return report_error(LISA_TD_EINVAL, "layers=%d must be in 1..16", layers);
  if (hidden != kH) return report_error(LISA_TD_EINVAL, "hidden=%d: only 128 is supported", hidden);
  if (max_batch < 1 || max_batch > (1 << 22)) return flow_err(LISA_TD_ERANGE, "max_batch out of [1, 2^22]");
  flow_ctx* f = (flow_ctx*)calloc(1, sizeof(flow_ctx));
  if (!f) return flow_err(LISA_TD_ENOMEM, "host allocation failed");
  FlowArgs& a = f->args;
  a.D = dim;
  a.L = layers;
  a.wait_polls = kWaitPolls;
  for (int k = 0; k < dim; ++k) {
    if (idx_host[k] < 0 || idx_host[k] > 14) { free_flow(f); return flow_err(LISA_TD_EINVAL, "idx entries must be in 0..14"); }
    for (int j = 0; j < k; ++j)
      if (idx_host[j] == idx_host[k]) { free_flow(f); return flow_err(LISA_TD_EINVAL, "idx entries must be distinct"); }
    a.idx[k] = idx_host[k];
  }
  int64_t off = 0;
  for (int l = 0; l < layers; ++l) {
    int seen = 0;
    for (int k = 0; k < dim; ++k) {
      const int p = perm_host[l * dim + k];
      if (p < 0 || p >= dim || (seen >> p) & 1) { free_flow(f); return flow_err(LISA_TD_EINVAL, "perm rows must be permutations of 0..dim-1"); }
      seen |= 1 << p;
      a.perm[l][k] = p;
    }
    a.da[l] = (l % 2 == 0) ? (dim + 1) / 2 : dim / 2;
    const int da = a.da[l], db = dim - da;
    const int sizes[6] = {kH * da, kH, kH * kH, kH, 2 * db * kH, 2 * db};
    for (int q = 0; q < 6; ++q) {
      a.off[l][q] = (int)off;
      off += sizes[q];
    }
  }
  f->nparams = off;
  f->max_batch = max_batch;
  f->max_train = max_batch < kMaxTrain ? max_batch : kMaxTrain;
  const int64_t mt_pad = (f->max_train + kRows - 1) / kRows * kRows;
  cudaStream_t s = (cudaStream_t)stream;
  struct { void** p; size_t bytes; } allocs[] = {
      {(void**)&f->master, sizeof(float) * off}, {(void**)&f->adam_m, sizeof(float) * off},
      {(void**)&f->adam_v, sizeof(float) * off}, {(void**)&f->tiles, (size_t)kTileLayer * layers},
      {(void**)&f->mu, sizeof(double) * 15},      {(void**)&f->scale, sizeof(double) * kMaxD},
      {(void**)&f->err, sizeof(int)},
      {(void**)&f->store, sizeof(float) * (layers + 1) * mt_pad * dim},
      {(void**)&f->logq_ws, sizeof(double) * mt_pad},
      {(void**)&f->part, sizeof(float) * (mt_pad / kRows) * off},
      {(void**)&f->grad_ws, sizeof(float) * off},
      {(void**)&f->batch_ws, sizeof(double) * mt_pad * 15},
  };
  for (auto& al : allocs) {
    cudaError_t e = cudaMalloc(al.p, al.bytes);
    if (e != cudaSuccess) {
      *al.p = nullptr;
      free_flow(f);
      cudaGetLastError();
      return cuda_err(e, "flow_create: cudaMalloc");
    }
  }
  cudaError_t e = cudaMallocHost((void**)&f->err_host, sizeof(int));
  if (e != cudaSuccess) { free_flow(f); return cuda_err(e, "flow_create: cudaMallocHost"); }
  *f->err_host = 0;
  a.tiles = f->tiles;
  a.master = f->master;
  a.mu = f->mu;
  a.scale = f->scale;
  e = cudaMemsetAsync(f->master, 0, sizeof(float) * off, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->adam_m, 0, sizeof(float) * off, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->adam_v, 0, sizeof(float) * off, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    frame_init_kernel<<<1, 32, 0, s>>>(f->mu, f->scale, dim);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = refresh_tiles(f, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { free_flow(f); return cuda_err(e, "flow_create"); }
  *out = f;
  return LISA_TD_OK;
}

int flow_set_wait_limit(flow_ctx* f, int64_t polls) {
  if (!f) return flow_err(LISA_TD_EINVAL, "NULL context");
  if (polls > (int64_t)kWaitPolls) return flow_err(LISA_TD_ERANGE, "polls above the default limit");
  f->args.wait_polls = polls < 0 ? kWaitPolls : (uint32_t)polls;
  return LISA_TD_OK;
}

int flow_nparams(const flow_ctx* f, int64_t* n) {
  if (!f || !n) return flow_err(LISA_TD_EINVAL, "NULL argument");
  *n = f->nparams;
  return LISA_TD_OK;
}

int flow_set_params(flow_ctx* f, const float* params_dev, void* stream) {
  if (!f || !params_dev) return flow_err(LISA_TD_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(f->master, params_dev, sizeof(float) * f->nparams,
                                  cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->adam_m, 0, sizeof(float) * f->nparams, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->adam_v, 0, sizeof(float) * f->nparams, s);
  if (e == cudaSuccess) e = refresh_tiles(f, s);
  if (e != cudaSuccess) return cuda_err(e, "flow_set_params");
  f->adam_t = 0;
  return LISA_TD_OK;
}

int flow_get_params(const flow_ctx* f, float* params_dev, void* stream) {
  if (!f || !params_dev) return flow_err(LISA_TD_EINVAL, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(params_dev, f->master, sizeof(float) * f->nparams,
                                  cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? LISA_TD_OK : cuda_err(e, "flow_get_params");
}

int flow_set_frame(flow_ctx* f, const double* mu_dev, const double* scale_dev, void* stream) {
  if (!f || !mu_dev || !scale_dev) return flow_err(LISA_TD_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(f->mu, mu_dev, sizeof(double) * 15, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f->scale, scale_dev, sizeof(double) * f->args.D, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? LISA_TD_OK : cuda_err(e, "flow_set_frame");
}

int flow_logprob(flow_ctx* f, const double* x_dev, int32_t W, double* logq_dev, void* stream) {
  if (!f || !x_dev || !logq_dev) return flow_err(LISA_TD_EINVAL, "NULL argument");
  if (W < 1 || W > f->max_batch) return report_error(LISA_TD_ERANGE, "W=%d out of [1, max_batch]", W);
  int rc = check_timeout(f);
  if (rc) return rc;
  return run_fwd(f, 0, x_dev, W, nullptr, logq_dev, nullptr, 0, (cudaStream_t)stream);
}

int flow_propose(flow_ctx* f, const double* z_dev, int32_t W, double* x_dev, double* logq_dev,
                 void* stream) {
  if (!f || !z_dev || !x_dev || !logq_dev) return flow_err(LISA_TD_EINVAL, "NULL argument");
  if (W < 1 || W > f->max_batch) return report_error(LISA_TD_ERANGE, "W=%d out of [1, max_batch]", W);
  int rc = check_timeout(f);
  if (rc) return rc;
  return run_fwd(f, 1, z_dev, W, x_dev, logq_dev, nullptr, 0, (cudaStream_t)stream);
}

int flow_grad(flow_ctx* f, const double* x_dev, int32_t B, float* loss_dev, float* grad_dev,
              void* stream) {
  if (!f || !x_dev) return flow_err(LISA_TD_EINVAL, "NULL argument");
  if (B < 1 || B > f->max_train)
    return report_error(LISA_TD_ERANGE, "B=%d out of [1, %d] (training batch limit)", B, f->max_train);
  int rc = check_timeout(f);
  if (rc) return rc;
  return run_grad(f, x_dev, B, loss_dev, nullptr, 0.0f, grad_dev ? grad_dev : f->grad_ws,
                  (cudaStream_t)stream);
}

int flow_adam(flow_ctx* f, const float* grad_dev, float lr, void* stream) {
  if (!f || !grad_dev) return flow_err(LISA_TD_EINVAL, "NULL argument");
  if (!(lr > 0.0f)) return flow_err(LISA_TD_EINVAL, "lr must be > 0");
  return run_adam(f, grad_dev, lr, (cudaStream_t)stream);
}

int flow_train(flow_ctx* f, const double* samples_dev, int64_t S, int32_t epochs, int32_t batch,
               float lr, float* loss_dev, void* stream) {
  if (!f || !samples_dev) return flow_err(LISA_TD_EINVAL, "NULL argument");
  if (epochs < 1 || !(lr > 0.0f)) return flow_err(LISA_TD_EINVAL, "epochs >= 1 and lr > 0 required");
  if (batch < 1 || batch > f->max_train)
    return report_error(LISA_TD_ERANGE, "batch=%d out of [1, %d]", batch, f->max_train);
  if (S < batch) return flow_err(LISA_TD_EINVAL, "fewer samples than one batch");
  int rc = check_timeout(f);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nb = S / batch;
  if (loss_dev) {
    cudaError_t e = cudaMemsetAsync(loss_dev, 0, sizeof(float) * epochs, s);
    if (e != cudaSuccess) return cuda_err(e, "flow_train");
  }
  static const int64_t kPrimes[] = {1000003, 999983, 1000033, 999979, 1000037, 999961,
                                    1000039, 999959, 1000081, 999953};
  for (int ep = 0; ep < epochs; ++ep) {
    // stateless shuffle: position i -> sample (a i + c) mod S, gcd(a, S) = 1
    int64_t mul = 1;
    for (int q = 0; q < 10; ++q) {
      int64_t cand = kPrimes[(ep + q) % 10] % S, x = cand, y = S;
      while (y) { int64_t t = x % y; x = y; y = t; }
      if (cand > 0 && x == 1) { mul = cand; break; }
    }
    const int64_t add = ((int64_t)ep * 7919) % S;
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t n = (int64_t)batch * 15;
      flow_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(samples_dev, S, b * batch,
                                                                     batch, mul, add, f->batch_ws);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_err(e, "flow_train: gather");
      rc = run_grad(f, f->batch_ws, batch, nullptr, loss_dev ? loss_dev + ep : nullptr,
                    1.0f / (float)nb, f->grad_ws, s);
      if (rc) return rc;
      rc = run_adam(f, f->grad_ws, lr, s);
      if (rc) return rc;
    }
  }
  return LISA_TD_OK;
}

void flow_destroy(flow_ctx* f) { free_flow(f); }

}  // extern "C"
