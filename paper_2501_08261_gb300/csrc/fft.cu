// DFT of the A, E, T residuals and the PSD-weighted norm (Sec. II.B):
//   logL = -1/2 sum_c 4 df sum_{k in band} |dt DFT(h_c - d_c)_k|^2 / S_c(f_k).
//
// Four-step mixed-radix FFT, n = n1 * n2, input index i = n2 * a + b, output
// bin k = k1 + n1 * k2.  Two real series (walkers 2p and 2p+1, adjacent in the
// walker-minor layout) form one complex sequence z = x_2p + i x_2p+1.
//   pass 1: for each b, an n1-point transform over a, times W_n^{b k1}
//   pass 2: for each row pair (k1, n1 - k1), n2-point transforms over b; the
//           two rows hold every bin together with its mirror n - k, so the two
//           walkers separate as X = (Z_k + conj Z_{n-k})/2, Y = (Z_k - conj Z_{n-k})/2i,
//           and the weighted |.|^2 of the band bins (k <= n/2) is summed.
// The n1- and n2-point transforms are Stockham radix-2/3/4/5/7/8 stages in
// shared memory, pairs of walkers along the fast axis, plus at most one stage
// of a prime radix in [11, 127] evaluated as a direct DFT.
#include <math.h>

#include "internal.h"

namespace lisa {

namespace {

template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };

template <typename C>
__device__ inline C cmulv(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

struct Radices { int r[kMaxRadix]; int nr; };

// ---- small forward DFTs (W_R = exp(-2 pi i / R)), in registers ------------
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }   // -i a

template <int R, typename C> struct Dft;

template <typename C> struct Dft<2, C> {
  __device__ __forceinline__ static void run(C* a) {
    C t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};
template <typename C> struct Dft<4, C> {
  __device__ __forceinline__ static void run(C* a) {
    C s0 = cadd(a[0], a[2]), s1 = csub(a[0], a[2]);
    C s2 = cadd(a[1], a[3]), s3 = cmul_mi(csub(a[1], a[3]));
    a[0] = cadd(s0, s2);
    a[2] = csub(s0, s2);
    a[1] = cadd(s1, s3);
    a[3] = csub(s1, s3);
  }
};
template <typename C> struct Dft<8, C> {
  __device__ __forceinline__ static void run(C* a) {
    using T = decltype(a[0].x);
    const T h = (T)0.70710678118654752440;
    C e[4] = {a[0], a[2], a[4], a[6]}, o[4] = {a[1], a[3], a[5], a[7]};
    Dft<4, C>::run(e);
    Dft<4, C>::run(o);
    C w1, w3;                                       // W8 o1, W8^3 o3
    w1.x = h * (o[1].x + o[1].y);  w1.y = h * (o[1].y - o[1].x);
    C w2 = cmul_mi(o[2]);
    w3.x = h * (o[3].y - o[3].x);  w3.y = -h * (o[3].x + o[3].y);
    a[0] = cadd(e[0], o[0]); a[4] = csub(e[0], o[0]);
    a[1] = cadd(e[1], w1);   a[5] = csub(e[1], w1);
    a[2] = cadd(e[2], w2);   a[6] = csub(e[2], w2);
    a[3] = cadd(e[3], w3);   a[7] = csub(e[3], w3);
  }
};
template <typename C> struct Dft<3, C> {
  __device__ __forceinline__ static void run(C* a) {
    using T = decltype(a[0].x);
    const T s3 = (T)0.86602540378443864676;
    C t = cadd(a[1], a[2]), u = csub(a[1], a[2]);
    C m; m.x = a[0].x - (T)0.5 * t.x; m.y = a[0].y - (T)0.5 * t.y;
    a[0] = cadd(a[0], t);
    // -i sqrt3/2 u
    C v; v.x = s3 * u.y; v.y = -s3 * u.x;
    a[1] = cadd(m, v);
    a[2] = csub(m, v);
  }
};
// R = 5, 7: the symmetric form.  With W = exp(-2 pi i / R), pairs q, R - q
// combine as t_q = a_q + a_{R-q}, u_q = a_q - a_{R-q}, and
//   X_s = a_0 + sum_q t_q cos(2 pi q s / R) - i sum_q u_q sin(2 pi q s / R),
//   X_{R-s} = the same with +i,  q, s = 1 .. (R-1)/2.
// The cosines and sines are compile-time constants of the element type (a
// __constant__ FP64 table would cost an FP64 conversion per use on the FP32
// path, and GB300's FP64 pipe runs at 1/64 of FP32).
template <int R, typename C> struct DftSym {
  template <typename T>
  __device__ __forceinline__ static void run(C* a, const T (&cs)[(R - 1) / 2][(R - 1) / 2],
                                             const T (&sn)[(R - 1) / 2][(R - 1) / 2]) {
    constexpr int M = (R - 1) / 2;
    C t[M], u[M];
#pragma unroll
    for (int q = 0; q < M; ++q) {
      t[q] = cadd(a[q + 1], a[R - 1 - q]);
      u[q] = csub(a[q + 1], a[R - 1 - q]);
    }
    C x0 = a[0];
#pragma unroll
    for (int q = 0; q < M; ++q) x0 = cadd(x0, t[q]);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      C b = a[0], d;
      d.x = (T)0;
      d.y = (T)0;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        b.x += cs[s][q] * t[q].x;
        b.y += cs[s][q] * t[q].y;
        d.x += sn[s][q] * u[q].x;
        d.y += sn[s][q] * u[q].y;
      }
      // -i d = (d.y, -d.x)
      a[s + 1].x = b.x + d.y;
      a[s + 1].y = b.y - d.x;
      a[R - 1 - s].x = b.x - d.y;
      a[R - 1 - s].y = b.y + d.x;
    }
    a[0] = x0;
  }
};
template <typename C> struct Dft<5, C> {
  __device__ __forceinline__ static void run(C* a) {
    using T = decltype(a[0].x);
    // cos / sin (2 pi q s / 5), s, q = 1, 2
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
    const T cs[2][2] = {{c1, c2}, {c2, c1}};
    const T sn[2][2] = {{s1, s2}, {s2, -s1}};
    DftSym<5, C>::run(a, cs, sn);
  }
};
template <typename C> struct Dft<7, C> {
  __device__ __forceinline__ static void run(C* a) {
    using T = decltype(a[0].x);
    // cos / sin (2 pi k / 7), k = 1, 2, 3; entries at k = q s mod 7 (sin odd)
    const T c1 = (T)0.62348980185873353053, c2 = (T)-0.22252093395631440429,
            c3 = (T)-0.90096886790241912624;
    const T s1 = (T)0.78183148246802980871, s2 = (T)0.97492791218182360702,
            s3 = (T)0.43388373911755812048;
    const T cs[3][3] = {{c1, c2, c3}, {c2, c3, c1}, {c3, c1, c2}};
    const T sn[3][3] = {{s1, s2, s3}, {s2, -s3, -s1}, {s3, -s1, s2}};
    DftSym<7, C>::run(a, cs, sn);
  }
};

// one Stockham stage of radix RAD: A (natural sub-blocks of length L) -> B;
// tw is the m-point table W_m^j in shared memory.  P = 2^lgP columns; j / L
// by the multiply-high with magL = floor((2^32 - 1) / L) + 1, exact for
// j, L < 2^16 (checked by plan_fft), and j itself when L = 1
template <int RAD, typename C>
__device__ void stage(const C* __restrict__ A, C* __restrict__ B, int m, int L, unsigned magL,
                      int lgP, const C* __restrict__ tw, int tid, int nth) {
  const int nb = m / RAD;
  const int stride = m / (L * RAD);
  const int P = 1 << lgP;
  for (int item = tid; item < (nb << lgP); item += nth) {
    const int p = item & (P - 1), j = item >> lgP;
    const int jq = L == 1 ? j : (int)__umulhi((unsigned)j, magL);
    const int k = j - jq * L;
    C a[RAD];
#pragma unroll
    for (int q = 0; q < RAD; ++q) {
      a[q] = A[(j + q * nb) * P + p];
      if (q > 0 && k > 0) a[q] = cmulv(a[q], tw[k * q * stride]);
    }
    Dft<RAD, C>::run(a);
    const int base = (j - k) * RAD + k;
#pragma unroll
    for (int s = 0; s < RAD; ++s) B[(base + s * L) * P + p] = a[s];
  }
}

// one stage of a prime radix R in [11, 127] (at most one per plan), in two
// sweeps over shared memory:
//  1. the stage twiddles in place, y_q = A_q W_m^{q k stride} (k = j mod L);
//  2. the R-point DFT of y by conjugate pairs: with u_q = y_q + y_{R-q},
//     v_q = y_q - y_{R-q} and W_R^{q s} = c + i d for q, s in [1, h], h = (R-1)/2,
//       out_s     = y_0 + sum_q c u_q + i sum_q d v_q,
//       out_{R-s} = y_0 + sum_q c u_q - i sum_q d v_q,
//     and out_0 = y_0 + sum_q u_q (the s = 0 item, where W_R^0 = 1 and d = 0).
// One thread per (column, j, s <= h): R/2 pair loads and 4 FMA per output
// pair and q, with W_R^{q s} = W_m^{q s nb} read from the same table.
template <typename C>
__device__ void stage_prime(C* __restrict__ A, C* __restrict__ B, int m, int R, int L,
                            unsigned magL, int lgP, const C* __restrict__ tw, int tid, int nth) {
  const int nb = m / R;
  const int stride = m / (L * R);
  const int P = 1 << lgP;
  // i / d as umulhi(i, 2^32 / d + 1), exact for i, d < 2^16 and d > 1
  if (L > 1) {                                   // then nb >= L > 1
    const unsigned mag_nb = 0xFFFFFFFFu / (unsigned)nb + 1u;
    for (int item = tid; item < (m << lgP); item += nth) {
      const int p = item & (P - 1), i = item >> lgP;   // i = j + q nb
      const int q = (int)__umulhi((unsigned)i, mag_nb), j = i - q * nb;
      const int k = j - (int)__umulhi((unsigned)j, magL) * L;
      if (q > 0 && k > 0) A[item] = cmulv(A[item], tw[q * k * stride]);
    }
    __syncthreads();
  }
  const int h = (R - 1) / 2;
  const int nsj = h + 1;
  const unsigned mag_s = 0xFFFFFFFFu / (unsigned)nsj + 1u;
  for (int item = tid; item < ((nb * nsj) << lgP); item += nth) {
    const int p = item & (P - 1), js = item >> lgP;
    const int j = (int)__umulhi((unsigned)js, mag_s), s = js - j * nsj;
    const int jq = L == 1 ? j : (int)__umulhi((unsigned)j, magL);
    const int k = j - jq * L;
    const C* col = A + (size_t)j * P + p;
    C U, V;
    U.x = 0;
    U.y = 0;
    V.x = 0;
    V.y = 0;
    const int e = s * nb;                        // W_R^{q s} = tw[q e mod m]
    int idx = 0;
    for (int q = 1; q <= h; ++q) {
      const C a = col[(size_t)q * nb * P];
      const C b = col[(size_t)(R - q) * nb * P];
      idx += e;
      if (idx >= m) idx -= m;
      const C w = tw[idx];
      U.x += w.x * (a.x + b.x);
      U.y += w.x * (a.y + b.y);
      V.x += w.y * (a.x - b.x);
      V.y += w.y * (a.y - b.y);
    }
    const int base = (j - k) * R + k;
    const C y0 = col[0];
    C o;
    o.x = y0.x + U.x - V.y;
    o.y = y0.y + U.y + V.x;
    B[(size_t)(base + s * L) * P + p] = o;
    if (s > 0) {
      o.x = y0.x + U.x + V.y;
      o.y = y0.y + U.y - V.x;
      B[(size_t)(base + (R - s) * L) * P + p] = o;
    }
  }
}

// full m-point transform of 2^lgP columns; returns the buffer holding the result
template <typename C>
__device__ C* transform(C* buf0, C* buf1, int m, int lgP, const Radices& rd,
                        const C* __restrict__ tw) {
  C* A = buf0;
  C* B = buf1;
  int L = 1;
  for (int s = 0; s < rd.nr; ++s) {
    const int r = rd.r[s];
    const unsigned mag = L > 1 ? 0xFFFFFFFFu / (unsigned)L + 1u : 0u;
    switch (r) {
      case 2: stage<2>(A, B, m, L, mag, lgP, tw, threadIdx.x, blockDim.x); break;
      case 3: stage<3>(A, B, m, L, mag, lgP, tw, threadIdx.x, blockDim.x); break;
      case 4: stage<4>(A, B, m, L, mag, lgP, tw, threadIdx.x, blockDim.x); break;
      case 5: stage<5>(A, B, m, L, mag, lgP, tw, threadIdx.x, blockDim.x); break;
      case 7: stage<7>(A, B, m, L, mag, lgP, tw, threadIdx.x, blockDim.x); break;
      case 8: stage<8>(A, B, m, L, mag, lgP, tw, threadIdx.x, blockDim.x); break;
      default: stage_prime(A, B, m, r, L, mag, lgP, tw, threadIdx.x, blockDim.x); break;
    }
    __syncthreads();
    C* t = A;
    A = B;
    B = t;
    L *= r;
  }
  return A;
}

constexpr int kU = 8;   // global loads batched per thread in the staging loops

template <typename R>
__global__ void __launch_bounds__(512) pass1_kernel(const R* __restrict__ x,
                                                    typename CT<R>::T* __restrict__ fy, int64_t n,
                                                    int n1, int n2, int Pt, int lgPb, Radices rd,
                                                    const typename CT<R>::T* __restrict__ tw1,
                                                    const typename CT<R>::T* __restrict__ twn,
                                                    const int* __restrict__ chans,
                                                    int64_t cstride, int ldc) {
  using C = typename CT<R>::T;
  const int Pb = 1 << lgPb;
  extern __shared__ unsigned char smem_raw[];
  C* b0 = reinterpret_cast<C*>(smem_raw);
  C* b1 = b0 + (size_t)n1 * Pb;
  C* tws = b1 + (size_t)n1 * Pb;                   // W_n1^j, j < n1
  for (int j = threadIdx.x; j < n1; j += blockDim.x) tws[j] = tw1[j];
  const int b = blockIdx.x;
  const int pb0 = blockIdx.y * Pb;
  const int c = chans[blockIdx.z];
  // input rows of ldc complex values (walker pairs), channels cstride reals apart
  const C* xc = reinterpret_cast<const C*>(x + (int64_t)c * cstride);
  // staging: kU independent loads in flight per thread before the stores
  const int total = n1 * Pb;
  for (int base = threadIdx.x; base < total; base += blockDim.x * kU) {
    C v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int item = base + u * blockDim.x;
      if (item < total) {
        const int a = item >> lgPb, p = item & (Pb - 1);
        v[u] = xc[((int64_t)n2 * a + b) * ldc + pb0 + p];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int item = base + u * blockDim.x;
      if (item < total) b0[item] = v[u];
    }
  }
  __syncthreads();
  C* res = transform(b0, b1, n1, lgPb, rd, (const C*)tws);
  C* out = fy + (int64_t)c * n * Pt;
  for (int base = threadIdx.x; base < total; base += blockDim.x * kU) {
    C t[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int item = base + u * blockDim.x;
      if (item < total) t[u] = twn[(int64_t)b * (item >> lgPb)];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int item = base + u * blockDim.x;
      if (item < total) {
        const int k1 = item >> lgPb, p = item & (Pb - 1);
        out[((int64_t)k1 * n2 + b) * Pt + pb0 + p] = cmulv(res[item], t[u]);
      }
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(512) pass2_kernel(const typename CT<R>::T* __restrict__ fy,
                                                    double* __restrict__ partial, int64_t n,
                                                    int n1, int n2, int Pt, int lgPb, Radices rd,
                                                    const typename CT<R>::T* __restrict__ tw2,
                                                    const double* __restrict__ psdw,
                                                    const int* __restrict__ chans,
                                                    int klo, int khi) {
  using C = typename CT<R>::T;
  const int Pb = 1 << lgPb;
  extern __shared__ unsigned char smem_raw[];
  // rows rA and rB side by side: columns [0, Pb) of row rA, [Pb, 2 Pb) of row
  // rB, transformed together (one set of radix stages for both)
  const int P2 = 2 * Pb;
  C* u0 = reinterpret_cast<C*>(smem_raw);          // [n2][2 Pb]
  C* u1 = u0 + (size_t)n2 * P2;
  C* tws = u1 + (size_t)n2 * P2;                   // W_n2^j, j < n2
  for (int j = threadIdx.x; j < n2; j += blockDim.x) tws[j] = tw2[j];
  __shared__ double red[512];
  const int rp = blockIdx.x;
  const int pb0 = blockIdx.y * Pb;
  const int c = chans[blockIdx.z];
  const int rA = rp, rB = (n1 - rp) % n1;
  const bool single = (rA == rB);
  const C* in = fy + (int64_t)c * n * Pt;
  const int total = n2 * Pb;
  for (int base = threadIdx.x; base < total; base += blockDim.x * kU) {
    C va[kU], vc[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int item = base + u * blockDim.x;
      if (item < total) {
        const int j = item >> lgPb, p = item & (Pb - 1);
        va[u] = in[((int64_t)rA * n2 + j) * Pt + pb0 + p];
        vc[u] = in[((int64_t)rB * n2 + j) * Pt + pb0 + p];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int item = base + u * blockDim.x;
      if (item < total) {
        const int j = item >> lgPb, p = item & (Pb - 1);
        u0[j * P2 + p] = va[u];
        u0[j * P2 + Pb + p] = vc[u];
      }
    }
  }
  __syncthreads();
  const C* X = transform(u0, u1, n2, lgPb + 1, rd, (const C*)tws);
  const int nb = (int)(n / 2 + 1);               // n <= 2^24: bin indices fit int
  const double* wv = psdw + (c == 2 ? nb : 0);
  // FP32 path: the same weights as float x 2^-160, stored after the FP64 ones
  const float* wv32 = reinterpret_cast<const float*>(psdw + 2 * (int64_t)nb) + (c == 2 ? nb : 0);
  // walker 2p, 2p+1 (p fixed per thread).  FP64 transforms accumulate in FP64.
  // FP32 transforms accumulate in FP32 with exact power-of-two scalings: the
  // weights 4 df dt^2 / S reach 1e47 (x 2^-160: <= 1) and the spectra of
  // small residuals 1e-20 (x 2^64), so every product stays in FP32's normal
  // range; the per-thread sums are undone by 2^(160 - 128) in FP64 below
  double accx = 0.0, accy = 0.0;
  float faccx = 0.0f, faccy = 0.0f;
  const int nrow = single ? 1 : 2;
  for (int item = threadIdx.x; item < n2 * Pb; item += blockDim.x) {
    const int k2 = item >> lgPb, p = item & (Pb - 1);
    for (int rr = 0; rr < nrow; ++rr) {
      const int co = rr == 0 ? 0 : Pb;             // this row's columns
      const int cm = single ? 0 : Pb - co;         // its mirror row's columns
      const int row = rr == 0 ? rA : rB;
      const int k = row + n1 * k2;
      if (k >= nb || k < klo || k > khi) continue;   // outside a safe superset of the band
      const int km = (single && row == 0) ? (k2 == 0 ? 0 : n2 - k2) : n2 - 1 - k2;
      if constexpr (sizeof(R) == 4) {
        const float ws = wv32[k];
        if (ws == 0.0f) continue;
        const C z = X[k2 * P2 + co + p];
        const C zm = X[km * P2 + cm + p];
        const float zx = z.x * 0x1p64f, zy = z.y * 0x1p64f;
        const float mx = zm.x * 0x1p64f, my = zm.y * 0x1p64f;
        const float xr = 0.5f * (zx + mx), xi = 0.5f * (zy - my);
        const float yr = 0.5f * (zy + my), yi = -0.5f * (zx - mx);
        faccx = fmaf(ws, fmaf(xr, xr, xi * xi), faccx);
        faccy = fmaf(ws, fmaf(yr, yr, yi * yi), faccy);
      } else {
        const double wk = wv[k];
        if (wk == 0.0) continue;
        const C z = X[k2 * P2 + co + p];
        const C zm = X[km * P2 + cm + p];
        const double xr = 0.5 * ((double)z.x + (double)zm.x), xi = 0.5 * ((double)z.y - (double)zm.y);
        const double yr = 0.5 * ((double)z.y + (double)zm.y), yi = -0.5 * ((double)z.x - (double)zm.x);
        accx += wk * (xr * xr + xi * xi);
        accy += wk * (yr * yr + yi * yi);
      }
    }
  }
  if constexpr (sizeof(R) == 4) {
    accx = (double)faccx * 0x1p32;
    accy = (double)faccy * 0x1p32;
  }
  // per-column reduction in FP64: thread t served column t % Pb (Pb <= 16
  // divides 32); lanes of a warp with the same column combine by shuffles,
  // then the warps' sums add in a fixed order (deterministic)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int half = 0; half < 2; ++half) {
    double v = half == 0 ? accx : accy;
    for (int off = 16; off >= Pb; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane < Pb) red[wid * Pb + lane] = v;
    __syncthreads();
    if (threadIdx.x < Pb) {
      double sum = 0.0;
      for (int q = 0; q < nwarp; ++q) sum += red[q * Pb + threadIdx.x];
      partial[((int64_t)c * (n1 / 2 + 1) + rp) * (2 * Pt) + 2 * (pb0 + threadIdx.x) + half] = sum;
    }
    __syncthreads();
  }
}

// logL per walker from the per-row-pair partials: a block holds 32 walkers
// (lanes, coalesced) x kRedWarps warps; warp q sums the (channel, row pair)
// entries q, q + kRedWarps, ... of its lane's walker, then warp 0 adds the
// warps' sums in order (deterministic).  One thread per walker walking all
// 3 (n1/2 + 1) entries in series was bound by the latency of its L2 loads.
constexpr int kRedWarps = 16;
__global__ void __launch_bounds__(32 * kRedWarps) reduce_kernel(
    const double* __restrict__ partial, int nrp, int Wpad, int W, int mask,
    const WalkerRec* __restrict__ walkers, double* logl, int32_t* status) {
  __shared__ double part[kRedWarps][32];
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int w = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (w < W) {
    for (int c = 0; c < 3; ++c) {
      if (!((mask >> c) & 1)) continue;
      for (int r = q; r < nrp; r += kRedWarps) s += partial[((int64_t)c * nrp + r) * Wpad + w];
    }
  }
  part[q][lane] = s;
  __syncthreads();
  if (q != 0 || w >= W) return;
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < kRedWarps; ++k) t += part[k][lane];
  const int st = walkers[w].status;
  logl[w] = st ? -INFINITY : -0.5 * t;
  if (status) status[w] = st;
}

int pick_pb(int m, int nbuf, size_t csize, int Pt) {
  // pass 1 (two buffers) gathers strided rows: more, smaller blocks hide the
  // latency better (measured by the autotuner); pass 2 keeps wide blocks
  int pb = nbuf == 2 ? 4 : 16;
  auto bytes = [&](int q) { return ((size_t)nbuf * q + 1) * m * csize; };
  while (pb > 1 && (bytes(pb) > 200 * 1024 || Pt % pb != 0)) pb /= 2;
  return bytes(pb) > 200 * 1024 ? 0 : pb;
}

bool pb_fits(int m, int nbuf, size_t csize, int Pt, int pb) {
  return pb >= 1 && Pt % pb == 0 && ((size_t)nbuf * pb + 1) * m * csize <= 200 * 1024;
}

void radices_of(int m, Radices* rd) {
  rd->nr = 0;
  while (m % 8 == 0) { rd->r[rd->nr++] = 8; m /= 8; }
  while (m % 4 == 0) { rd->r[rd->nr++] = 4; m /= 4; }
  while (m % 2 == 0) { rd->r[rd->nr++] = 2; m /= 2; }
  while (m % 3 == 0) { rd->r[rd->nr++] = 3; m /= 3; }
  while (m % 5 == 0) { rd->r[rd->nr++] = 5; m /= 5; }
  while (m % 7 == 0) { rd->r[rd->nr++] = 7; m /= 7; }
  if (m > 1) rd->r[rd->nr++] = m;                  // the one prime factor in [11, 127]
}

template <typename R>
cudaError_t launch_t(const lisa_td_ctx* c, int Wpad, const void* r, int pass, cudaStream_t s) {
  using C = typename CT<R>::T;
  const FftPlan& p = c->plan;
  const int Pt = Wpad / 2;
  int chans_h[3], nch = 0;
  for (int q = 0; q < 3; ++q)
    if ((c->cfg.channel_mask >> q) & 1) chans_h[nch++] = q;
  Radices r1, r2;
  r1.nr = p.nr1;
  r2.nr = p.nr2;
  for (int q = 0; q < p.nr1; ++q) r1.r[q] = p.r1[q];
  for (int q = 0; q < p.nr2; ++q) r2.r[q] = p.r2[q];
  int pb1 = pick_pb(p.n1, 2, sizeof(C), Pt);
  int pb2 = pick_pb(p.n2, 4, sizeof(C), Pt);
  if (c->tune_pb1 > 0 && pb_fits(p.n1, 2, sizeof(C), Pt, c->tune_pb1)) pb1 = c->tune_pb1;
  if (c->tune_pb2 > 0 && pb_fits(p.n2, 4, sizeof(C), Pt, c->tune_pb2)) pb2 = c->tune_pb2;
  const int bs1 = c->tune_bs1 == 256 ? 256 : 512;   // threads per block (a multiple of pb)
  const int bs2 = c->tune_bs2 == 256 ? 256 : 512;
  if (pb1 == 0 || pb2 == 0) return cudaErrorInvalidValue;
  int lg1 = 0, lg2 = 0;
  while ((1 << lg1) < pb1) ++lg1;
  while ((1 << lg2) < pb2) ++lg2;
  if ((1 << lg1) != pb1 || (1 << lg2) != pb2) return cudaErrorInvalidValue;
  size_t sm1 = ((size_t)2 * pb1 + 1) * p.n1 * sizeof(C);
  size_t sm2 = ((size_t)4 * pb2 + 1) * p.n2 * sizeof(C);
  cudaFuncSetAttribute(pass1_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
  cudaFuncSetAttribute(pass2_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  const int* chans = c->chan_list;
  if (pass == 1) {
    dim3 g1((unsigned)p.n2, (unsigned)(Pt / pb1), (unsigned)nch);
    // the input block: the whole [3][n][Wpad] buffer, or one length class's
    // rows and columns inside a larger residual buffer (ragged batches)
    const R* x = (const R*)r;
    int64_t cstride = c->n * (int64_t)Wpad;
    int ldc = Pt;
    if (c->fft_ldr > 0) {
      x += c->fft_roff * (int64_t)c->fft_ldr + c->fft_col0;
      cstride = c->fft_cstride;
      ldc = c->fft_ldr / 2;
    }
    pass1_kernel<R><<<g1, bs1, sm1, s>>>(x, (C*)c->fy, c->n, p.n1, p.n2, Pt, lg1, r1,
                                         (const C*)p.tw1, (const C*)p.tw_n, chans, cstride, ldc);
  } else {
    dim3 g2((unsigned)(p.n1 / 2 + 1), (unsigned)(Pt / pb2), (unsigned)nch);
    // bins outside [klo, khi] have zero weight: a superset of the band by one
    // bin on each side (the weights themselves still decide inside it)
    const double df = 1.0 / ((double)c->n * c->cfg.dt);
    double flo = floor(c->cfg.f_lo / df) - 1.0, fhi = ceil(c->cfg.f_hi / df) + 1.0;
    const int klo = flo < 0.0 ? 0 : (int)flo;
    const int khi = fhi > (double)c->n ? (int)c->n : (int)fhi;
    pass2_kernel<R><<<g2, bs2, sm2, s>>>((const C*)c->fy, c->partial, c->n, p.n1, p.n2, Pt,
                                         lg2, r2, (const C*)p.tw2, c->psdw, chans, klo, khi);
  }
  return cudaGetLastError();
}

}  // namespace

int plan_fft(int64_t n, FftPlan* p) {
  int64_t m = n;
  for (int f : {2, 3, 5, 7})
    while (m % f == 0) m /= f;
  // besides 2, 3, 5, 7 at most one prime factor, in [11, 127] (the 61-day
  // window at 5 s is 2^7 3^3 5 61)
  bool prime = m >= 11 && m <= 127;
  for (int64_t d = 2; prime && d * d <= m; ++d)
    if (m % d == 0) prime = false;
  if ((m != 1 && !prime) || n < 4) return -1;
  int64_t best = 1;
  for (int64_t d = 1; d * d <= n; ++d)
    if (n % d == 0) best = d;
  if (n / best >= (1 << 16)) return -1;   // the stage index arithmetic needs m < 2^16
  p->n1 = (int)best;
  p->n2 = (int)(n / best);
  Radices a, b;
  radices_of(p->n1, &a);
  radices_of(p->n2, &b);
  p->nr1 = a.nr;
  p->nr2 = b.nr;
  for (int q = 0; q < a.nr; ++q) p->r1[q] = a.r[q];
  for (int q = 0; q < b.nr; ++q) p->r2[q] = b.r[q];
  return 0;
}

bool fft_pb_valid(const lisa_td_ctx* c, int Wpad, int pass, int pb) {
  const size_t cs = 2 * (size_t)c->esize;
  return pass == 1 ? pb_fits(c->plan.n1, 2, cs, Wpad / 2, pb)
                   : pb_fits(c->plan.n2, 4, cs, Wpad / 2, pb);
}

cudaError_t launch_fft_pass1(const lisa_td_ctx* c, int Wpad, const void* r, cudaStream_t s) {
  return c->cfg.precision == 0 ? launch_t<double>(c, Wpad, r, 1, s)
                               : launch_t<float>(c, Wpad, r, 1, s);
}

cudaError_t launch_fft_pass2(const lisa_td_ctx* c, int Wpad, cudaStream_t s) {
  return c->cfg.precision == 0 ? launch_t<double>(c, Wpad, nullptr, 2, s)
                               : launch_t<float>(c, Wpad, nullptr, 2, s);
}

cudaError_t launch_reduce(const lisa_td_ctx* c, int W, int Wpad, double* logl, int32_t* status,
                          cudaStream_t s) {
  reduce_kernel<<<(W + 31) / 32, 32 * kRedWarps, 0, s>>>(c->partial, c->plan.n1 / 2 + 1, Wpad, W,
                                                        c->cfg.channel_mask, c->walkers, logl,
                                                        status);
  return cudaGetLastError();
}

}  // namespace lisa
