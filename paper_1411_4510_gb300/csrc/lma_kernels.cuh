// Device kernels of the LMA hot path (templated on the working precision T:
// float for the mixed form, double for the plain FP64 form and the global
// summary).  Every kernel works on 64x64 tiles with 256 threads.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lma_types.cuh"

namespace lma {

template <typename T> __device__ __forceinline__ T dexp(T x);
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }

template <typename T> struct GemmSmem {
  T a[KS][TB + 4];
  T b[KS][TB + 4];
};

// acc[i][j] += sum_k A(r,k) B(c,k) for tile row r = ty + 16 i, tile column
// c = tx + 16 j.  fa/fb return one operand element; AK/BK select which index
// neighbouring threads walk while staging (true: k, for operands whose k is
// contiguous in memory; false: r).
template <typename T, bool AK, bool BK, class FA, class FB>
__device__ __forceinline__ void tile_mma(T (&acc)[4][4], int K, GemmSmem<T>& sm, FA fa, FB fb) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += KS) {
#pragma unroll
    for (int e = tid; e < TB * KS; e += NT) {
      int r = AK ? e / KS : e % TB;
      int kk = AK ? e % KS : e / TB;
      int k = k0 + kk;
      sm.a[kk][r] = (k < K) ? fa(r, k) : T(0);
    }
#pragma unroll
    for (int e = tid; e < TB * KS; e += NT) {
      int r = BK ? e / KS : e % TB;
      int kk = BK ? e % KS : e / TB;
      int k = k0 + kk;
      sm.b[kk][r] = (k < K) ? fb(r, k) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = sm.a[kk][ty + 16 * i];
        b[i] = sm.b[kk][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

// Error-free sum: hi + lo == a + b exactly (Knuth's TwoSum).
template <typename T>
__device__ __forceinline__ void two_sum(T& hi, T& lo, T b) {
  T s = hi + b;
  T bp = s - hi;
  T e = (hi - (s - bp)) + (b - bp);
  hi = s;
  lo += e;
}

// Same product as tile_mma, with the K sum split into chunks of KS terms:
// each chunk is accumulated in T and added into (hi, lo) with TwoSum, so the
// accumulation error is that of a KS-term sum rather than a K-term one.
template <typename T, bool AK, bool BK, class FA, class FB>
__device__ __forceinline__ void tile_mma_comp(T (&hi)[4][4], T (&lo)[4][4], int K, GemmSmem<T>& sm, FA fa, FB fb) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += KS) {
#pragma unroll
    for (int e = tid; e < TB * KS; e += NT) {
      int r = AK ? e / KS : e % TB;
      int kk = AK ? e % KS : e / TB;
      int k = k0 + kk;
      sm.a[kk][r] = (k < K) ? fa(r, k) : T(0);
    }
#pragma unroll
    for (int e = tid; e < TB * KS; e += NT) {
      int r = BK ? e / KS : e % TB;
      int kk = BK ? e % KS : e / TB;
      int k = k0 + kk;
      sm.b[kk][r] = (k < K) ? fb(r, k) : T(0);
    }
    __syncthreads();
    T c[4][4] = {};
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = sm.a[kk][ty + 16 * i];
        b[i] = sm.b[kk][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[i][j] = fma(a[i], b[j], c[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) two_sum(hi[i][j], lo[i][j], c[i][j]);
    __syncthreads();
  }
}

__device__ __forceinline__ void tri_index(int t, int& I, int& J) {
  int i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  I = i;
  J = t - i * (i + 1) / 2;
}

// ---------------------------------------------------------------------------
// Scaled coordinates: xs = x / l (SE-ARD, Section 5), in FP64 and in T.
template <typename T>
__global__ void k_scale(const double* __restrict__ X, int64_t n, int d, const double* __restrict__ inv_ell,
                        double* __restrict__ xs64, T* __restrict__ xsT) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * d) return;
  double v = X[i] * inv_ell[i % d];
  if (xs64) xs64[i] = v;
  if (xsT) xsT[i] = (T)v;
}

// r = y - mu in T and FP64
template <typename T>
__global__ void k_center(const double* __restrict__ y, int64_t n, double mu, T* __restrict__ rT) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) rT[i] = (T)(y[i] - mu);
}

// Sigma_SS + jitter I into a factorisation buffer with s extra identity rows
// (the sweep then yields L_SS and L_SS^-T).  One thread per element.
__global__ void k_build_kss(const double* __restrict__ ss, int s, int d, double ss2, double jitter,
                            int npad, double* __restrict__ buf) {
  int64_t total = (int64_t)(npad + s) * npad;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  int i = (int)(e / npad), j = (int)(e % npad);
  double v;
  if (i < npad) {
    if (i < s && j < s) {
      double d2 = 0.0;
      for (int q = 0; q < d; ++q) {
        double t = ss[i * d + q] - ss[j * d + q];
        d2 += t * t;
      }
      v = ss2 * exp(-0.5 * d2) + (i == j ? jitter : 0.0);
    } else {
      v = (i == j) ? 1.0 : 0.0;
    }
  } else {
    v = ((i - npad) == j) ? 1.0 : 0.0;
  }
  buf[e] = v;
}

// Covariance between points and the support set: K[p][k] = ss2 exp(-|xs_p - ss_k|^2 / 2)
template <typename T>
__global__ void __launch_bounds__(NT) k_kds(const T* __restrict__ xs, int64_t n, int d, const T* __restrict__ ss,
                                            int s, T ss2, T* __restrict__ out) {
  __shared__ T xp[TB][MAXD + 1];
  __shared__ T xk[TB][MAXD + 1];
  const int64_t p0 = (int64_t)blockIdx.y * TB;
  const int k0 = blockIdx.x * TB;
  for (int e = threadIdx.x; e < TB * d; e += NT) {
    int r = e / d, q = e % d;
    xp[r][q] = (p0 + r < n) ? xs[(p0 + r) * d + q] : T(0);
    xk[r][q] = (k0 + r < s) ? ss[(int64_t)(k0 + r) * d + q] : T(0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TB * TB; e += NT) {
    int r = e / TB, c = e % TB;
    if (p0 + r < n && k0 + c < s) {
      T d2 = 0;
      for (int q = 0; q < d; ++q) {
        T t = xp[r][q] - xk[c][q];
        d2 = fma(t, t, d2);
      }
      out[(p0 + r) * s + k0 + c] = ss2 * dexp<T>(T(-0.5) * d2);
    }
  }
}

// Vt[p][i] = sum_{k <= i} Kds[p][k] ET[k][i] with ET[k][i] = (L_SS^-1)[i][k]:
// the whitened support coordinates V = L_SS^-1 Sigma_SD, stored point-major.
template <typename T>
__global__ void __launch_bounds__(NT) k_proj(const T* __restrict__ Kds, int64_t n, int s, const T* __restrict__ ET,
                                             T* __restrict__ Vt, int ldo) {
  __shared__ GemmSmem<T> sm;
  const int64_t p0 = (int64_t)blockIdx.y * TB;
  const int i0 = blockIdx.x * TB;
  int K = i0 + TB;
  if (K > s) K = s;
  T acc[4][4] = {};
  auto fa = [&](int r, int k) -> T { return (p0 + r < n) ? Kds[(p0 + r) * s + k] : T(0); };
  auto fb = [&](int r, int k) -> T { return (i0 + r < s) ? ET[(int64_t)k * s + i0 + r] : T(0); };
  tile_mma<T, true, false>(acc, K, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t p = p0 + ty + 16 * i;
      int c = i0 + tx + 16 * j;
      if (p < n && c < s) Vt[p * ldo + c] = acc[i][j];
    }
}

// The same product with 128 x 128 tiles and an 8 x 8 register block per
// thread (FP32 FMA in the same k order as k_proj, so the same rounding):
// Vt[p][i] = sum_{k <= i} Kds[p][k] ET[k][i].  Needs s % 4 == 0 (float4 rows).
__global__ void __launch_bounds__(256) k_proj128(const float* __restrict__ Kds, int64_t n, int s,
                                                 const float* __restrict__ ET, float* __restrict__ Vt, int ldo) {
  constexpr int BM = 128, BK = 8;
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BM + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t p0 = (int64_t)blockIdx.y * BM;
  const int i0 = blockIdx.x * BM;
  const int K = min(s, i0 + BM);  // ET[k][i] = 0 for k > i
  // loader mapping: A: row ar = tid / 2 (128 rows), k offset 4 (tid & 1); B: row br = tid / 32 (8 rows), cols 4 (tid & 31)
  const int ar = tid >> 1, ak = (tid & 1) * 4;
  const int br = tid >> 5, bc = (tid & 31) * 4;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  auto ldA = [&](int k0) -> float4 {
    const int64_t p = p0 + ar;
    const int k = k0 + ak;
    if (p >= n || k >= K) return make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v = *reinterpret_cast<const float4*>(Kds + p * s + k);
    if (k + 4 > K) {
      v.y = (k + 1 < K) ? v.y : 0.f;
      v.z = (k + 2 < K) ? v.z : 0.f;
      v.w = 0.f;
    }
    return v;
  };
  auto ldB = [&](int k0) -> float4 {
    const int k = k0 + br, i = i0 + bc;
    if (k >= K || i >= s) return make_float4(0.f, 0.f, 0.f, 0.f);
    return *reinterpret_cast<const float4*>(ET + (int64_t)k * s + i);  // s % 4 == 0: whole float4 in range
  };
  auto stash = [&](int buf, float4 a, float4 b) {
    As[buf][ak + 0][ar] = a.x;
    As[buf][ak + 1][ar] = a.y;
    As[buf][ak + 2][ar] = a.z;
    As[buf][ak + 3][ar] = a.w;
    *reinterpret_cast<float4*>(&Bs[buf][br][bc]) = b;
  };
  float4 a = ldA(0), b = ldB(0);
  stash(0, a, b);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) {
      a = ldA(k0 + BK);
      b = ldB(k0 + BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float ra[8], rb[8];
      *reinterpret_cast<float4*>(ra) = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
      *reinterpret_cast<float4*>(ra + 4) = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
      *reinterpret_cast<float4*>(rb) = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 8]);
      *reinterpret_cast<float4*>(rb + 4) = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 8 + 4]);
#pragma unroll
      for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(ra[x], rb[y], acc[x][y]);
    }
    if (more) {
      stash(buf ^ 1, a, b);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int x = 0; x < 8; ++x) {
    const int64_t p = p0 + ty * 8 + x;
    if (p >= n) continue;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const int i = i0 + tx * 8 + y;
      if (i < s) Vt[p * ldo + i] = acc[x][y];
    }
  }
}

// Residual over a window (Section 3): R = Sigma - Q with
// Sigma = K + sigma_n^2 I and Q = Vt Vt^T, written blanket-first into the
// window buffer (lower 64x64 tiles; padding rows/columns = identity).
template <typename T>
__global__ void __launch_bounds__(NT) k_resid(const Win* __restrict__ wins, const T* __restrict__ xs, int d,
                                              const T* __restrict__ Vt, int s, T ss2, T sn2, T* __restrict__ buf) {
  const Win w = wins[blockIdx.y];
  const int nt = w.npad / TB;
  if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
  int I, J;
  tri_index(blockIdx.x, I, J);
  __shared__ GemmSmem<T> sm;
  __shared__ T xr[TB][MAXD + 1];
  __shared__ T xc[TB][MAXD + 1];
  const int r0 = I * TB, c0 = J * TB;
  for (int e = threadIdx.x; e < TB * d; e += NT) {
    int r = e / d, q = e % d;
    xr[r][q] = (r0 + r < w.n) ? xs[(w.g_end - 1 - (r0 + r)) * d + q] : T(0);
    xc[r][q] = (c0 + r < w.n) ? xs[(w.g_end - 1 - (c0 + r)) * d + q] : T(0);
  }
  T acc[4][4] = {}, lo[4][4] = {};
  auto fa = [&](int r, int k) -> T { int i = r0 + r; return i < w.n ? Vt[(w.g_end - 1 - i) * s + k] : T(0); };
  auto fb = [&](int r, int k) -> T { int i = c0 + r; return i < w.n ? Vt[(w.g_end - 1 - i) * s + k] : T(0); };
  // R = K - Q cancels O(sigma_s^2) terms down to O(sigma_n^2): the Q sum is
  // accumulated with compensation in the reduced precision.
  if (sizeof(T) == 4) tile_mma_comp<T, true, true>(acc, lo, s, sm, fa, fb);
  else tile_mma<T, true, true>(acc, s, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T* A = buf + w.base;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = ty + 16 * i, c = tx + 16 * j;
      int gi = r0 + r, gj = c0 + c;
      T v;
      if (gi < w.n && gj < w.n) {
        T d2 = 0;
        for (int q = 0; q < d; ++q) {
          T t = xr[r][q] - xc[c][q];
          d2 = fma(t, t, d2);
        }
        v = (ss2 * dexp<T>(T(-0.5) * d2) - acc[i][j]) - lo[i][j];
        if (gi == gj) v += sn2;
      } else {
        v = (gi == gj) ? T(1) : T(0);
      }
      A[(int64_t)gi * w.npad + gj] = v;
    }
}

// dst |= src (one device status word into another).
__global__ void k_or_flag(const int* __restrict__ src, int* __restrict__ dst) {
  if (threadIdx.x == 0 && *src) atomicOr(dst, *src);
}

// Residual entries shared between windows.  A pair of training points (p, q),
// p <= q (global order), lies in every window that holds both; in the window
// of p's block, p is a point of the window's own block, and the residual
// kernel always computes the pair's tile there.  Rows [0, nB) of window k
// (its blanket, blocks m+1 .. m+B in reversed order) hold only such pairs
// with p in a later block, so the residual kernel skips window k's 128 x 128
// tiles inside [0, L)^2 (L[k] = nB rounded down to 128; 0 when a blanket
// block has no window in this fit) and this kernel copies their lower
// triangle from the window of each row point's block (local row i of window
// k is local row i + off of window k', off = g_end(k') - g_end(k)), writing
// zeros above the diagonal.  Grid: x = row, y = window.
template <typename T>
__global__ void k_copy_shared_tiles(const Win* __restrict__ wins, int nwin, int B, const int* __restrict__ Ls,
                                    T* __restrict__ buf) {
  const int k = blockIdx.y;
  const int L = Ls[k];
  const int i = blockIdx.x;
  if (i >= L) return;
  const Win w = wins[k];
  const int64_t p = w.g_end - 1 - i;
  int src = -1;
  for (int kk = k + 1; kk <= k + B && kk < nwin; ++kk) {
    const Win v = wins[kk];
    if (p >= v.g_end - v.n && p < v.g_end - v.nB) {
      src = kk;
      break;
    }
  }
  if (src < 0) return;  // not reached: the host sets L = 0 unless every blanket block has a window
  const Win v = wins[src];
  const int64_t off = v.g_end - w.g_end;
  const int jmax = (i / 128 + 1) * 128;
  const T* sp = buf + v.base + (i + off) * (int64_t)v.npad + off;
  T* dst = buf + w.base + (int64_t)i * w.npad;
  for (int j = threadIdx.x; j < jmax; j += blockDim.x) dst[j] = j <= i ? sp[j] : T(0);
}

// Extra rows Y^T of a window: row 0 = r (y - mu), row 1+k = V[k][.] over the
// window's points (blanket-first order); padding columns are 0.
template <typename T>
__global__ void __launch_bounds__(NT) k_fill_ext(const Win* __restrict__ wins, const T* __restrict__ Vt,
                                                 const T* __restrict__ r, int s, T* __restrict__ buf) {
  const Win w = wins[blockIdx.z];
  const int c0 = blockIdx.x * TB;
  const int e0 = blockIdx.y * TB;
  if (c0 >= w.npad || e0 >= s + 1) return;
  __shared__ T tile[TB][TB + 1];
  for (int q = threadIdx.x; q < TB * TB; q += NT) {
    int ci = q / TB, ee = q % TB;
    int i = c0 + ci, e = e0 + ee;
    T v = T(0);
    if (i < w.n && e < s + 1) {
      int64_t g = w.g_end - 1 - i;
      v = (e == 0) ? r[g] : Vt[g * s + (e - 1)];
    }
    tile[ci][ee] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < TB * TB; q += NT) {
    int ee = q / TB, ci = q % TB;
    int e = e0 + ee;
    if (e < s + 1) buf[w.base + (int64_t)(w.npad + e) * w.npad + c0 + ci] = tile[ci][ee];
  }
}

// k_fill_ext for FP32 windows with 16-byte accesses: block (x, y, window z)
// transposes points [64 x, 64 x + 64) (reversed order) x support coordinates
// k in [64 y, 64 y + 64) of V into extra rows 1 + k; y = ceil(s / 64) writes
// row 0 (r).  Loads take four consecutive k of one point (scalar when the
// row length s is not a multiple of 4), stores four consecutive columns.
__global__ void __launch_bounds__(256) k_fill_ext4(const Win* __restrict__ wins, const float* __restrict__ Vt,
                                                   const float* __restrict__ r, int s, float* __restrict__ buf) {
  const Win w = wins[blockIdx.z];
  const int c0 = blockIdx.x * 64;
  if (c0 >= w.npad) return;
  const int ky = (s + 63) / 64;
  float* ext = buf + w.base + (int64_t)w.npad * w.npad;  // extra row e at ext + e * npad
  const int t = threadIdx.x;
  if ((int)blockIdx.y == ky) {  // row 0: r over the window's points
    for (int c = t; c < 64; c += blockDim.x) {
      const int i = c0 + c;
      ext[c0 + c] = i < w.n ? r[w.g_end - 1 - i] : 0.f;
    }
    return;
  }
  const int k0 = blockIdx.y * 64;
  __shared__ float tile[64][65];  // [point][k]
  const bool vec = (s & 3) == 0;
#pragma unroll
  for (int rep = 0; rep < 4; ++rep) {
    const int ci = (t >> 4) + 16 * rep, kq = (t & 15) * 4;
    const int i = c0 + ci, k = k0 + kq;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < w.n) {
      const float* src = Vt + (w.g_end - 1 - i) * (int64_t)s + k;
      if (vec && k + 3 < s) {
        v = *reinterpret_cast<const float4*>(src);
      } else {
        v.x = k < s ? src[0] : 0.f;
        v.y = k + 1 < s ? src[1] : 0.f;
        v.z = k + 2 < s ? src[2] : 0.f;
        v.w = k + 3 < s ? src[3] : 0.f;
      }
    }
    tile[ci][kq] = v.x;
    tile[ci][kq + 1] = v.y;
    tile[ci][kq + 2] = v.z;
    tile[ci][kq + 3] = v.w;
  }
  __syncthreads();
#pragma unroll
  for (int rep = 0; rep < 4; ++rep) {
    const int kk = (t >> 4) + 16 * rep, cq = (t & 15) * 4;
    const int k = k0 + kk;
    if (k < s)
      *reinterpret_cast<float4*>(ext + (int64_t)(1 + k) * w.npad + c0 + cq) =
          make_float4(tile[cq][kk], tile[cq + 1][kk], tile[cq + 2][kk], tile[cq + 3][kk]);
  }
}

// ---------------------------------------------------------------------------
// Left-looking blocked Cholesky sweep, one 64-wide column panel kp per
// launch pair.  k_chol_step: for every row tile i >= kp of every window,
// T_ik = A_ik - A_{i,0:kp} A_{kp,0:kp}^T.  The diagonal tile is factorised in
// shared memory (and its inverse stored); the other tiles keep T_ik until
// k_chol_trsm multiplies them by inv(L_kk)^T.  Extra rows below the matrix
// ride along, so after the last panel they hold (L^-1 Y)^T.
template <typename T>
struct CholSmem {
  GemmSmem<T> g;
  T D[TB][TB + 1];
  T X[TB][TB + 1];
};

// Cholesky of the N x N diagonal tile held in D (shared memory, lower part
// significant) together with the inverse of the factor; L (zeros above the
// diagonal) goes to Lout (leading dim ld), inv(L) to Dv (N x N, row-major).
// Called by all threads of the CTA, which must have at least 4N threads.
//
// Thread t < 4N keeps row t / 4 of the working matrix and of the inverse in
// registers (columns congruent to t mod 4).  Step j: the owners publish
// column j and the (unscaled) inverse row j to shared memory; after one
// barrier every row below j applies the rank-1 update
//   D_rc -= D_rj D_cj / D_jj,   Xt_rc -= D_rj / D_jj  Xt_jc,
// which is the right-looking Cholesky and the right-looking solve of
// L X = I in one sweep (X row j = Xt row j / L_jj).  The reciprocal square
// root of pivot j is taken by the owner of the diagonal as soon as its last
// update lands, overlapping the other rows' updates of the previous step.
// A non-positive or NaN pivot is recorded in *info (first failing column +
// 1, offset k0) and replaced by 1 so the sweep stays finite.
template <typename T, int N = TB>
__device__ void diag_factor(T (*D)[N + 1], T* Lout, int64_t ld, T* Dv, int* info, int k0) {
  constexpr int NQ = N / 4;
  constexpr int VW = 16 / sizeof(T);  // values per 16-byte shared-memory load
  // published column j and inverse row j, stored phase-major: element
  // p + 4 q at [p][q], so a thread reads its NQ values with 16-byte loads
  __shared__ __align__(16) T colb[2][4][NQ];
  __shared__ __align__(16) T xrow[2][4][NQ];
  __shared__ T rjs[2];
  const int t = threadIdx.x, rr = t >> 2, p = t & 3;
  const bool act = t < 4 * N;
  T d[NQ], x[NQ];
  __syncthreads();  // the caller's stores to D are visible
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    d[q] = act ? D[rr][p + 4 * q] : T(0);
    x[q] = (act && p + 4 * q == rr) ? T(1) : T(0);
  }
  __syncthreads();  // D is overwritten with L below
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const int qj = j >> 2, pj = j & 3;
    T(*cb)[NQ] = colb[j & 1];
    T(*xb)[NQ] = xrow[j & 1];
    if (act && rr >= j) {
      if (p == pj) cb[rr & 3][rr >> 2] = d[qj];
      if (rr == j) {
#pragma unroll
        for (int q = 0; q <= qj; ++q)
          if (p + 4 * q <= j) xb[p][q] = x[q];
        if (p == pj) {
          T piv = d[qj];
          if (!(piv > T(0))) {
            if (*info == 0) *info = k0 + j + 1;
            piv = T(1);
          }
          const T r = rsqrt(piv);
          rjs[j & 1] = r;
          D[j][j] = piv * r;
        }
      }
    }
    __syncthreads();
    const T rj = rjs[j & 1];
    if (act && rr == j) {
#pragma unroll
      for (int q = 0; q <= qj; ++q) x[q] *= rj;
    } else if (act && rr > j) {
      const T lr = cb[rr & 3][rr >> 2];
      const T l = lr * rj;
      const T a = l * rj;
      if (p == pj) D[rr][j] = l;
      T cv[NQ], xv[NQ];
#pragma unroll
      for (int q = 0; q < NQ; q += VW) {
        *reinterpret_cast<float4*>(&cv[q]) = *reinterpret_cast<const float4*>(&cb[p][q]);
        *reinterpret_cast<float4*>(&xv[q]) = *reinterpret_cast<const float4*>(&xb[p][q]);
      }
#pragma unroll
      for (int q = qj; q < NQ; ++q) {
        const int cc = p + 4 * q;
        if (cc > j && cc <= rr) d[q] = fma(-a, cv[q], d[q]);
      }
#pragma unroll
      for (int q = 0; q <= qj; ++q) {
        const int c = p + 4 * q;
        if (c <= j) x[q] = fma(-a, xv[q], x[q]);
      }
    }
  }
  __syncthreads();
  for (int q = t; q < N * N; q += blockDim.x) {
    const int r = q / N, c = q % N;
    Lout[(int64_t)r * ld + c] = (c <= r) ? D[r][c] : T(0);
  }
  if (act)
#pragma unroll
    for (int q = 0; q < NQ; ++q) Dv[rr * N + p + 4 * q] = x[q];
}

template <typename T>
__global__ void __launch_bounds__(NT) k_chol_step(const Win* __restrict__ wins, T* __restrict__ buf,
                                                  T* __restrict__ dinv, int* __restrict__ info, int kp) {
  const Win w = wins[blockIdx.y];
  if (kp * TB >= w.npad) return;
  const int i = kp + blockIdx.x;
  const int r0 = i * TB;
  if (r0 >= w.rows) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  CholSmem<T>& sm = *reinterpret_cast<CholSmem<T>*>(smraw);
  T* A = buf + w.base;
  const int64_t ld = w.npad;
  const int k0 = kp * TB;
  T acc[4][4] = {};
  auto fa = [&](int r, int k) -> T { int row = r0 + r; return row < w.rows ? A[row * ld + k] : T(0); };
  auto fb = [&](int r, int k) -> T { return A[(int64_t)(k0 + r) * ld + k]; };
  tile_mma<T, true, true>(acc, k0, sm.g, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (i != kp) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int row = r0 + ty + 16 * a;
        if (row < w.rows) A[row * ld + k0 + tx + 16 * b] -= acc[a][b];
      }
    return;
  }
  // diagonal tile: factorise in shared memory
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int r = ty + 16 * a, c = tx + 16 * b;
      sm.D[r][c] = A[(int64_t)(k0 + r) * ld + k0 + c] - acc[a][b];
    }
  diag_factor<T>(sm.D, A + (int64_t)k0 * ld + k0, ld, dinv + w.dinv + (int64_t)kp * TB * TB, info + blockIdx.y,
                 k0);
}

template <typename T>
struct TrsmSmem {
  T Ts[TB][TB + 1];
  T Xs[TB][TB + 1];
};

// A[i-tile][kp-panel] = T_ik inv(L_kk)^T for row tiles i > kp.
// nid > 0: the first nid appended rows are identity rows (row k has its 1 in
// column k), so an appended-row tile e whose rows all lie below nid is still
// zero at panel kp < e and is skipped.
template <typename T>
__global__ void __launch_bounds__(NT) k_chol_trsm(const Win* __restrict__ wins, T* __restrict__ buf,
                                                  const T* __restrict__ dinv, int kp, int nid) {
  const Win w = wins[blockIdx.y];
  if (kp * TB >= w.npad) return;
  const int i = kp + 1 + blockIdx.x;
  const int r0 = i * TB;
  if (r0 >= w.rows) return;
  {
    const int e = i - w.npad / TB;
    if (e > kp && (e + 1) * TB <= nid) return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  TrsmSmem<T>& sm = *reinterpret_cast<TrsmSmem<T>*>(smraw);
  T* A = buf + w.base;
  const int64_t ld = w.npad;
  const int k0 = kp * TB;
  const T* Dv = dinv + w.dinv + (int64_t)kp * TB * TB;
  for (int q = threadIdx.x; q < TB * TB; q += NT) {
    int r = q / TB, c = q % TB;
    sm.Ts[r][c] = (r0 + r < w.rows) ? A[(int64_t)(r0 + r) * ld + k0 + c] : T(0);
    sm.Xs[r][c] = Dv[q];
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4] = {};
  for (int j = 0; j < TB; ++j) {
    T a[4], b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = sm.Ts[ty + 16 * q][j];
      b[q] = sm.Xs[tx + 16 * q][j];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int row = r0 + ty + 16 * p;
      if (row < w.rows) A[row * ld + k0 + tx + 16 * q] = acc[p][q];
    }
}

// ---------------------------------------------------------------------------
// Local summaries reduced into the global summary (Definition 2), whitened:
// G = sum_m E_m E_m^T with E_m = extra rows [0, s] x block columns [nB, n)
// of window m, i.e. [z_m | Z_m]^T with z_m = L_m^-1 y-dot_m-part and
// Z_m = L_m^-1 V-part.  G[0][0] = quad, G[1+i][0] = y_i, G[1+i][1+j] = A_ij.
// Each CTA accumulates one lower tile over a chunk of windows (T within a
// window, FP64 across windows); k_gram_reduce adds the chunks in order.
template <typename T>
__global__ void __launch_bounds__(NT) k_gram(const Win* __restrict__ wins, int nwin, int chunk, int s,
                                             const T* __restrict__ buf, double* __restrict__ partial) {
  int I, J;
  tri_index(blockIdx.x, I, J);
  const int se = s + 1;
  __shared__ GemmSmem<T> sm;
  const int r0 = I * TB, c0 = J * TB;
  double accd[4][4] = {};
  const int w0 = blockIdx.y * chunk;
  const int w1 = min(nwin, w0 + chunk);
  for (int wi = w0; wi < w1; ++wi) {
    const Win w = wins[wi];
    const T* E = buf + w.base + (int64_t)w.npad * w.npad;
    const int64_t ld = w.npad;
    T acc[4][4] = {};
    auto fa = [&](int r, int k) -> T { int e = r0 + r; return e < se ? E[e * ld + w.nB + k] : T(0); };
    auto fb = [&](int r, int k) -> T { int e = c0 + r; return e < se ? E[e * ld + w.nB + k] : T(0); };
    tile_mma<T, true, true>(acc, w.n - w.nB, sm, fa, fb);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) accd[a][b] += (double)acc[a][b];
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double* P = partial + (int64_t)blockIdx.y * se * se;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int e1 = r0 + ty + 16 * a, e2 = c0 + tx + 16 * b;
      if (e1 < se && e2 < se) P[(int64_t)e1 * se + e2] = accd[a][b];
    }
}

__global__ void k_gram_reduce(const double* __restrict__ partial, int nchunk, int se, double* __restrict__ G,
                              int tile) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)se * se) return;
  int i = (int)(e / se), j = (int)(e % se);
  (void)tile;
  int a = i, b = j;
  if (a < b) { a = j; b = i; }  // the lower triangle is computed; mirror it exactly
  double sum = 0.0;
  for (int c = 0; c < nchunk; ++c) sum += partial[(int64_t)c * se * se + (int64_t)a * se + b];
  G[e] = sum;
}

// log|R-dot_m^-1| per window = 2 sum log diag of the trailing (block) factor
template <typename T>
__global__ void k_logdet(const Win* __restrict__ wins, const T* __restrict__ buf, double* __restrict__ out) {
  const Win w = wins[blockIdx.x];
  __shared__ double red[NT];
  double sum = 0.0;
  for (int i = w.nB + threadIdx.x; i < w.n; i += NT)
    sum += log((double)buf[w.base + (int64_t)i * w.npad + i]);
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = 2.0 * red[0];
}

// ordered sum of n doubles (single thread: deterministic)
__global__ void k_sum_ordered(const double* __restrict__ v, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i];
    *out = s;
  }
}

// Sigma-ddot_SS whitened: C = I + A, with appended rows [I; y] (the sweep
// then yields L_C, L_C^-T and L_C^-1 y; identity rows first so they stay
// 64-aligned for the zero-tile skip).
__global__ void k_build_global(const double* __restrict__ G, int s, int npad, double* __restrict__ buf) {
  const int se = s + 1;
  int64_t total = (int64_t)(npad + 1 + s) * npad;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  int i = (int)(e / npad), j = (int)(e % npad);
  double v;
  if (i < npad) {
    if (i < s && j < s) v = G[(int64_t)(1 + i) * se + 1 + j] + (i == j ? 1.0 : 0.0);
    else v = (i == j) ? 1.0 : 0.0;
  } else if (i < npad + s) {
    v = ((i - npad) == j) ? 1.0 : 0.0;
  } else {
    v = (j < s) ? G[(int64_t)(1 + j) * se] : 0.0;
  }
  buf[e] = v;
}

// beta = L_C^-T w (w = L_C^-1 y, the appended y row of the factor) as a
// matrix-vector product with the explicit L_C^-T rows: one warp per row k,
// coalesced, lane partial sums combined by shuffles (8 rows per CTA).  CTA 0
// also writes scalars[0] = quad, [1] = w^T w, [2] = log|C|.
__global__ void __launch_bounds__(NT) k_global_finish(const double* __restrict__ buf, const double* __restrict__ G,
                                                      int s, int npad, double* __restrict__ beta,
                                                      double* __restrict__ scalars) {
  const double* E = buf + (int64_t)npad * npad;  // row k = (L_C^-T)[k][.]
  const double* w = E + (int64_t)s * npad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * (NT / 32) + warp;
  if (k < s) {
    const double* row = E + (int64_t)k * npad;
    double sum = 0.0;
    for (int i = lane; i < s; i += 32) sum = fma(row[i], w[i], sum);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if (lane == 0) beta[k] = sum;
  }
  if (blockIdx.x != 0) return;
  __shared__ double red[2][NT];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < s; i += NT) {
    a += w[i] * w[i];
    b += log(buf[(int64_t)i * npad + i]);
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scalars[0] = G[0];
    scalars[1] = red[0][0];
    scalars[2] = 2.0 * red[1][0];
  }
}

// Copy an s x s block with leading dimension ld (FP64) into T with ld s.
template <typename T>
__global__ void k_copy_block(const double* __restrict__ src, int64_t ld, int s, T* __restrict__ dst) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)s * s) return;
  int i = (int)(e / s), j = (int)(e % s);
  dst[e] = (T)src[(int64_t)i * ld + j];
}

// Per window: L^-1 e over the window, with e = r - Vt beta (the residual
// after the support-set fit), from the extra rows: X0 - sum_k beta_k X_{1+k}.
template <typename T>
__global__ void k_ew(const Win* __restrict__ wins, const T* __restrict__ buf, const double* __restrict__ beta, int s,
                     T* __restrict__ ew) {
  const Win w = wins[blockIdx.y];
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= w.npad) return;
  const T* E = buf + w.base + (int64_t)w.npad * w.npad;
  double v = (double)E[c];
  for (int k = 0; k < s; ++k) v -= beta[k] * (double)E[(int64_t)(1 + k) * w.npad + c];
  ew[w.ew + c] = (T)v;
}

// The same for FP32 extra rows without FP64 arithmetic (scarce on this part):
// beta_k = bh_k + bl_k as two floats (k_split_beta), each product
// bh_k x = p + e exactly (e from an FMA), bl_k x added to e, and the p are
// summed with TwoSum into (hi, lo), which keeps about 48 bits of the sum.
__global__ void k_split_beta(const double* __restrict__ beta, int s, float2* __restrict__ bs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= s) return;
  const float h = (float)beta[k];
  bs[k] = make_float2(h, (float)(beta[k] - (double)h));
}
__global__ void k_ew_f32(const Win* __restrict__ wins, const float* __restrict__ buf, const float2* __restrict__ bs,
                         int s, float* __restrict__ ew) {
  const Win w = wins[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= w.npad) return;
  const float* E = buf + w.base + (int64_t)w.npad * w.npad;
  float hi = 0.f, lo = 0.f;
  int k = 0;
  for (; k + 8 <= s; k += 8) {  // eight loads in flight ahead of the dependent sums
    float x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = E[(int64_t)(1 + k + q) * w.npad + c];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float2 b = bs[k + q];
      const float p = b.x * x[q];
      const float e = fmaf(b.x, x[q], -p);
      lo += fmaf(b.y, x[q], e);
      two_sum(hi, lo, p);
    }
  }
  for (; k < s; ++k) {
    const float x = E[(int64_t)(1 + k) * w.npad + c];
    const float2 b = bs[k];
    const float p = b.x * x;
    const float e = fmaf(b.x, x, -p);
    lo += fmaf(b.y, x, e);
    two_sum(hi, lo, p);
  }
  ew[w.ew + c] = (float)((double)E[c] - ((double)hi + (double)lo));
}

// ---------------------------------------------------------------------------
// Prediction, local route.  For a test point u of block n and each window m
// in [n-B, n], P_m[u][.] = (L_m^-1 R_{W_m u})^T.  The kept columns (block part
// for m < n, all for m == n) are the rows of the Lemma-1 factor of the
// sub-chain n-B..n+B, so that z_u e_J, z_u R_{D_J u} and Sigma_{S D_J} z_u
// become dot products with the fit's extra rows.

// RHS rows: P[u][i] = K(xu_u, x_g(i)) - Vu[u] . Vt[g(i)]   (tile list items:
// x = pair, y = u tile, z = column tile)
template <typename T>
__global__ void __launch_bounds__(NT) k_pred_rhs(const Pair* __restrict__ pairs, const int4* __restrict__ items,
                                                 const Win* __restrict__ wins, const T* __restrict__ xs,
                                                 const T* __restrict__ xu, int d, const T* __restrict__ Vt,
                                                 const T* __restrict__ Vu, int s, T ss2, T* __restrict__ P) {
  const int4 it = items[blockIdx.x];
  const Pair pr = pairs[it.x];
  const Win w = wins[pr.win];
  const int u0 = it.y * TB, c0 = it.z * TB;
  __shared__ GemmSmem<T> sm;
  __shared__ T xr[TB][MAXD + 1];
  __shared__ T xc[TB][MAXD + 1];
  for (int e = threadIdx.x; e < TB * d; e += NT) {
    int r = e / d, q = e % d;
    xr[r][q] = (u0 + r < pr.nu) ? xu[(int64_t)(pr.u0 + u0 + r) * d + q] : T(0);
    xc[r][q] = (c0 + r < w.n) ? xs[(w.g_end - 1 - (c0 + r)) * d + q] : T(0);
  }
  T acc[4][4] = {}, lo[4][4] = {};
  auto fa = [&](int r, int k) -> T { return (u0 + r < pr.nu) ? Vu[(int64_t)(pr.u0 + u0 + r) * s + k] : T(0); };
  auto fb = [&](int r, int k) -> T { int i = c0 + r; return i < w.n ? Vt[(w.g_end - 1 - i) * s + k] : T(0); };
  if (sizeof(T) == 4) tile_mma_comp<T, true, true>(acc, lo, s, sm, fa, fb);
  else tile_mma<T, true, true>(acc, s, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T* Pp = P + pr.pbase;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int r = ty + 16 * a, c = tx + 16 * b;
      int uu = u0 + r, i = c0 + c;
      if (uu >= pr.nu) continue;
      T v = T(0);
      if (i < w.n) {
        T d2 = 0;
        for (int q = 0; q < d; ++q) {
          T t = xr[r][q] - xc[c][q];
          d2 = fma(t, t, d2);
        }
        v = (ss2 * dexp<T>(T(-0.5) * d2) - acc[a][b]) - lo[a][b];
      }
      Pp[(int64_t)uu * w.npad + i] = v;
    }
}

// Forward solve of P^T by the stored factor, one CTA per (pair, 64 test rows),
// sweeping the window's column panels left to right (items: x = pair, y = u tile).
template <typename T>
__global__ void __launch_bounds__(NT) k_pred_sweep(const Pair* __restrict__ pairs, const int2* __restrict__ items,
                                                   const Win* __restrict__ wins, const T* __restrict__ buf,
                                                   const T* __restrict__ dinv, T* __restrict__ P) {
  const int2 it = items[blockIdx.x];
  const Pair pr = pairs[it.x];
  const Win w = wins[pr.win];
  const int u0 = it.y * TB;
  extern __shared__ __align__(16) unsigned char smraw[];
  CholSmem<T>& sm = *reinterpret_cast<CholSmem<T>*>(smraw);
  const T* L = buf + w.base;
  const int64_t ld = w.npad;
  T* Pp = P + pr.pbase;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int npan = w.npad / TB;
  for (int kp = 0; kp < npan; ++kp) {
    const int k0 = kp * TB;
    T acc[4][4] = {};
    auto fa = [&](int r, int k) -> T { return (u0 + r < pr.nu) ? Pp[(int64_t)(u0 + r) * ld + k] : T(0); };
    auto fb = [&](int r, int k) -> T { return L[(int64_t)(k0 + r) * ld + k]; };
    tile_mma<T, true, true>(acc, k0, sm.g, fa, fb);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int r = ty + 16 * a, c = tx + 16 * b;
        sm.D[r][c] = (u0 + r < pr.nu) ? Pp[(int64_t)(u0 + r) * ld + k0 + c] - acc[a][b] : T(0);
      }
    const T* Dv = dinv + w.dinv + (int64_t)kp * TB * TB;
    for (int q = threadIdx.x; q < TB * TB; q += NT) sm.X[q / TB][q % TB] = Dv[q];
    __syncthreads();
    T o[4][4] = {};
    for (int j = 0; j < TB; ++j) {
      T a4[4], b4[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a4[q] = sm.D[ty + 16 * q][j];
        b4[q] = sm.X[tx + 16 * q][j];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) o[p][q] = fma(a4[p], b4[q], o[p][q]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int r = ty + 16 * a;
        if (u0 + r < pr.nu) Pp[(int64_t)(u0 + r) * ld + k0 + tx + 16 * b] = o[a][b];
      }
    __syncthreads();
  }
}

// h[u][k] = sum over the pairs of block n of P[u][c] X_{1+k}[c] (kept columns)
// minus Vu[u][k]   (items: x = test block's first pair, y = pair count,
// z = u tile, w = s tile)
template <typename T>
__global__ void __launch_bounds__(NT) k_pred_accum(const Pair* __restrict__ pairs, const int4* __restrict__ items,
                                                   const Win* __restrict__ wins, const T* __restrict__ buf,
                                                   const T* __restrict__ P, const T* __restrict__ Vu, int s,
                                                   T* __restrict__ h) {
  const int4 it = items[blockIdx.x];
  const int u0 = it.z * TB, k0 = it.w * TB;
  __shared__ GemmSmem<T> sm;
  T acc[4][4] = {};
  const Pair first = pairs[it.x];
  for (int pi = 0; pi < it.y; ++pi) {
    const Pair pr = pairs[it.x + pi];
    const Win w = wins[pr.win];
    const T* Pp = P + pr.pbase;
    const T* E = buf + w.base + (int64_t)w.npad * w.npad;
    const int64_t ld = w.npad;
    auto fa = [&](int r, int k) -> T { return (u0 + r < pr.nu) ? Pp[(int64_t)(u0 + r) * ld + pr.c0 + k] : T(0); };
    auto fb = [&](int r, int k) -> T { return (k0 + r < s) ? E[(int64_t)(1 + k0 + r) * ld + pr.c0 + k] : T(0); };
    tile_mma<T, true, true>(acc, pr.c1 - pr.c0, sm, fa, fb);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int uu = u0 + ty + 16 * a, k = k0 + tx + 16 * b;
      if (uu < first.nu && k < s) {
        int64_t row = first.u0 + uu;
        h[row * s + k] = acc[a][b] - Vu[row * s + k];
      }
    }
}

// t1[u] = sum_pairs sum_c P[u][c] ew[c];  t2[u] = sum_pairs sum_c P[u][c]^2
// (one warp per test point; items: x = first pair, y = pair count, z = u)
template <typename T>
__global__ void k_pred_t12(const Pair* __restrict__ pairs, const int4* __restrict__ items, int nitems,
                           const Win* __restrict__ wins, const T* __restrict__ P, const T* __restrict__ ew,
                           double* __restrict__ t1, double* __restrict__ t2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nitems) return;
  const int4 it = items[warp];
  double a = 0.0, b = 0.0;
  int64_t row = 0;
  for (int pi = 0; pi < it.y; ++pi) {
    const Pair pr = pairs[it.x + pi];
    const Win w = wins[pr.win];
    const T* Pp = P + pr.pbase + (int64_t)it.z * w.npad;
    row = pr.u0 + it.z;
    for (int c = pr.c0 + lane; c < pr.c1; c += 32) {
      double p = (double)Pp[c];
      a += p * (double)ew[w.ew + c];
      b += p * p;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    t1[row] = a;
    t2[row] = b;
  }
}

// partial[it][u] = sum_{i in tile it} (sum_{k<=i} LcT[k][i] h[u][k])^2
// = contribution of column tile it to |L_C^-1 h_u|^2
template <typename T>
__global__ void __launch_bounds__(NT) k_var_gemm(const T* __restrict__ h, int64_t U, int s, const T* __restrict__ LcT,
                                                 double* __restrict__ partial) {
  __shared__ GemmSmem<T> sm;
  __shared__ double red[TB][17];
  const int64_t u0 = (int64_t)blockIdx.y * TB;
  const int i0 = blockIdx.x * TB;
  int K = min(s, i0 + TB);
  T acc[4][4] = {};
  auto fa = [&](int r, int k) -> T { return (u0 + r < U) ? h[(u0 + r) * s + k] : T(0); };
  auto fb = [&](int r, int k) -> T { return (i0 + r < s) ? LcT[(int64_t)k * s + i0 + r] : T(0); };
  tile_mma<T, true, false>(acc, K, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double v = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double q = (double)acc[a][b];
      if (i0 + tx + 16 * b < s) v += q * q;
    }
    red[ty + 16 * a][tx] = v;
  }
  __syncthreads();
  if (threadIdx.x < TB) {
    double v = 0.0;
    for (int q = 0; q < 16; ++q) v += red[threadIdx.x][q];
    if (u0 + threadIdx.x < U) partial[(int64_t)blockIdx.x * U + u0 + threadIdx.x] = v;
  }
}

// out[u] = |g_u|^2 (FP64 sum) for g = L_C^-1 h formed by k_proj128 (U rows of
// s values): the variance term of k_var_gemm as one partial (ntile = 1).
__global__ void k_row_sqnorm(const float* __restrict__ g, int64_t U, int s, double* __restrict__ out) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= U) return;
  double v = 0.0;
  for (int k = lane; k < s; k += 32) {
    const double q = (double)g[row * s + k];
    v += q * q;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) out[row] = v;
}

// g_u = L_C^-1 h_u for the block covariance: g[u][i] = sum_k h[u][k] LcT[k][i]
template <typename T>
__global__ void __launch_bounds__(NT) k_lc_apply(const T* __restrict__ h, int64_t U, int s, const T* __restrict__ LcT,
                                                 T* __restrict__ g) {
  __shared__ GemmSmem<T> sm;
  const int64_t u0 = (int64_t)blockIdx.y * TB;
  const int i0 = blockIdx.x * TB;
  const int K = min(s, i0 + TB);
  T acc[4][4] = {};
  auto fa = [&](int r, int k) -> T { return (u0 + r < U) ? h[(u0 + r) * s + k] : T(0); };
  auto fb = [&](int r, int k) -> T { return (i0 + r < s) ? LcT[(int64_t)k * s + i0 + r] : T(0); };
  tile_mma<T, true, false>(acc, K, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t u = u0 + ty + 16 * a;
      const int i = i0 + tx + 16 * b;
      if (u < U && i < s) g[u * s + i] = acc[a][b];
    }
}

// Predictive covariance between test blocks n and n2 (Eq. vapvar on
// U_n x U_n2), one 64 x 64 tile of one requested block per CTA
// (items: x = request, y / z = 64-row tiles of U_n / U_n2).  With
// g = L_C^-1 h (the low-rank term of the variance) and, for u in U_n and u'
// in U_n2,
//   Cov(u, u') = g_u . g_u' + [|n - n2| <= B] ( K(u, u') [+ sigma_n^2 delta]
//                - Vu_u . Vu_u' - sum_m P_(n,m)[u] . P_(n2,m)[u'] ),
// the sum over the windows m = max(n, n2) - B .. min(n, n2) on their kept
// columns (block columns for m < min(n, n2), all columns for m = min(n, n2)).
// Off the band the residual part of the covariance vanishes (Eq. ares runs
// through the training blankets only), and in the band windows before
// max(n, n2) - B drop out of the sum (their block rows of
// L_m^-1 R-bar_{W_m u'} are zero); within one block (n = n2) this is the
// local route of the variance.
template <typename T>
__global__ void __launch_bounds__(NT) k_pred_xcov(const Pair* __restrict__ pairs, const CovReq* __restrict__ reqs,
                                                  const int4* __restrict__ items, const Win* __restrict__ wins,
                                                  const T* __restrict__ xu, int d, const T* __restrict__ Vu,
                                                  const T* __restrict__ P, const T* __restrict__ g, int s, double ss2,
                                                  double noise, double* __restrict__ cov) {
  const int4 it = items[blockIdx.x];
  const CovReq rq = reqs[it.x];
  const int a0 = it.y * TB, b0 = it.z * TB, nua = rq.nua, nub = rq.nub;
  const int64_t ua = rq.u0a, ub = rq.u0b;
  const bool band = rq.nm > 0;
  __shared__ GemmSmem<T> sm;
  __shared__ T xa[TB][MAXD + 1];
  __shared__ T xb[TB][MAXD + 1];
  T sub[4][4] = {}, add[4][4] = {};
  if (band) {
    for (int e = threadIdx.x; e < TB * d; e += NT) {
      const int r = e / d, q = e % d;
      xa[r][q] = (a0 + r < nua) ? xu[(ua + a0 + r) * d + q] : T(0);
      xb[r][q] = (b0 + r < nub) ? xu[(ub + b0 + r) * d + q] : T(0);
    }
    {
      auto fa = [&](int r, int k) -> T { return (a0 + r < nua) ? Vu[(ua + a0 + r) * s + k] : T(0); };
      auto fb = [&](int r, int k) -> T { return (b0 + r < nub) ? Vu[(ub + b0 + r) * s + k] : T(0); };
      tile_mma<T, true, true>(sub, s, sm, fa, fb);
    }
    for (int j = 0; j < rq.nm; ++j) {
      const Pair pa = pairs[rq.pa + j], pb = pairs[rq.pb + j];
      const Win w = wins[pa.win];  // pb.win is the same window
      const int c0 = (rq.m_lo + j < rq.lo) ? w.nB : 0;
      const T* Pa = P + pa.pbase;
      const T* Pb = P + pb.pbase;
      const int64_t ld = w.npad;
      auto fa = [&](int r, int k) -> T { return (a0 + r < nua) ? Pa[(int64_t)(a0 + r) * ld + c0 + k] : T(0); };
      auto fb = [&](int r, int k) -> T { return (b0 + r < nub) ? Pb[(int64_t)(b0 + r) * ld + c0 + k] : T(0); };
      tile_mma<T, true, true>(sub, w.n - c0, sm, fa, fb);
    }
  }
  {
    auto fa = [&](int r, int k) -> T { return (a0 + r < nua) ? g[(ua + a0 + r) * s + k] : T(0); };
    auto fb = [&](int r, int k) -> T { return (b0 + r < nub) ? g[(ub + b0 + r) * s + k] : T(0); };
    tile_mma<T, true, true>(add, s, sm, fa, fb);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double* C = cov + rq.off;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = ty + 16 * a, c = tx + 16 * b;
      const int i = a0 + r, j = b0 + c;
      if (i < nua && j < nub) {
        double v = (double)add[a][b];
        if (band) {
          double d2 = 0.0;
          for (int q = 0; q < d; ++q) {
            const double t = (double)xa[r][q] - (double)xb[c][q];
            d2 += t * t;
          }
          v += ss2 * exp(-0.5 * d2) - (double)sub[a][b];
          if (rq.same && i == j) v += noise;
        }
        C[(int64_t)i * nub + j] = v;
      }
    }
}

// mean_u = mu + Vu_u . beta + t1_u ; var_u = sigma_s^2 [+ sigma_n^2] - |Vu_u|^2 - t2_u + |L_C^-1 h_u|^2
template <typename T>
__global__ void k_pred_final(const T* __restrict__ Vu, int64_t U, int s, const double* __restrict__ beta,
                             const double* __restrict__ t1, const double* __restrict__ t2,
                             const double* __restrict__ partial, int ntile, double mu, double prior,
                             double* __restrict__ mean, double* __restrict__ var) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= U) return;
  double a = 0.0, b = 0.0;
  for (int k = lane; k < s; k += 32) {
    double v = (double)Vu[warp * s + k];
    a += v * beta[k];
    b += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    double g = 0.0;
    for (int t = 0; t < ntile; ++t) g += partial[(int64_t)t * U + warp];
    mean[warp] = mu + a + t1[warp];
    var[warp] = prior - b - t2[warp] + g;
  }
}

}  // namespace lma
