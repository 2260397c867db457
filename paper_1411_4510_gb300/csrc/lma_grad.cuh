// Kernels of the hand-written adjoint of the LMA log-likelihood.
//
// Forward (whitened support coordinates, Vt = Sigma_DS L_SS^-T, C = I + A):
//   loglik = -1/2 (quad - y^T C^-1 y) - 1/2 (sum_m log|R_W| - log|R_B| + log|C|) - N/2 log 2 pi
// with, per window W = D_m u D^B_m and blanket B = D^B_m (Lemma 1):
//   quad, y, A = sum_m  Y_W^T R_W^-1 Y_W - Y_B^T R_B^-1 Y_B,   Y = [r | Vt].
// Reverse sweep, beta = C^-1 y, e = r - Vt beta, Lc = chol(C),
// Y-hat = [e | Vt Lc^-T], Phi_X = R_X^-1 Y-hat_X:
//   G_m   = 1/2 [Phi_W Phi_W^T - pad(Phi_B Phi_B^T) - (R_W^-1 - pad R_B^-1)]
//   Vt-bar += (Phi_W - pad Phi_B)[:,0] beta^T - (Phi_W - pad Phi_B)[:,1:] Lc^-1 - 2 G_m Vt_W
//   theta-bar += <G_m, dK_W/dtheta> + 2 sigma_n^2 tr G_m
// then K_DS-bar = Vt-bar L_SS^-1, L_SS-bar = -L_SS^-T Vt-bar^T Vt and the
// Cholesky adjoint back to Sigma_SS.  With the window factor L (blanket first,
// R_W = L L^T) every R^-1 product is a backward solve with L:
//   Phi_W = L^-T [L^-1 Y-hat],  pad Phi_B = L^-T [L^-1 Y-hat with block rows zeroed],
//   R_W^-1 - pad R_B^-1 = T T^T with T = L^-T [0; I_b].
#pragma once
#include "lma_kernels.cuh"

namespace lma {

// Backward right-hand sides of window w, stored as rows (length npad):
//   [0, s]        L^-1 Y-hat   (row 0 = L^-1 e, rows 1+i = (L^-1 Vt Lc^-T)[:, i])
//   [s+1, 2s+1]   the same with the block-part columns [nB, n) zeroed
//   [2s+2, ...)   unit rows e_{nB+t}, t < b
struct GWin {
  int64_t q;    // element offset of the RHS rows
  int64_t g;    // element offset of this window's G (npad x npad)
  int64_t gv;   // element offset of G^T-product rows (s x npad)
  int nrows;    // 2(s+1) + b
  int pad_;
};

// rows 1+i and s+2+i: sum_{k<=i} Lc^-1[i][k] X_{1+k}[c]  (LcT[k][i] = Lc^-1[i][k])
template <typename T>
__global__ void __launch_bounds__(NT) k_grad_rhs(const Win* __restrict__ wins, const GWin* __restrict__ gw,
                                                 const T* __restrict__ buf, const T* __restrict__ LcT, int s,
                                                 T* __restrict__ Q) {
  const Win w = wins[blockIdx.z];
  const GWin g = gw[blockIdx.z];
  const int c0 = blockIdx.x * TB, i0 = blockIdx.y * TB;
  if (c0 >= w.npad || i0 >= s) return;
  __shared__ GemmSmem<T> sm;
  const T* X = buf + w.base + (int64_t)w.npad * w.npad;  // extra rows of the forward sweep
  const int64_t ld = w.npad;
  const int K = min(s, i0 + TB);
  T acc[4][4] = {};
  auto fa = [&](int r, int k) -> T { return (i0 + r < s) ? LcT[(int64_t)k * s + i0 + r] : T(0); };
  auto fb = [&](int r, int k) -> T { return X[(int64_t)(1 + k) * ld + c0 + r]; };
  tile_mma<T, false, false>(acc, K, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T* Qw = Q + g.q;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = i0 + ty + 16 * a, c = c0 + tx + 16 * b;
      if (i >= s) continue;
      T v = (c < w.n) ? acc[a][b] : T(0);
      Qw[(int64_t)(1 + i) * ld + c] = v;
      Qw[(int64_t)(s + 2 + i) * ld + c] = (c >= w.nB) ? T(0) : v;
    }
}

// rows 0, s+1 (from L^-1 e) and the unit rows
template <typename T>
__global__ void k_grad_rhs_fill(const Win* __restrict__ wins, const GWin* __restrict__ gw,
                                const T* __restrict__ ew, int s, T* __restrict__ Q) {
  const Win w = wins[blockIdx.y];
  const GWin g = gw[blockIdx.y];
  T* Qw = Q + g.q;
  const int ld = w.npad;
  const int b = w.n - w.nB;
  const int64_t total = (int64_t)(2 + b) * ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(e / ld), c = (int)(e % ld);
    if (r == 0) {
      Qw[c] = (c < w.n) ? ew[w.ew + c] : T(0);
    } else if (r == 1) {
      Qw[(int64_t)(s + 1) * ld + c] = (c < w.nB) ? ew[w.ew + c] : T(0);
    } else {
      int t = r - 2;
      Qw[(int64_t)(2 * s + 2 + t) * ld + c] = (c == w.nB + t) ? T(1) : T(0);
    }
  }
}

// Backward sweep: each RHS row q becomes x with x L = q (x = (L^-T q^T)^T),
// column panels from the last to the first (items: x = window, y = row tile).
template <typename T>
__global__ void __launch_bounds__(NT) k_bwd_sweep(const int2* __restrict__ items, const Win* __restrict__ wins,
                                                  const GWin* __restrict__ gw, const T* __restrict__ buf,
                                                  const T* __restrict__ dinv, T* __restrict__ Q) {
  const int2 it = items[blockIdx.x];
  const Win w = wins[it.x];
  const GWin g = gw[it.x];
  const int u0 = it.y * TB;
  extern __shared__ __align__(16) unsigned char smraw[];
  CholSmem<T>& sm = *reinterpret_cast<CholSmem<T>*>(smraw);
  const T* L = buf + w.base;
  const int64_t ld = w.npad;
  T* Qw = Q + g.q;
  const int nr = g.nrows;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int npan = w.npad / TB;
  for (int kp = npan - 1; kp >= 0; --kp) {
    const int k0 = kp * TB;
    const int t0 = k0 + TB;
    T acc[4][4] = {};
    auto fa = [&](int r, int k) -> T { return (u0 + r < nr) ? Qw[(int64_t)(u0 + r) * ld + t0 + k] : T(0); };
    auto fb = [&](int r, int k) -> T { return L[(int64_t)(t0 + k) * ld + k0 + r]; };
    tile_mma<T, true, false>(acc, w.npad - t0, sm.g, fa, fb);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int r = ty + 16 * a, c = tx + 16 * b;
        sm.D[r][c] = (u0 + r < nr) ? Qw[(int64_t)(u0 + r) * ld + k0 + c] - acc[a][b] : T(0);
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
        b4[q] = sm.X[j][tx + 16 * q];
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
        if (u0 + r < nr) Qw[(int64_t)(u0 + r) * ld + k0 + tx + 16 * b] = o[a][b];
      }
    __syncthreads();
  }
}

// G_m tiles (lower, items: x = window, y = tile index) with the covariance
// derivative contraction fused in.  partial[blockIdx.x][0..d-1] log-length-scale
// terms, [d] log sigma_s, [d+1] log sigma_n.
template <typename T>
__global__ void __launch_bounds__(NT) k_grad_G(const int2* __restrict__ items, const Win* __restrict__ wins,
                                               const GWin* __restrict__ gw, const T* __restrict__ Q,
                                               const T* __restrict__ xs, int d, int s, double ss2, double sn2,
                                               T* __restrict__ Gbuf, double* __restrict__ partial) {
  const int2 it = items[blockIdx.x];
  const Win w = wins[it.x];
  const GWin g = gw[it.x];
  int I, J;
  tri_index(it.y, I, J);
  const int r0 = I * TB, c0 = J * TB;
  __shared__ GemmSmem<T> sm;
  __shared__ T xr[TB][MAXD + 1];
  __shared__ T xc[TB][MAXD + 1];
  __shared__ double red[NT];
  for (int e = threadIdx.x; e < TB * d; e += NT) {
    int r = e / d, q = e % d;
    xr[r][q] = (r0 + r < w.n) ? xs[(w.g_end - 1 - (r0 + r)) * d + q] : T(0);
    xc[r][q] = (c0 + r < w.n) ? xs[(w.g_end - 1 - (c0 + r)) * d + q] : T(0);
  }
  const T* Qw = Q + g.q;
  const int64_t ld = w.npad;
  const int b = w.n - w.nB;
  T acc[4][4] = {};
  {
    auto fa = [&](int r, int k) -> T { return Qw[(int64_t)k * ld + r0 + r]; };
    auto fb = [&](int r, int k) -> T { return Qw[(int64_t)k * ld + c0 + r]; };
    tile_mma<T, false, false>(acc, s + 1, sm, fa, fb);
  }
  {
    const T* P = Qw + (int64_t)(s + 1) * ld;
    auto fa = [&](int r, int k) -> T { return P[(int64_t)k * ld + r0 + r]; };
    auto fb = [&](int r, int k) -> T { return -P[(int64_t)k * ld + c0 + r]; };
    tile_mma<T, false, false>(acc, s + 1, sm, fa, fb);
  }
  {
    const T* P = Qw + (int64_t)(2 * s + 2) * ld;
    auto fa = [&](int r, int k) -> T { return P[(int64_t)k * ld + r0 + r]; };
    auto fb = [&](int r, int k) -> T { return -P[(int64_t)k * ld + c0 + r]; };
    tile_mma<T, false, false>(acc, b, sm, fa, fb);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const double wgt = (I == J) ? 1.0 : 2.0;
  double gl[MAXD];
  for (int q = 0; q < d; ++q) gl[q] = 0.0;
  double gsig = 0.0, gnoise = 0.0;
  T* G = Gbuf + g.g;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      int r = ty + 16 * a, c = tx + 16 * bb;
      int gi = r0 + r, gj = c0 + c;
      T v = T(0.5) * acc[a][bb];
      if (gi < w.n && gj < w.n) {
        double d2 = 0.0;
        for (int q = 0; q < d; ++q) {
          double t = (double)xr[r][q] - (double)xc[c][q];
          d2 += t * t;
        }
        double kg = (double)v * ss2 * exp(-0.5 * d2) * wgt;
        for (int q = 0; q < d; ++q) {
          double t = (double)xr[r][q] - (double)xc[c][q];
          gl[q] += kg * t * t;
        }
        gsig += 2.0 * kg;
        if (gi == gj) gnoise += 2.0 * sn2 * (double)v;
      } else {
        v = T(0);
      }
      G[(int64_t)gi * ld + gj] = v;
      if (I != J) G[(int64_t)gj * ld + gi] = v;
    }
  // block reduction of d+2 values
  double* P = partial + (int64_t)blockIdx.x * (d + 2);
  for (int q = 0; q < d + 2; ++q) {
    double v = (q < d) ? gl[q] : (q == d ? gsig : gnoise);
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) P[q] = red[0];
    __syncthreads();
  }
}

// GVt_w[k][i] = sum_j Vt[g(j)][k] G[j][i]   (grid: npad tiles, s tiles, windows)
template <typename T>
__global__ void __launch_bounds__(NT) k_grad_gv(const Win* __restrict__ wins, const GWin* __restrict__ gw,
                                                const T* __restrict__ Gbuf, const T* __restrict__ Vt, int s,
                                                T* __restrict__ GV) {
  const Win w = wins[blockIdx.z];
  const GWin g = gw[blockIdx.z];
  const int c0 = blockIdx.x * TB, k0 = blockIdx.y * TB;
  if (c0 >= w.npad || k0 >= s) return;
  __shared__ GemmSmem<T> sm;
  const T* G = Gbuf + g.g;
  const int64_t ld = w.npad;
  T acc[4][4] = {};
  auto fa = [&](int r, int j) -> T { return (k0 + r < s && j < w.n) ? Vt[(w.g_end - 1 - j) * s + k0 + r] : T(0); };
  auto fb = [&](int r, int j) -> T { return G[(int64_t)j * ld + c0 + r]; };
  tile_mma<T, false, false>(acc, w.n, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T* O = GV + g.gv;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int k = k0 + ty + 16 * a, c = c0 + tx + 16 * b;
      if (k < s) O[(int64_t)k * ld + c] = acc[a][b];
    }
}

// Gather the per-window contributions onto training rows (fixed window order):
//   PsiT[k][p] = sum_{m: p in W_m} (Phi_W - pad Phi_B)[k][i_m(p)]     k in [0, s]
//   GVT[k][p]  = sum_{m: p in W_m} GVt_m[k][i_m(p)]                   k in [0, s)
// over the windows of the gradient only: window of block m is wins[m - w0],
// taken when m - w0 is in [k_lo, k_hi), its backward layout gw[m - w0 - k_lo].
// (grid: x over rows p, y over k in [0, 2s+1))
template <typename T>
__global__ void k_grad_gather(const Win* __restrict__ wins, const GWin* __restrict__ gw,
                              const int64_t* __restrict__ bptr, int M, int B, int64_t n, int s,
                              const T* __restrict__ Q, const T* __restrict__ GV, T* __restrict__ PsiT,
                              T* __restrict__ GVT, int w0, int k_lo, int k_hi) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (p >= n) return;
  int lo = 0, hi = M;  // block of row p: bptr[j] <= p < bptr[j+1]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (bptr[mid] <= p) lo = mid;
    else hi = mid;
  }
  const int j = lo;
  double acc = 0.0;
  for (int m = max(0, j - B); m <= j; ++m) {
    const int wi = m - w0;  // window index in the model
    if (wi < k_lo || wi >= k_hi) continue;
    const Win w = wins[wi];
    const GWin g = gw[wi - k_lo];
    const int i = (int)(w.g_end - 1 - p);
    if (k <= s) {
      const T* Qw = Q + g.q;
      acc += (double)Qw[(int64_t)k * w.npad + i] - (double)Qw[(int64_t)(s + 1 + k) * w.npad + i];
    } else {
      acc += (double)GV[g.gv + (int64_t)(k - s - 1) * w.npad + i];
    }
  }
  if (k <= s) PsiT[(int64_t)k * n + p] = (T)acc;
  else GVT[(int64_t)(k - s - 1) * n + p] = (T)acc;
}

// VbT[k][p] = beta_k Psi_e[p] - sum_{j>=k} Lc^-1[j][k] Psi_{1+j}[p] - 2 GVT[k][p]
template <typename T>
__global__ void __launch_bounds__(NT) k_grad_vbar(const T* __restrict__ PsiT, const T* __restrict__ GVT,
                                                  const T* __restrict__ LcT, const double* __restrict__ beta,
                                                  int64_t n, int s, T* __restrict__ VbT) {
  __shared__ GemmSmem<T> sm;
  const int k0 = blockIdx.y * TB;
  const int64_t p0 = (int64_t)blockIdx.x * TB;
  const int K = s - k0;
  T acc[4][4] = {};
  auto fa = [&](int r, int jj) -> T { return (k0 + r < s) ? LcT[(int64_t)(k0 + r) * s + k0 + jj] : T(0); };
  auto fb = [&](int r, int jj) -> T { return (p0 + r < n) ? PsiT[(int64_t)(1 + k0 + jj) * n + p0 + r] : T(0); };
  tile_mma<T, true, false>(acc, K, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int k = k0 + ty + 16 * a;
      int64_t p = p0 + tx + 16 * b;
      if (k < s && p < n)
        VbT[(int64_t)k * n + p] = (T)(beta[k] * (double)PsiT[p]) - acc[a][b] - T(2) * GVT[(int64_t)k * n + p];
    }
}

// K_DS-bar^T[k][p] = sum_{i>=k} (L_SS^-1)[i][k] VbT[i][p]  (ET[k][i] = L_SS^-1[i][k]),
// contracted on the fly with dK_DS/dtheta (no storage).
template <typename T>
__global__ void __launch_bounds__(NT) k_grad_kds(const T* __restrict__ VbT, const T* __restrict__ ET,
                                                 const T* __restrict__ xs, const T* __restrict__ ss, int d,
                                                 int64_t n, int s, double ss2, double* __restrict__ partial) {
  __shared__ GemmSmem<T> sm;
  __shared__ T xp[TB][MAXD + 1];
  __shared__ T xk[TB][MAXD + 1];
  __shared__ double red[NT];
  const int k0 = blockIdx.y * TB;
  const int64_t p0 = (int64_t)blockIdx.x * TB;
  for (int e = threadIdx.x; e < TB * d; e += NT) {
    int r = e / d, q = e % d;
    xk[r][q] = (k0 + r < s) ? ss[(int64_t)(k0 + r) * d + q] : T(0);
    xp[r][q] = (p0 + r < n) ? xs[(p0 + r) * d + q] : T(0);
  }
  const int K = s - k0;
  T acc[4][4] = {};
  auto fa = [&](int r, int ii) -> T { return (k0 + r < s) ? ET[(int64_t)(k0 + r) * s + k0 + ii] : T(0); };
  auto fb = [&](int r, int ii) -> T { return (p0 + r < n) ? VbT[(int64_t)(k0 + ii) * n + p0 + r] : T(0); };
  tile_mma<T, true, false>(acc, K, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double gl[MAXD];
  for (int q = 0; q < d; ++q) gl[q] = 0.0;
  double gsig = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int kr = ty + 16 * a, pc = tx + 16 * b;
      if (k0 + kr < s && p0 + pc < n) {
        double d2 = 0.0;
        for (int q = 0; q < d; ++q) {
          double t = (double)xk[kr][q] - (double)xp[pc][q];
          d2 += t * t;
        }
        double kg = (double)acc[a][b] * ss2 * exp(-0.5 * d2);
        for (int q = 0; q < d; ++q) {
          double t = (double)xk[kr][q] - (double)xp[pc][q];
          gl[q] += kg * t * t;
        }
        gsig += 2.0 * kg;
      }
    }
  double* P = partial + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * (d + 2);
  for (int q = 0; q < d + 1; ++q) {
    red[threadIdx.x] = (q < d) ? gl[q] : gsig;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) P[q] = red[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) P[d + 1] = 0.0;
}

// M1 = Vt-bar^T Vt (s x s) by chunks of rows p; FP64 partials per chunk.
template <typename T>
__global__ void __launch_bounds__(NT) k_grad_m1(const T* __restrict__ VbT, const T* __restrict__ Vt, int64_t n,
                                                int s, int64_t chunk, double* __restrict__ partial) {
  __shared__ GemmSmem<T> sm;
  const int i0 = blockIdx.y * TB, j0 = blockIdx.x * TB;
  const int64_t pb = blockIdx.z * chunk;
  const int64_t pe = min(n, pb + chunk);
  double accd[4][4] = {};
  for (int64_t q0 = pb; q0 < pe; q0 += 1024) {
    const int K = (int)min((int64_t)1024, pe - q0);
    T acc[4][4] = {};
    auto fa = [&](int r, int k) -> T { return (i0 + r < s) ? VbT[(int64_t)(i0 + r) * n + q0 + k] : T(0); };
    auto fb = [&](int r, int k) -> T { return (j0 + r < s) ? Vt[(q0 + k) * s + j0 + r] : T(0); };
    tile_mma<T, true, false>(acc, K, sm, fa, fb);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) accd[a][b] += (double)acc[a][b];
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double* P = partial + (int64_t)blockIdx.z * s * s;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < s && j < s) P[(int64_t)i * s + j] = accd[a][b];
    }
}

__global__ void k_sum_chunks(const double* __restrict__ partial, int nchunk, int64_t len, double* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= len) return;
  double v = 0.0;
  for (int c = 0; c < nchunk; ++c) v += partial[(int64_t)c * len + e];
  out[e] = v;
}

// Dense FP64 product C = alpha op(A) op(B) (s x s, row-major, leading dims lda/ldb/ldc).
template <bool TA, bool TBm>
__global__ void __launch_bounds__(NT) k_dgemm(const double* __restrict__ A, int64_t lda, const double* __restrict__ Bm,
                                              int64_t ldb, double* __restrict__ C, int64_t ldc, int s, double alpha) {
  __shared__ GemmSmem<double> sm;
  const int i0 = blockIdx.y * TB, j0 = blockIdx.x * TB;
  double acc[4][4] = {};
  auto fa = [&](int r, int k) -> double {
    int i = i0 + r;
    return i < s ? (TA ? A[(int64_t)k * lda + i] : A[(int64_t)i * lda + k]) : 0.0;
  };
  auto fb = [&](int r, int k) -> double {
    int j = j0 + r;
    return j < s ? (TBm ? Bm[(int64_t)j * ldb + k] : Bm[(int64_t)k * ldb + j]) : 0.0;
  };
  tile_mma<double, !TA, TBm>(acc, s, sm, fa, fb);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < s && j < s) C[(int64_t)i * ldc + j] = alpha * acc[a][b];
    }
}

// Phi(X): lower triangle with halved diagonal, in place (s x s, ld s)
static __global__ void k_phi(double* __restrict__ X, int s) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)s * s) return;
  int i = (int)(e / s), j = (int)(e % s);
  if (j > i) X[e] = 0.0;
  else if (j == i) X[e] *= 0.5;
}

// after k_phi on a copy of L: restore the diagonal halved by k_phi (x2)
static __global__ void k_tril_fix(double* __restrict__ X, int s) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)s * s) return;
  int i = (int)(e / s), j = (int)(e % s);
  if (i == j) X[e] *= 2.0;
}

// <Sigma-bar_SS, dK_SS/dtheta> (jitter held fixed); one CTA row-chunk per block
static __global__ void k_grad_kss(const double* __restrict__ Sb, const double* __restrict__ ss, int s, int d,
                                  double ss2, double* __restrict__ partial) {
  __shared__ double red[NT];
  double gl[MAXD];
  for (int q = 0; q < d; ++q) gl[q] = 0.0;
  double gsig = 0.0;
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < s; j += NT) {
    double d2 = 0.0;
    for (int q = 0; q < d; ++q) {
      double t = ss[(int64_t)i * d + q] - ss[(int64_t)j * d + q];
      d2 += t * t;
    }
    double kg = Sb[(int64_t)i * s + j] * ss2 * exp(-0.5 * d2);
    for (int q = 0; q < d; ++q) {
      double t = ss[(int64_t)i * d + q] - ss[(int64_t)j * d + q];
      gl[q] += kg * t * t;
    }
    gsig += 2.0 * kg;
  }
  double* P = partial + (int64_t)i * (d + 2);
  for (int q = 0; q < d + 1; ++q) {
    red[threadIdx.x] = (q < d) ? gl[q] : gsig;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) P[q] = red[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) P[d + 1] = 0.0;
}

}  // namespace lma
