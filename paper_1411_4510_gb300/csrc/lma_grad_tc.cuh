// Tensor-core (3xTF32, tcgen05) forms of the adjoint's window products, for
// the mixed form.  They compute what the SIMT kernels of lma_grad.cuh compute
// (the reverse sweep of the log-likelihood, Definition 2 and Theorem 2
// differentiated through Lemma 1's window factors), with the operands that
// are read along columns staged transposed by tc::tile_product2.
//
// Every kernel: 256 threads, one 128 x 64 output tile per CTA, the product in
// tensor memory (64 columns), read back by warp w for rows 32 (w mod 4) + lane
// and columns 32 (w / 4) + j.
#pragma once
#include "lma_grad.cuh"
#include "lma_tc.cuh"

namespace lma {

namespace gtc {

// Shared set-up / tear-down of the one-tile kernels.
__device__ __forceinline__ uint32_t setup(tc::TcSmem<64>& sm) {
  using namespace tc;
  if (threadIdx.x == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(&sm.tmem, 64);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  return sm.tmem;
}

__device__ __forceinline__ void teardown(tc::TcSmem<64>& sm) {
  using namespace tc;
  fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(sm.tmem, 64);
}

// This thread's 32 accumulator values.
__device__ __forceinline__ void read_acc(uint32_t tmem, float (&v)[32]) {
  using namespace tc;
  const int warp = threadIdx.x >> 5;
  const uint32_t a = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (warp >> 2) * 32;
  float t[16];
  tmem_ld16(a, t);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = t[j];
  tmem_ld16(a + 16, t);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[16 + j] = t[j];
}

}  // namespace gtc

// Rows 1 + i and s + 2 + i of the backward right-hand sides (see GWin):
// sum_{k <= i} Lc^-1[i][k] X_{1+k}[c], X = the forward sweep's extra rows
// (LcT[k][i] = Lc^-1[i][k]).  Grid: (64-column tiles, 128-row tiles of i, windows).
__global__ void __launch_bounds__(256, 2) k_grad_rhs_tc(const Win* __restrict__ wins, const GWin* __restrict__ gw,
                                                     const float* __restrict__ buf, const float* __restrict__ LcT,
                                                     int s, float* __restrict__ Q, int* __restrict__ err) {
  const Win w = wins[blockIdx.z];
  const GWin g = gw[blockIdx.z];
  const int c0 = blockIdx.x * 64, i0 = blockIdx.y * 128;
  if (c0 >= w.npad || i0 >= s) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  tc::TcSmem<64>& sm = tc::tc_smem<64>(smraw);
  const uint32_t tmem = gtc::setup(sm);
  const int64_t ld = w.npad;
  const float* X = buf + w.base + (int64_t)w.npad * w.npad;
  const int K = min(s, i0 + 128);
  tc::TcPipe pipe;
  auto rowA = [&](int k) -> const float* { return k < K ? LcT + (int64_t)k * s + i0 : nullptr; };
  auto rowB = [&](int k) -> const float* { return k < K ? X + (int64_t)(1 + k) * ld + c0 : nullptr; };
  const bool ok = tc::tile_product2<64, true, true>(sm, pipe, tmem, K, rowA, rowB, s - i0, 64, false, false);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  if (ok) {
    float v[32];
    gtc::read_acc(tmem, v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = i0 + (warp & 3) * 32 + lane;
    const int cb = c0 + (warp >> 2) * 32;
    if (i < s) {
      float* Qa = Q + g.q + (int64_t)(1 + i) * ld + cb;
      float* Qb = Q + g.q + (int64_t)(s + 2 + i) * ld + cb;
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4) {
        float4 a, b;
        float* pa = &a.x;
        float* pb = &b.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int c = cb + 4 * j4 + e;
          const float x = c < w.n ? v[4 * j4 + e] : 0.f;
          pa[e] = x;
          pb[e] = c >= w.nB ? 0.f : x;
        }
        *reinterpret_cast<float4*>(Qa + 4 * j4) = a;
        *reinterpret_cast<float4*>(Qb + 4 * j4) = b;
      }
    }
  }
  gtc::teardown(sm);
}

// Backward sweep: every right-hand-side row q of the window becomes x with
// x L = q, column panels from the last to the first:
//   T = Q[:, panel] - Q[:, t0:npad] L[t0:npad, panel],   Q[:, panel] = T inv(L_kk)
// (t0 = k0 + 64; L's panel columns and inv(L_kk) enter transposed).
// items: x = window, y = 128-row tile of the window's right-hand sides.
__global__ void __launch_bounds__(256, 2) k_bwd_sweep_tc(const int2* __restrict__ items, const Win* __restrict__ wins,
                                                      const GWin* __restrict__ gw, const float* __restrict__ buf,
                                                      const float* __restrict__ dinv, float* __restrict__ Q,
                                                      int* __restrict__ err) {
  const int2 it = items[blockIdx.x];
  const Win w = wins[it.x];
  const GWin g = gw[it.x];
  const int u0 = it.y * 128;
  extern __shared__ __align__(16) unsigned char smraw[];
  tc::TcSmem<64>& sm = tc::tc_smem<64>(smraw);
  const uint32_t tmem = gtc::setup(sm);
  const float* L = buf + w.base;
  const int64_t ld = w.npad;
  float* Qw = Q + g.q;
  const int nr = g.nrows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rl = (warp & 3) * 32 + lane, half = warp >> 2;
  const bool live = u0 + rl < nr;
  float* myrow = Qw + (int64_t)(u0 + rl) * ld;
  tc::TcPipe pipe;
  bool ok = true;
  for (int kp = w.npad / TB - 1; kp >= 0 && ok; --kp) {
    const int k0 = kp * TB, t0 = k0 + TB, K = w.npad - t0;
    float v[32];
    if (K > 0) {
      auto rowA = [&](int r) -> const float* { return u0 + r < nr ? Qw + (int64_t)(u0 + r) * ld + t0 : nullptr; };
      auto rowB = [&](int k) -> const float* { return L + (int64_t)(t0 + k) * ld + k0; };
      ok = tc::tile_product2<64, false, true>(sm, pipe, tmem, K, rowA, rowB, 128, 64, false, false);
      if (!ok) break;
      gtc::read_acc(tmem, v);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = 0.f;
    }
    if (live) {
      float* dst = myrow + k0 + half * 32;
      float4 av[8];
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4) av[j4] = *reinterpret_cast<const float4*>(dst + 4 * j4);
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4) {
        float4 a = av[j4];
        a.x -= v[4 * j4 + 0];
        a.y -= v[4 * j4 + 1];
        a.z -= v[4 * j4 + 2];
        a.w -= v[4 * j4 + 3];
        *reinterpret_cast<float4*>(dst + 4 * j4) = a;
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    const float* Dv = dinv + w.dinv + (int64_t)kp * TB * TB;
    auto rowT = [&](int r) -> const float* { return u0 + r < nr ? Qw + (int64_t)(u0 + r) * ld + k0 : nullptr; };
    auto rowD = [&](int k) -> const float* { return Dv + (int64_t)k * TB; };
    ok = tc::tile_product2<64, false, true>(sm, pipe, tmem, TB, rowT, rowD, 128, 64, false, false);
    if (!ok) break;
    gtc::read_acc(tmem, v);
    if (live) {
      float* dst = myrow + k0 + half * 32;
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4)
        *reinterpret_cast<float4*>(dst + 4 * j4) = make_float4(v[4 * j4], v[4 * j4 + 1], v[4 * j4 + 2], v[4 * j4 + 3]);
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  gtc::teardown(sm);
}

// G_m tiles with the covariance-derivative contraction fused in:
//   G = 1/2 [sum_{k<=s} Q_k Q_k^T - sum_{k<=s} Q_{s+1+k} Q_{s+1+k}^T - sum_{t<b} Q_{2s+2+t} Q_{2s+2+t}^T]
// over rows [128 I, 128 I + 128) x columns [64 J, 64 J + 64) of the window's
// lower triangle (items: window, I, J; J <= 2 I + 1).  Each element (i, j),
// j <= i, of the window adds wgt G_ij dK_ij/dtheta (wgt 2 below the diagonal)
// to partial[item][0 .. d+1] and is written to G[i][j] and G[j][i].
__global__ void __launch_bounds__(256, 2) k_grad_G_tc(const int4* __restrict__ items, const Win* __restrict__ wins,
                                                   const GWin* __restrict__ gw, const float* __restrict__ Q,
                                                   const float* __restrict__ xs, int d, int s, float ss2, double sn2,
                                                   float* __restrict__ Gbuf, double* __restrict__ partial,
                                                   int* __restrict__ err) {
  const int4 it = items[blockIdx.x];
  const Win w = wins[it.x];
  const GWin g = gw[it.x];
  const int r0 = it.y * 128, c0 = it.z * 64;
  extern __shared__ __align__(16) unsigned char smraw[];
  tc::TcSmem<64>& sm = tc::tc_smem<64>(smraw);
  __shared__ float xc[64][MAXD + 1];
  __shared__ double red[8][MAXD + 2];
  for (int e = threadIdx.x; e < 64 * d; e += blockDim.x) {
    const int c = e / d, q = e % d;
    xc[c][q] = (c0 + c < w.n) ? xs[(w.g_end - 1 - (c0 + c)) * d + q] : 0.f;
  }
  const uint32_t tmem = gtc::setup(sm);
  const float* Qw = Q + g.q;
  const int64_t ld = w.npad;
  const int b = w.n - w.nB;
  const int alim = w.npad - r0;
  tc::TcPipe pipe;
  bool ok = true;
  {
    const int K = s + 1;
    auto rowA = [&](int k) -> const float* { return k < K ? Qw + (int64_t)k * ld + r0 : nullptr; };
    auto rowB = [&](int k) -> const float* { return k < K ? Qw + (int64_t)k * ld + c0 : nullptr; };
    ok = tc::tile_product2<64, true, true>(sm, pipe, tmem, K, rowA, rowB, alim, 64, false, false);
  }
  if (ok) {
    const int K = s + 1;
    const float* P = Qw + (int64_t)(s + 1) * ld;
    auto rowA = [&](int k) -> const float* { return k < K ? P + (int64_t)k * ld + r0 : nullptr; };
    auto rowB = [&](int k) -> const float* { return k < K ? P + (int64_t)k * ld + c0 : nullptr; };
    ok = tc::tile_product2<64, true, true>(sm, pipe, tmem, K, rowA, rowB, alim, 64, true, true);
  }
  if (ok && b > 0) {
    const float* P = Qw + (int64_t)(2 * s + 2) * ld;
    auto rowA = [&](int k) -> const float* { return k < b ? P + (int64_t)k * ld + r0 : nullptr; };
    auto rowB = [&](int k) -> const float* { return k < b ? P + (int64_t)k * ld + c0 : nullptr; };
    ok = tc::tile_product2<64, true, true>(sm, pipe, tmem, b, rowA, rowB, alim, 64, true, true);
  }
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double gl[MAXD];
#pragma unroll
  for (int q = 0; q < MAXD; ++q) gl[q] = 0.0;
  double gsig = 0.0, gnoise = 0.0;
  if (ok) {
    float v[32];
    gtc::read_acc(tmem, v);
    const int gi = r0 + (warp & 3) * 32 + lane;
    const int cb = (warp >> 2) * 32;
    float xr[MAXD];
#pragma unroll
    for (int q = 0; q < MAXD; ++q) xr[q] = (q < d && gi < w.n) ? xs[(w.g_end - 1 - gi) * d + q] : 0.f;
    float* G = Gbuf + g.g;
    if (gi < w.npad) {
      // the thread's 32 terms are summed in FP32 (a short sum of products
      // that are themselves FP32), then added to the FP64 sums once
      float glf[MAXD];
#pragma unroll
      for (int q = 0; q < MAXD; ++q) glf[q] = 0.f;
      float gsf = 0.f;
      for (int j = 0; j < 32; ++j) {
        const int gj = c0 + cb + j;
        if (gj > gi) break;
        float val = 0.5f * v[j];
        if (gi < w.n && gj < w.n) {
          float d2 = 0.f;
          for (int q = 0; q < d; ++q) {
            const float t = xr[q] - xc[cb + j][q];
            d2 = fmaf(t, t, d2);
          }
          const float kg = val * ss2 * expf(-0.5f * d2) * (gi == gj ? 1.f : 2.f);
          for (int q = 0; q < d; ++q) {
            const float t = xr[q] - xc[cb + j][q];
            glf[q] = fmaf(kg, t * t, glf[q]);
          }
          gsf += kg;
          if (gi == gj) gnoise += 2.0 * sn2 * (double)val;
        } else {
          val = 0.f;
        }
        G[(int64_t)gi * ld + gj] = val;
        G[(int64_t)gj * ld + gi] = val;
      }
      for (int q = 0; q < d; ++q) gl[q] += (double)glf[q];
      gsig += 2.0 * (double)gsf;
    }
  }
  // block reduction of the d + 2 sums: warp shuffles, then one value per warp
  for (int q = 0; q < d + 2; ++q) {
    double x = q < d ? gl[q] : (q == d ? gsig : gnoise);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < d + 2) {
    double x = 0.0;
    for (int k = 0; k < 8; ++k) x += red[k][threadIdx.x];
    partial[(int64_t)blockIdx.x * (d + 2) + threadIdx.x] = x;
  }
  gtc::teardown(sm);
}

// GVt_w[k][i] = sum_j Vt[g(j)][k] G[j][i] (G symmetric, so row i of G is the
// B operand; Vt's rows enter transposed).  Grid: (64-column tiles of i,
// 128-row tiles of k, windows).
__global__ void __launch_bounds__(256, 2) k_grad_gv_tc(const Win* __restrict__ wins, const GWin* __restrict__ gw,
                                                    const float* __restrict__ Gbuf, const float* __restrict__ Vt,
                                                    int s, float* __restrict__ GV, int* __restrict__ err) {
  const Win w = wins[blockIdx.z];
  const GWin g = gw[blockIdx.z];
  const int c0 = blockIdx.x * 64, k0 = blockIdx.y * 128;
  if (c0 >= w.npad || k0 >= s) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  tc::TcSmem<64>& sm = tc::tc_smem<64>(smraw);
  const uint32_t tmem = gtc::setup(sm);
  const float* G = Gbuf + g.g;
  const int64_t ld = w.npad;
  tc::TcPipe pipe;
  auto rowA = [&](int j) -> const float* { return j < w.n ? Vt + (w.g_end - 1 - j) * s + k0 : nullptr; };
  auto rowB = [&](int c) -> const float* { return G + (int64_t)(c0 + c) * ld; };
  const bool ok = tc::tile_product2<64, true, false>(sm, pipe, tmem, w.n, rowA, rowB, s - k0, 64, false, false);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  if (ok) {
    float v[32];
    gtc::read_acc(tmem, v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = k0 + (warp & 3) * 32 + lane;
    if (k < s) {
      float* O = GV + g.gv + (int64_t)k * ld + c0 + (warp >> 2) * 32;
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4)
        *reinterpret_cast<float4*>(O + 4 * j4) = make_float4(v[4 * j4], v[4 * j4 + 1], v[4 * j4 + 2], v[4 * j4 + 3]);
    }
  }
  gtc::teardown(sm);
}

}  // namespace lma
