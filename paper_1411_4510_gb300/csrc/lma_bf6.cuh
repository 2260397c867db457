// Support-set projection on the tensor cores with FP32-accurate products
// (mixed form): V^T = K_DS L_SS^-T, i.e. Vt[p][i] = sum_{k <= i} K(x_p, s_k)
// (L_SS^-1)[i][k] (Section 3: Q = Sigma_DS Sigma_SS^-1 Sigma_SD = Vt Vt^T with
// V = L_SS^-1 Sigma_SD), and the prediction's variance term L_C^-1 h of the
// same triangular shape.
//
// Operands are split into three bfloat16 pieces, x = x1 + x2 + x3 (8 + 8 + 8
// significant bits, exact for an FP32 x up to the last bit of x3), and a
// product is taken as a1 b1 + (a1 b2 + a2 b1 + a1 b3 + a2 b2 + a3 b1): the
// six kind::f16 MMAs keep every term down to 2^-16 of the leading one, so each
// product is accurate to about 2^-24 relative (the published bf16x6 split of
// Henry, Tang and Heinecke, 2019), at the issue cost of three TF32 MMAs.
// The leading term accumulates in its own tensor-memory accumulator and the
// five correction terms in a second one, so the truncating FP32 accumulation
// of the tensor core acts on each at its own scale; both are drained into
// FP32 registers (round to nearest) every 64 values of K.  A numpy emulation
// of this scheme (truncating 16-wide MMA steps) gave a smaller error on V
// than sequential FP32 FMA: 2.1e-5 vs 2.4e-5 relative at |S| = 64 with
// cond(Sigma_SS) ~ 1e7, 2.6e-6 vs 5.0e-6 at |S| = 512.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lma_tc.cuh"

namespace lma {
namespace bf6 {

constexpr int KC = 64;        // K values per chunk: one 128-byte swizzled row of bfloat16
constexpr int NST = 2;        // pipeline stages
constexpr int NWK = 16;       // worker warps (4 lane quarters x 4 groups of 32 columns)
constexpr int NTHR = 32 * (NWK + 2);  // + MMA warp + TMA warp
constexpr uint32_t kTileBytes = 128u * KC * 2u;  // one 128 x 64 bfloat16 box (16 KB)

// Three bfloat16 pieces of an FP32 value (round to nearest each time; the
// two differences are exact in FP32).
__device__ __forceinline__ uint32_t bf16x2_rn(float lo_elem, float hi_elem) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_elem), "f"(lo_elem));
  return r;
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

// Splits two FP32 values into three packed bfloat16 pairs p[0..2].
__device__ __forceinline__ void split3x2(float x0, float x1, uint32_t (&p)[3]) {
  p[0] = bf16x2_rn(x0, x1);
  const float r0 = x0 - bf16_lo(p[0]), r1 = x1 - bf16_hi(p[0]);
  p[1] = bf16x2_rn(r0, r1);
  const float s0 = r0 - bf16_lo(p[1]), s1 = r1 - bf16_hi(p[1]);
  p[2] = bf16x2_rn(s0, s1);
}

// Instruction descriptor of kind::f16 with bfloat16 A and B (K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

struct alignas(1024) Stage {
  uint16_t a[3][128 * KC];
  uint16_t b[3][128 * KC];
};
struct Smem {
  Stage st[NST];
  uint64_t full[NST], empty[NST], done[2], drained[2], fin;
  uint32_t tmem;
  int abort;
};
__device__ __forceinline__ Smem& smem_of(unsigned char* raw) {
  uintptr_t p = reinterpret_cast<uintptr_t>(raw);
  p = (p + 1023) & ~uintptr_t(1023);
  return *reinterpret_cast<Smem*>(p);
}
inline size_t smem_bytes() { return sizeof(Smem) + 1024; }

// Persistent loop over output tiles: the CTA's k-th tile is order(k) (a
// negative value ends the loop; every role walks the same sequence).  Tile t
// accumulates, over its chunks c < chunks(t), the
// product of the 128 x 64 boxes at (x, ya) of A and (x, yb) of B with
// (x, ya, yb) = at(coords(t), c); plane q of an operand is the box at row
// offset q * (plane rows) of its tensor map.  Workers drain the two
// accumulators after every chunk and call after(t, acc) with worker warp w's
// row 32 (w mod 4) + lane and columns 32 (w / 4) + j in acc[j].  Every wait
// has an iteration limit; on a timeout all roles stop, no copy is left
// landing, and false is returned in every thread.
template <class Order, class Chunks, class Coords, class At, class After>
__device__ bool persistent(Smem& sm, const CUtensorMap* amap, int arows, const CUtensorMap* bmap, int brows,
                           Order order, Chunks chunks, Coords coords, At at, After after) {
  using namespace tc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_flag = &sm.abort;
  if (warp < NWK) {
    const int q = warp & 3, half = warp >> 2;
    const uint32_t tlane = sm.tmem + ((uint32_t)(q * 32) << 16) + half * 32;
    int G = 0;  // chunks drained so far by this CTA
    bool ok = true;
    for (int k = 0;; ++k) {
      const int t = order(k);
      if (t < 0) break;
      float acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0.f;
      const int nchunk = chunks(t);
      for (int c = 0; c < nchunk && ok; ++c, ++G) {
        const int a = G & 1;
        int okw = 1;
        if (lane == 0) okw = mbar_wait(&sm.done[a], (G >> 1) & 1) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        fence_after_sync();
        float m[16], e[16];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tmem_ld16(tlane + 256 * a + 16 * h, m);
          tmem_ld16(tlane + 256 * a + 128 + 16 * h, e);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[16 * h + j] += m[j] + e[j];
        }
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.drained[a]);
      }
      ok = worker_sync_and(ok && !*abort_flag);
      if (!ok) break;
      after(t, acc);
    }
  } else if (warp == NWK) {
    // MMA warp: the whole warp runs the loops, lane 0 waits and issues
    const uint32_t idesc = idesc_bf16(128, 128);
    int C = 0;  // chunks issued so far by this CTA
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int t = order(k);
      if (t < 0) break;
      const int nchunk = chunks(t);
      for (int c = 0; c < nchunk; ++c, ++C) {
        const int s = C % NST, a = C & 1;
        int okw = 1;
        if (lane == 0) {
          okw = mbar_wait(&sm.full[s], (C / NST) & 1) ? 1 : 0;
          if (okw && C >= 2) okw = mbar_wait(&sm.drained[a], ((C - 2) >> 1) & 1) ? 1 : 0;
        }
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw || *abort_flag) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        fence_after_sync();
        if (lane == 0) {
          Stage& S = sm.st[s];
          uint32_t ad[3], bd[3];
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            ad[p] = smem_addr(S.a[p]);
            bd[p] = smem_addr(S.b[p]);
          }
          const uint32_t dm = sm.tmem + 256 * a, de = dm + 128;
#pragma unroll
          for (int ks = 0; ks < KC / 16; ++ks) {
            const uint32_t o = ks * 32;  // 16 bfloat16 values of K per MMA
            const uint32_t first = ks > 0 ? 1u : 0u;
            mma_bf16(dm, sdesc_sw128(ad[0] + o), sdesc_sw128(bd[0] + o), idesc, first);
            mma_bf16(de, sdesc_sw128(ad[0] + o), sdesc_sw128(bd[1] + o), idesc, first);
            mma_bf16(de, sdesc_sw128(ad[1] + o), sdesc_sw128(bd[0] + o), idesc, 1u);
            mma_bf16(de, sdesc_sw128(ad[0] + o), sdesc_sw128(bd[2] + o), idesc, 1u);
            mma_bf16(de, sdesc_sw128(ad[1] + o), sdesc_sw128(bd[1] + o), idesc, 1u);
            mma_bf16(de, sdesc_sw128(ad[2] + o), sdesc_sw128(bd[0] + o), idesc, 1u);
          }
          mma_commit(&sm.empty[s]);  // the stage may be refilled
          mma_commit(&sm.done[a]);   // the accumulators may be drained
        }
        __syncwarp();
      }
    }
    if (lane == 0) mma_commit(&sm.fin);  // arrives once every MMA issued above has completed
    __syncwarp();
  } else {
    // TMA producer: the whole warp runs the loops, lane 0 waits and issues
    int C = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int t = order(k);
      if (t < 0) break;
      const int4 base = coords(t);
      const int nchunk = chunks(t);
      for (int c = 0; c < nchunk; ++c, ++C) {
        const int s = C % NST;
        int okw = 1;
        if (lane == 0 && C >= NST) okw = mbar_wait(&sm.empty[s], (C / NST - 1) & 1) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw || *abort_flag) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        if (lane == 0) {
          Stage& S = sm.st[s];
          const int3 y = at(base, c);
          mbar_arrive_expect_tx(&sm.full[s], 6u * kTileBytes);
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            tma_load_2d(S.a[p], amap, y.x, y.y + p * arows, &sm.full[s]);
            tma_load_2d(S.b[p], bmap, y.x, y.z + p * brows, &sm.full[s]);
          }
        }
        __syncwarp();
      }
    }
    // no copy may still be landing in shared memory when the CTA leaves
    if (lane == 0)
      for (int c = C > NST ? C - NST : 0; c < C; ++c) mbar_wait(&sm.full[c % NST], (c / NST) & 1);
    __syncwarp();
  }
  const bool w = mbar_wait(&sm.fin, 0);
  return __syncthreads_and(w && !*abort_flag) != 0;
}

// persistent() with the chunks' results added by TwoSum into (hi, lo), for
// products whose K runs long (thousands of values): after(t, hi, lo).
template <class Order, class Chunks, class Coords, class At, class After>
__device__ bool persistent_comp(Smem& sm, const CUtensorMap* amap, int arows, const CUtensorMap* bmap, int brows,
                           Order order, Chunks chunks, Coords coords, At at, After after) {
  using namespace tc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_flag = &sm.abort;
  if (warp < NWK) {
    const int q = warp & 3, half = warp >> 2;
    const uint32_t tlane = sm.tmem + ((uint32_t)(q * 32) << 16) + half * 32;
    int G = 0;  // chunks drained so far by this CTA
    bool ok = true;
    for (int k = 0;; ++k) {
      const int t = order(k);
      if (t < 0) break;
      float hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.f;
      const int nchunk = chunks(t);
      for (int c = 0; c < nchunk && ok; ++c, ++G) {
        const int a = G & 1;
        int okw = 1;
        if (lane == 0) okw = mbar_wait(&sm.done[a], (G >> 1) & 1) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        fence_after_sync();
        float m[8], e[8];  // eight columns at a time keeps the TwoSum state in registers
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          tmem_ld8(tlane + 256 * a + 8 * h, m);
          tmem_ld8(tlane + 256 * a + 128 + 8 * h, e);
#pragma unroll
          for (int j = 0; j < 8; ++j) two_sum(hi[8 * h + j], lo[8 * h + j], m[j] + e[j]);
        }
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.drained[a]);
      }
      ok = worker_sync_and(ok && !*abort_flag);
      if (!ok) break;
      after(t, hi, lo);
    }
  } else if (warp == NWK) {
    // MMA warp: the whole warp runs the loops, lane 0 waits and issues
    const uint32_t idesc = idesc_bf16(128, 128);
    int C = 0;  // chunks issued so far by this CTA
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int t = order(k);
      if (t < 0) break;
      const int nchunk = chunks(t);
      for (int c = 0; c < nchunk; ++c, ++C) {
        const int s = C % NST, a = C & 1;
        int okw = 1;
        if (lane == 0) {
          okw = mbar_wait(&sm.full[s], (C / NST) & 1) ? 1 : 0;
          if (okw && C >= 2) okw = mbar_wait(&sm.drained[a], ((C - 2) >> 1) & 1) ? 1 : 0;
        }
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw || *abort_flag) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        fence_after_sync();
        if (lane == 0) {
          Stage& S = sm.st[s];
          uint32_t ad[3], bd[3];
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            ad[p] = smem_addr(S.a[p]);
            bd[p] = smem_addr(S.b[p]);
          }
          const uint32_t dm = sm.tmem + 256 * a, de = dm + 128;
#pragma unroll
          for (int ks = 0; ks < KC / 16; ++ks) {
            const uint32_t o = ks * 32;  // 16 bfloat16 values of K per MMA
            const uint32_t first = ks > 0 ? 1u : 0u;
            mma_bf16(dm, sdesc_sw128(ad[0] + o), sdesc_sw128(bd[0] + o), idesc, first);
            mma_bf16(de, sdesc_sw128(ad[0] + o), sdesc_sw128(bd[1] + o), idesc, first);
            mma_bf16(de, sdesc_sw128(ad[1] + o), sdesc_sw128(bd[0] + o), idesc, 1u);
            mma_bf16(de, sdesc_sw128(ad[0] + o), sdesc_sw128(bd[2] + o), idesc, 1u);
            mma_bf16(de, sdesc_sw128(ad[1] + o), sdesc_sw128(bd[1] + o), idesc, 1u);
            mma_bf16(de, sdesc_sw128(ad[2] + o), sdesc_sw128(bd[0] + o), idesc, 1u);
          }
          mma_commit(&sm.empty[s]);  // the stage may be refilled
          mma_commit(&sm.done[a]);   // the accumulators may be drained
        }
        __syncwarp();
      }
    }
    if (lane == 0) mma_commit(&sm.fin);  // arrives once every MMA issued above has completed
    __syncwarp();
  } else {
    // TMA producer: the whole warp runs the loops, lane 0 waits and issues
    int C = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int t = order(k);
      if (t < 0) break;
      const int4 base = coords(t);
      const int nchunk = chunks(t);
      for (int c = 0; c < nchunk; ++c, ++C) {
        const int s = C % NST;
        int okw = 1;
        if (lane == 0 && C >= NST) okw = mbar_wait(&sm.empty[s], (C / NST - 1) & 1) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw || *abort_flag) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        if (lane == 0) {
          Stage& S = sm.st[s];
          const int3 y = at(base, c);
          mbar_arrive_expect_tx(&sm.full[s], 6u * kTileBytes);
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            tma_load_2d(S.a[p], amap, y.x, y.y + p * arows, &sm.full[s]);
            tma_load_2d(S.b[p], bmap, y.x, y.z + p * brows, &sm.full[s]);
          }
        }
        __syncwarp();
      }
    }
    // no copy may still be landing in shared memory when the CTA leaves
    if (lane == 0)
      for (int c = C > NST ? C - NST : 0; c < C; ++c) mbar_wait(&sm.full[c % NST], (c / NST) & 1);
    __syncwarp();
  }
  const bool w = mbar_wait(&sm.fin, 0);
  return __syncthreads_and(w && !*abort_flag) != 0;
}

__device__ __forceinline__ void setup(Smem& sm) {
  using namespace tc;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&sm.done[a], 1);
      mbar_init(&sm.drained[a], NWK);
    }
    mbar_init(&sm.fin, 1);
    sm.abort = 0;
    mbar_fence_init();
  }
  if ((threadIdx.x >> 5) == NWK) tmem_alloc(&sm.tmem, 512);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}
__device__ __forceinline__ void teardown(Smem& sm) {
  using namespace tc;
  fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == NWK) tmem_dealloc(sm.tmem, 512);
}

}  // namespace bf6

// SE-ARD covariances between points and the support set, split into three
// bfloat16 planes: plane q, row p, column k holds piece q of
// K(x_p, s_k) = ss2 exp(-|xs_p - ss_k|^2 / 2) (FP32), zero for k >= s; planes
// are n rows of ld (a multiple of 64) values, plane q at rows [q n, q n + n).
// CTA: 32 points x 64 support points; thread: one point, 8 consecutive k.
// The support coordinates sit in shared memory dimension-major, so a thread
// reads its 8 values of one dimension with two 16-byte loads.
template <int D>
__global__ void __launch_bounds__(256) k_kds_bf3(const float* __restrict__ xs, int64_t n, int d,
                                                 const float* __restrict__ ss, int s, float ss2, int ld,
                                                 uint16_t* __restrict__ out) {
  __shared__ __align__(16) float sk[D][64];
  const int tid = threadIdx.x;
  const int k0 = blockIdx.x * 64;
  const int64_t p = (int64_t)blockIdx.y * 32 + (tid >> 3);
  for (int e = tid; e < 64 * D; e += 256) {
    const int r = e % 64, q = e / 64;
    sk[q][r] = (k0 + r < s && q < d) ? ss[(int64_t)(k0 + r) * d + q] : 0.f;
  }
  __syncthreads();
  if (p >= n) return;
  const int kk = (tid & 7) * 8;
  float d2[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) d2[j] = 0.f;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    if (q >= d) break;
    const float x = xs[p * d + q];
    const float4 a = *reinterpret_cast<const float4*>(&sk[q][kk]);
    const float4 b = *reinterpret_cast<const float4*>(&sk[q][kk + 4]);
    const float t[8] = {x - a.x, x - a.y, x - a.z, x - a.w, x - b.x, x - b.y, x - b.z, x - b.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) d2[j] = fmaf(t[j], t[j], d2[j]);
  }
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = (k0 + kk + j < s) ? ss2 * expf(-0.5f * d2[j]) : 0.f;
  uint32_t pk[3][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t t[3];
    bf6::split3x2(v[2 * j], v[2 * j + 1], t);
    pk[0][j] = t[0];
    pk[1][j] = t[1];
    pk[2][j] = t[2];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q)
    *reinterpret_cast<uint4*>(out + ((int64_t)q * n + p) * ld + k0 + kk) = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
}

// Three bfloat16 planes of an FP32 matrix A (rows x cols, leading dimension
// lda), columns padded with zeros to ld (a multiple of 8): plane q at rows
// [q rows, q rows + rows); with reverse, in reversed row order.  Thread: 8
// consecutive columns of one row.
__global__ void k_split_bf3(const float* __restrict__ A, int64_t rows, int cols, int64_t lda, int ld,
                            uint16_t* __restrict__ out, int reverse) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int per = ld / 8;
  if (e >= rows * per) return;
  const int64_t r = e / per;
  const int c0 = (int)(e - r * per) * 8;
  const int64_t rs = reverse ? rows - 1 - r : r;  // source row (reverse: output row r holds row rows-1-r)
  uint32_t pk[3][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + 2 * j;
    const float x0 = c < cols ? A[rs * lda + c] : 0.f, x1 = c + 1 < cols ? A[rs * lda + c + 1] : 0.f;
    uint32_t t[3];
    bf6::split3x2(x0, x1, t);
    pk[0][j] = t[0];
    pk[1][j] = t[1];
    pk[2][j] = t[2];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q)
    *reinterpret_cast<uint4*>(out + ((int64_t)q * rows + r) * ld + c0) = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
}

// Three bfloat16 planes of the lower-triangular inverse factor L^-1 (s x s)
// from the FP64 factorisation buffer: appended row k holds (L^-T)[k][.], so
// (L^-1)[i][k] = E[k][i] with E = buf + npad * npad (leading dimension npad).
// Plane q at rows [q rows, q rows + rows) (rows >= s), ld >= s columns; zero
// outside the s x s matrix.  The pieces are taken from the FP64 value.
__global__ void k_linv_bf3(const double* __restrict__ buf, int64_t npad, int s, int rows, int ld,
                           uint16_t* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * ld) return;
  const int i = (int)(e / ld), k = (int)(e % ld);
  const double x = (i < s && k < s) ? buf[(npad + k) * npad + i] : 0.0;
  const float h1 = __uint_as_float(bf6::bf16x2_rn((float)x, 0.f) << 16);
  const double r1 = x - (double)h1;
  const float h2 = __uint_as_float(bf6::bf16x2_rn((float)r1, 0.f) << 16);
  const double r2 = r1 - (double)h2;
  const float h3 = __uint_as_float(bf6::bf16x2_rn((float)r2, 0.f) << 16);
  const float hh[3] = {h1, h2, h3};
#pragma unroll
  for (int q = 0; q < 3; ++q) out[((int64_t)q * rows + i) * ld + k] = (uint16_t)(__float_as_uint(hh[q]) >> 16);
}

// Block-part summary rows of the owned windows in three bfloat16 planes for
// k_gram_bf6: window wi's extra rows e < se = s + 1, columns [nB, n) (its
// [z_m | Z_m]^T, Definition 1 whitened) go to row wi se + e of each plane,
// columns [0, n - nB), row length kmax (a multiple of 64, zero pad); plane q
// at rows [q nown se, (q + 1) nown se).  Block (x, window y): rows
// e = 4 x + threadIdx.y, eight values per thread and step.
__global__ void k_split_summary_bf3(const Win* __restrict__ wins, const float* __restrict__ buf, int se, int nown,
                                    int kmax, uint16_t* __restrict__ out) {
  const Win w = wins[blockIdx.y];
  const int e = blockIdx.x * blockDim.y + threadIdx.y;
  if (e >= se) return;
  const int nb = w.n - w.nB;
  const float* src = buf + w.base + (int64_t)(w.npad + e) * w.npad + w.nB;
  const int64_t row = (int64_t)blockIdx.y * se + e, plane = (int64_t)nown * se;
  for (int j = 8 * threadIdx.x; j < kmax; j += 8 * blockDim.x) {
    uint32_t pk[3][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = j + 2 * q;
      const float x0 = c < nb ? src[c] : 0.f, x1 = c + 1 < nb ? src[c + 1] : 0.f;
      uint32_t t[3];
      bf6::split3x2(x0, x1, t);
      pk[0][q] = t[0];
      pk[1][q] = t[1];
      pk[2][q] = t[2];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
      *reinterpret_cast<uint4*>(out + (q * plane + row) * kmax + j) = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
  }
}

// Gram of the local summaries on the tensor cores (mixed form), bf16x6
// products, one persistent CTA per SM: item t = (128 x 128 tile (I, J) of
// the lower triangle of G, window group g) adds sum over the windows of group
// g of [z_m | Z_m]^T [z_m | Z_m] with K running window by window (kmax / 64
// chunks each); the chunks are added with TwoSum and the item's sum goes to
// its group's FP64 partial (k_gram_reduce adds the groups in order).  sb:
// tensor map of the three planes of k_split_summary_bf3 (srows rows each).
__global__ void __launch_bounds__(bf6::NTHR, 1) k_gram_bf6(const int2* __restrict__ tiles, int ntile, int nwin,
                                                           int group, int se, int kmax,
                                                           const __grid_constant__ CUtensorMap sb, int srows,
                                                           double* __restrict__ partial, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  bf6::Smem& sm = bf6::smem_of(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bf6::setup(sm);
  const int cpw = kmax / bf6::KC;
  const int ngroup = (nwin + group - 1) / group;
  const int nitems = ntile * ngroup;
  auto order = [&](int k) -> int {
    const int64_t t = blockIdx.x + (int64_t)k * gridDim.x;
    return t < nitems ? (int)t : -1;
  };
  auto chunks = [&](int t) {
    const int g = t / ntile;
    return (min(nwin, (g + 1) * group) - g * group) * cpw;
  };
  auto coords = [&](int t) -> int4 {
    const int2 tl = tiles[t % ntile];
    return make_int4(tl.x * 128, tl.y * 128, (t / ntile) * group, 0);
  };
  auto at = [&](int4 b, int c) {
    const int wi = b.z + c / cpw;
    return make_int3(bf6::KC * (c % cpw), wi * se + b.x, wi * se + b.y);
  };
  auto after = [&](int t, float(&hi)[32], float(&lo)[32]) {
    const int2 tl = tiles[t % ntile];
    const int q = warp & 3, half = warp >> 2;
    const int e1 = tl.x * 128 + q * 32 + lane;
    const int cg = tl.y * 128 + half * 32;
    if (e1 >= se) return;
    double* P = partial + (int64_t)(t / ntile) * se * se + (int64_t)e1 * se;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (cg + j < se) P[cg + j] = (double)hi[j] + (double)lo[j];
  };
  const bool ok = bf6::persistent_comp(sm, &sb, srows, &sb, srows, order, chunks, coords, at, after);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  bf6::teardown(sm);
}

// Residual tiles on the tensor cores with bf16x6 products (mixed form), one
// persistent CTA per SM walking the item list: item (window, I, J) is rows
// [128 I, 128 I + 128) x columns [128 J, 128 J + 128) of the window's
// R = K + sigma_n^2 I - Vt Vt^T, blanket-first, with the Vt Vt^T sum over
// s (kc chunks of 64) added with TwoSum.  vb: tensor map of the three
// bfloat16 planes of V in reversed point order (row nrev - 1 - p holds point
// p), nrev rows per plane.  Rows and columns past the window's order read
// other points' rows or zeros: the epilogue writes the identity there.
template <int D>
__global__ void __launch_bounds__(bf6::NTHR, 1) k_resid_bf6(const int4* __restrict__ items, int nitems,
                                                            const Win* __restrict__ wins, const float* __restrict__ xs,
                                                            int d, const __grid_constant__ CUtensorMap vb, int nrev,
                                                            int kc, float ss2, float sn2, float* __restrict__ buf,
                                                            int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  bf6::Smem& sm = bf6::smem_of(smraw);
  __shared__ __align__(16) float xc[128][D];  // scaled inputs of the tile's columns, zero-padded
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  bf6::setup(sm);
  auto order = [&](int k) -> int {
    const int64_t t = blockIdx.x + (int64_t)k * gridDim.x;
    return t < nitems ? (int)t : -1;
  };
  auto chunks = [&](int) { return kc; };
  auto coords = [&](int t) -> int4 {
    const int4 it = items[t];
    const int base = nrev - (int)wins[it.x].g_end;
    return make_int4(base + it.y * 128, base + it.z * 128, 0, 0);
  };
  auto at = [](int4 b, int c) { return make_int3(bf6::KC * c, b.x, b.y); };
  auto after = [&](int t, float(&hi)[32], float(&lo)[32]) {
    const int4 it = items[t];
    const Win w = wins[it.x];
    const int r0 = it.y * 128, c0 = it.z * 128;
    worker_sync_and(true);  // every worker is done with the previous tile's columns
    for (int e = tid; e < 128 * D; e += bf6::NWK * 32) {
      const int r = e / D, q = e % D;
      xc[r][q] = (c0 + r < w.n && q < d) ? xs[(w.g_end - 1 - (c0 + r)) * d + q] : 0.f;
    }
    worker_sync_and(true);
    const int q = warp & 3, half = warp >> 2;
    const int i = r0 + q * 32 + lane;
    const int cg = c0 + half * 32;
    if (i >= w.npad || cg >= w.npad) return;
    float xr[D];
#pragma unroll
    for (int t2 = 0; t2 < D; ++t2) xr[t2] = (i < w.n && t2 < d) ? xs[(w.g_end - 1 - i) * d + t2] : 0.f;
    float* dst = buf + w.base + (int64_t)i * w.npad + cg;
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
      float out[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = 4 * j4 + k, cl = half * 32 + j, jj = c0 + cl;
        float v;
        if (i < w.n && jj < w.n) {
          const float d2 = dist2<D>(xr, xc[cl]);
          v = (ss2 * expf(-0.5f * d2) - hi[j]) - lo[j];
          if (i == jj) v += sn2;
        } else {
          v = (i == jj) ? 1.f : 0.f;
        }
        out[k] = v;
      }
      *reinterpret_cast<float4*>(dst + 4 * j4) = make_float4(out[0], out[1], out[2], out[3]);
    }
  };
  const bool ok = bf6::persistent_comp(sm, &vb, nrev, &vb, nrev, order, chunks, coords, at, after);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  bf6::teardown(sm);
}

// Right-hand sides R_{u W} of the prediction (mixed form) with bf16x6
// products: item (pair, 128-row u tile, 128-column tile of the window) gives
// P[u][c] = K(x_u, x_c) - Vu[u] . Vt[c] for the pair's test rows and window
// columns (zero past the window's order).  ub / vb: three bfloat16 planes of
// the test points' V (U rows per plane) and of V in reversed point order.
template <int D>
__global__ void __launch_bounds__(bf6::NTHR, 1) k_pred_rhs_bf6(const Pair* __restrict__ pairs,
                                                               const int4* __restrict__ items, int nitems,
                                                               const Win* __restrict__ wins,
                                                               const float* __restrict__ xs,
                                                               const float* __restrict__ xu, int d,
                                                               const __grid_constant__ CUtensorMap ub, int urows,
                                                               const __grid_constant__ CUtensorMap vb, int nrev,
                                                               int kc, float ss2, float* __restrict__ P,
                                                               int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  bf6::Smem& sm = bf6::smem_of(smraw);
  __shared__ __align__(16) float xc[128][D];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  bf6::setup(sm);
  auto order = [&](int k) -> int {
    const int64_t t = blockIdx.x + (int64_t)k * gridDim.x;
    return t < nitems ? (int)t : -1;
  };
  auto chunks = [&](int) { return kc; };
  auto coords = [&](int t) -> int4 {
    const int4 it = items[t];
    const Pair pr = pairs[it.x];
    return make_int4(pr.u0 + it.y * 128, nrev - (int)wins[pr.win].g_end + it.z * 128, 0, 0);
  };
  auto at = [](int4 b, int c) { return make_int3(bf6::KC * c, b.x, b.y); };
  auto after = [&](int t, float(&hi)[32], float(&lo)[32]) {
    const int4 it = items[t];
    const Pair pr = pairs[it.x];
    const Win w = wins[pr.win];
    const int u0 = it.y * 128, c0 = it.z * 128;
    worker_sync_and(true);
    for (int e = tid; e < 128 * D; e += bf6::NWK * 32) {
      const int r = e / D, q = e % D;
      xc[r][q] = (c0 + r < w.n && q < d) ? xs[(w.g_end - 1 - (c0 + r)) * d + q] : 0.f;
    }
    worker_sync_and(true);
    const int q = warp & 3, half = warp >> 2;
    const int uu = u0 + q * 32 + lane;
    const int cg = c0 + half * 32;
    if (uu >= pr.nu || cg >= w.npad) return;
    float xr[D];
#pragma unroll
    for (int t2 = 0; t2 < D; ++t2) xr[t2] = t2 < d ? xu[(int64_t)(pr.u0 + uu) * d + t2] : 0.f;
    float* dst = P + pr.pbase + (int64_t)uu * w.npad + cg;
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
      float out[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = 4 * j4 + k, cl = half * 32 + j;
        float v = 0.f;
        if (c0 + cl < w.n) {
          const float d2 = dist2<D>(xr, xc[cl]);
          v = (ss2 * expf(-0.5f * d2) - hi[j]) - lo[j];
        }
        out[k] = v;
      }
      *reinterpret_cast<float4*>(dst + 4 * j4) = make_float4(out[0], out[1], out[2], out[3]);
    }
  };
  const bool ok = bf6::persistent_comp(sm, &ub, urows, &vb, nrev, order, chunks, coords, at, after);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  bf6::teardown(sm);
}

// Out[p][i] = sum_{k <= i} A[p][k] Binv[i][k] for p < nrows, i < s (a
// triangular right factor: K runs to min(s, i0 + 128) for the 128-column
// tile at i0), A and Binv given as three bfloat16 planes behind the tensor
// maps amap (arows rows per plane) and bmap (brows rows per plane), 64 x 128
// boxes, 128-byte swizzle; Out FP32 with leading dimension ldo.  Item t =
// (128-row tile t / nct, 128-column tile t mod nct): the tiles of one row
// block are consecutive, so the CTAs working on them at the same time share
// its A boxes through L2.
__global__ void __launch_bounds__(bf6::NTHR, 1) k_proj_tc(const __grid_constant__ CUtensorMap amap, int arows,
                                                          const __grid_constant__ CUtensorMap bmap, int brows,
                                                          int64_t nrows, int s, float* __restrict__ out, int64_t ldo,
                                                          int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  bf6::Smem& sm = bf6::smem_of(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bf6::setup(sm);
  const int nct = (s + 127) / 128;
  const int64_t nrt = (nrows + 127) / 128;
  const int ntiles = (int)(nrt * nct);
  auto chunks = [&](int t) { return (min(s, (t % nct) * 128 + 128) + bf6::KC - 1) / bf6::KC; };
  auto coords = [&](int t) -> int4 { return make_int4((t / nct) * 128, (t % nct) * 128, 0, 0); };
  auto at = [](int4 b, int c) { return make_int3(bf6::KC * c, b.x, b.y); };
  auto after = [&](int t, float(&acc)[32]) {
    const int q = warp & 3, half = warp >> 2;
    const int64_t row = (int64_t)(t / nct) * 128 + q * 32 + lane;
    const int c0 = (t % nct) * 128 + half * 32;
    if (row >= nrows || c0 >= s) return;
    float* dst = out + row * ldo + c0;
    if (c0 + 32 <= s && (ldo & 3) == 0) {
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4)
        *reinterpret_cast<float4*>(dst + 4 * j4) = make_float4(acc[4 * j4], acc[4 * j4 + 1], acc[4 * j4 + 2], acc[4 * j4 + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < s) dst[j] = acc[j];
    }
  };
  // Tile order: with an even number of column tiles, the CTA's tiles come in
  // pairs (column tile j, column tile nct - 1 - j) of one row block, which
  // have the same number of K chunks together (the product is triangular),
  // so all CTAs advance at the same rate and those working at the same time
  // share a few row blocks' A boxes in L2.
  auto order = [&](int k) -> int {
    if (nct & 1) {
      const int64_t t = blockIdx.x + (int64_t)k * gridDim.x;
      return t < ntiles ? (int)t : -1;
    }
    const int P = nct / 2;
    const int64_t u = blockIdx.x + (int64_t)(k >> 1) * gridDim.x;
    if (u >= nrt * P) return -1;
    const int pt = (int)(u / P), j = (int)(u % P);
    return pt * nct + ((k & 1) ? nct - 1 - j : j);
  };
  const bool ok = bf6::persistent(sm, &amap, arows, &bmap, brows, order, chunks, coords, at, after);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  bf6::teardown(sm);
}

}  // namespace lma
