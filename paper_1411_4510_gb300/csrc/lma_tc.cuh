// 5th-generation tensor-core (tcgen05) building blocks for sm_103a, written
// as inline PTX: tensor-memory allocation and loads, shared-memory matrix
// descriptors (K-major, 128-byte swizzle), the TF32 MMA and mbarrier waits
// with an iteration limit.
//
// FP32 operands are used as a 3-term TF32 split: x = hi + lo with hi the
// TF32 rounding of x; a.b ~ hi_a hi_b + hi_a lo_b + lo_a hi_b accumulated in
// FP32 tensor memory (the published "3xTF32" technique), which keeps about
// 22 bits of every product.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lma {
namespace tc {

constexpr uint32_t kSpinLimit = 1u << 22;   // iterations before a wait gives up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier --------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// ---- TMA ---------------------------------------------------------------------
// 2-D tiled load of the box at (x = column, y = row) of `map` into shared
// memory; completion is counted in bytes on *bar.  x * 4 bytes must be a
// multiple of 16; y may be negative or past the end (those rows read zero).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// ---- fences ----------------------------------------------------------------
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- tensor memory ---------------------------------------------------------
// whole warp; the allocated column base is written to *dst (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns (lane = warp quadrant * 32 + laneid)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- descriptors -----------------------------------------------------------
// K-major operand tile in shared memory with the 128-byte swizzle: rows of
// 128 bytes (32 FP32/TF32 values of K), 8-row atoms 1024 bytes apart; the
// tile base must be 1024-byte aligned.  Advancing K by 8 TF32 values inside
// the atom advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // [0,14)  start address >> 4
  d |= (uint64_t)1 << 16;                             // [16,30) leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                   // [32,46) stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                             // [46,49) fixed 0b001
  d |= (uint64_t)2 << 61;                             // [61,64) 128-byte swizzle
  return d;
}
// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t M, uint32_t N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
// byte offset of element (row, k) (k < 32) in a 128B-swizzled K-major tile
__device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t k) {
  return row * 128u + ((((k >> 2) ^ (row & 7u)) & 7u) << 4) + (k & 3u) * 4u;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on *bar once every previously issued MMA of this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// TF32 rounding (nearest, ties away) of an FP32 value; the result keeps the
// FP32 encoding with the 13 low mantissa bits cleared.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tc
}  // namespace lma

namespace lma {
namespace tc {

// Shared-memory stage of a 128 x BN tile product over 32 values of K:
// TF32 hi/lo halves of both operands, each 128B-swizzled and 1024-aligned.
template <int BN>
struct alignas(1024) TcStage {
  float a_hi[128 * 32];
  float a_lo[128 * 32];
  float b_hi[BN * 32];
  float b_lo[BN * 32];
};
template <int BN>
struct TcSmem {
  TcStage<BN> st[2];
  uint64_t bar[2];
  uint32_t tmem;
};
constexpr size_t kTcAlignSlack = 1024;

template <int BN>
__device__ __forceinline__ TcSmem<BN>& tc_smem(unsigned char* raw) {
  uintptr_t p = reinterpret_cast<uintptr_t>(raw);
  p = (p + 1023) & ~uintptr_t(1023);
  return *reinterpret_cast<TcSmem<BN>*>(p);
}

// Split a float4 of K-consecutive values into TF32 hi/lo and store both at
// (row, k..k+3) of a swizzled tile.
// The remainder is rounded to TF32 as well: the MMA would otherwise read
// its FP32 encoding truncated, a one-sided error of up to 2^-23 |x|.
__device__ __forceinline__ void store_split4(float* hi, float* lo, uint32_t row, uint32_t k, float4 v) {
  float4 h, l;
  h.x = tf32_round(v.x); l.x = tf32_round(v.x - h.x);
  h.y = tf32_round(v.y); l.y = tf32_round(v.y - h.y);
  h.z = tf32_round(v.z); l.z = tf32_round(v.z - h.z);
  h.w = tf32_round(v.w); l.w = tf32_round(v.w - h.w);
  const uint32_t off = sw128_offset(row, k) >> 2;
  *reinterpret_cast<float4*>(hi + off) = h;
  *reinterpret_cast<float4*>(lo + off) = l;
}

}  // namespace tc

// Self-check kernel: C[M x N] = A[M x K] B[N x K]^T (row-major FP32, K % 32 == 0,
// lda/ldb % 4 == 0), one CTA per 128 x BN output tile, 3xTF32 on tcgen05.
template <int BN>
__global__ void __launch_bounds__(256) k_tc_gemm(const float* __restrict__ A, int64_t lda,
                                                 const float* __restrict__ Bm, int64_t ldb, float* __restrict__ C,
                                                 int64_t ldc, int M, int N, int K, int* __restrict__ err) {
  using namespace tc;
  extern __shared__ __align__(16) unsigned char smraw[];
  TcSmem<BN>& sm = tc_smem<BN>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * BN;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&sm.tmem, BN < 32 ? 32 : BN);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = sm.tmem;
  const uint32_t idesc = idesc_tf32(128, BN);
  const int nchunk = K / 32;
  bool ok = true;
  for (int c = 0; c < nchunk; ++c) {
    const int s = c & 1;
    if (c >= 2) {
      // every thread waits (bounded), then all agree on the outcome
      const bool w = mbar_wait(&sm.bar[s], ((c >> 1) - 1) & 1);
      ok = __syncthreads_and(w) != 0;
      if (!ok) break;
    }
    TcStage<BN>& S = sm.st[s];
    const int k0 = c * 32;
    for (int i = tid; i < 128 * 8; i += 256) {
      const int row = i >> 3, c4 = i & 7;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m0 + row < M) v = *reinterpret_cast<const float4*>(A + (int64_t)(m0 + row) * lda + k0 + c4 * 4);
      store_split4(S.a_hi, S.a_lo, row, c4 * 4, v);
    }
    for (int i = tid; i < BN * 8; i += 256) {
      const int row = i >> 3, c4 = i & 7;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (n0 + row < N) v = *reinterpret_cast<const float4*>(Bm + (int64_t)(n0 + row) * ldb + k0 + c4 * 4);
      store_split4(S.b_hi, S.b_lo, row, c4 * 4, v);
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid < 32) {
      if (tid == 0) {
        const uint32_t ah = smem_addr(S.a_hi), al = smem_addr(S.a_lo);
        const uint32_t bh = smem_addr(S.b_hi), bl = smem_addr(S.b_lo);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t o = ks * 32;
          mma_tf32(tmem, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, (c > 0 || ks > 0) ? 1u : 0u);
          mma_tf32(tmem, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
          mma_tf32(tmem, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
        }
        mma_commit(&sm.bar[s]);
      }
      __syncwarp();  // lanes 1-31 wait here, so no divergent wait stalls the issuing lane
    }
  }
  if (ok && nchunk > 0) {
    const bool w = mbar_wait(&sm.bar[(nchunk - 1) & 1], ((nchunk - 1) >> 1) & 1);
    ok = __syncthreads_and(w) != 0;
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  fence_after_sync();
  if (ok) {
    const int q = warp & 3, half = warp >> 2;
    const int row = m0 + q * 32 + (tid & 31);
    for (int cb = half * (BN / 2); cb < (half + 1) * (BN / 2); cb += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + cb, v);
      if (row < M)
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (n0 + cb + j < N) C[(int64_t)row * ldc + n0 + cb + j] = v[j];
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN < 32 ? 32 : BN);
}

}  // namespace lma

namespace lma {
namespace tc {

// Completion bookkeeping of the two stage barriers (identical in every thread).
struct TcPipe {
  uint32_t cnt[2] = {0, 0};      // commits issued on each barrier
  bool pending[2] = {false, false};
};

// Collective, bounded wait for the most recent commit on stage s.
template <int BN>
__device__ __forceinline__ bool tc_drain(TcSmem<BN>& sm, TcPipe& p, int s) {
  if (!p.pending[s]) return true;
  const bool w = mbar_wait(&sm.bar[s], (p.cnt[s] - 1u) & 1u);
  p.pending[s] = false;
  return __syncthreads_and(w) != 0;
}

// D (tensor memory, 128 lanes x BN FP32 columns) = sum_{k<K} A(r,k) B(c,k),
// r < 128, c < BN, K % 32 == 0.  rowA(r) / rowB(c) return a 16-byte-aligned
// pointer to the K values of that row, or nullptr for a zero row.  All 256
// threads call it; returns false (in every thread) if a wait timed out.
//
// The global loads of a 32-wide K chunk are issued DEPTH chunks ahead into
// a register ring (DEPTH x 24 KB per CTA for BN = 64), so with two CTAs per
// SM several chunks are in flight while the current one is split into TF32
// hi/lo, stored to the swizzled stage and multiplied.
template <int BN, int DEPTH = 3, bool CGB = false, class RA, class RB>
__device__ bool tile_product(TcSmem<BN>& sm, TcPipe& p, uint32_t tmem, int K, RA rowA, RB rowB, int nacc = 1) {
  constexpr int NA = 128 * 8 / 256;          // float4 of A per thread per chunk
  constexpr int NB = (BN * 8 + 255) / 256;   // float4 of B per thread per chunk
  const int tid = threadIdx.x;
  const uint32_t idesc = idesc_tf32(128, BN);
  const int nchunk = K / 32;
  float4 ra[DEPTH][NA], rb[DEPTH][NB];
  auto load = [&](int c, float4 (&xa)[NA], float4 (&xb)[NB]) {
    const int k0 = c * 32;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int i = tid + 256 * j, row = i >> 3, c4 = i & 7;
      const float* src = rowA(row);
      xa[j] = src ? *reinterpret_cast<const float4*>(src + k0 + c4 * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int i = tid + 256 * j, row = i >> 3, c4 = i & 7;
      const float* src = (i < BN * 8) ? rowB(row) : nullptr;
      if (CGB)  // B written by another CTA of this launch: read it from L2
        xb[j] = src ? __ldcg(reinterpret_cast<const float4*>(src + k0 + c4 * 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
      else
        xb[j] = src ? *reinterpret_cast<const float4*>(src + k0 + c4 * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
#pragma unroll
  for (int d = 0; d < DEPTH; ++d)
    if (d < nchunk) load(d, ra[d], rb[d]);
  for (int cb = 0; cb < nchunk; cb += DEPTH) {
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) {
      const int c = cb + d;
      if (c >= nchunk) break;
      const int s = c & 1;
      if (!tc_drain(sm, p, s)) return false;
      TcStage<BN>& S = sm.st[s];
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int i = tid + 256 * j;
        store_split4(S.a_hi, S.a_lo, i >> 3, (i & 7) * 4, ra[d][j]);
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int i = tid + 256 * j;
        if (i < BN * 8) store_split4(S.b_hi, S.b_lo, i >> 3, (i & 7) * 4, rb[d][j]);
      }
      if (c + DEPTH < nchunk) load(c + DEPTH, ra[d], rb[d]);
      fence_async_smem();
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (tid < 32) {
        if (tid == 0) {
          const uint32_t ah = smem_addr(S.a_hi), al = smem_addr(S.a_lo);
          const uint32_t bh = smem_addr(S.b_hi), bl = smem_addr(S.b_lo);
          // split-K: chunk c accumulates into accumulator c mod nacc (columns
          // [BN a, BN a + BN)); accumulators 0 .. min(nacc, nchunk) - 1 are written
          const int a = c % nacc;
          const bool first = c < nacc;
          const uint32_t dd = tmem + (uint32_t)(BN * a);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t o = ks * 32;
            mma_tf32(dd, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, (!first || ks > 0) ? 1u : 0u);
            mma_tf32(dd, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
            mma_tf32(dd, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
          }
          mma_commit(&sm.bar[s]);
        }
        __syncwarp();  // lanes 1-31 wait here, so no divergent wait stalls the issuing lane
      }
      p.cnt[s] += 1;
      p.pending[s] = true;
    }
  }
  bool ok = tc_drain(sm, p, 0);
  ok = tc_drain(sm, p, 1) && ok;
  fence_after_sync();
  return ok;
}

// Four consecutive floats from p with at most lim of them valid (the rest
// zero); one 16-byte load when p is aligned and all four are valid.
__device__ __forceinline__ float4 load4_lim(const float* p, int lim) {
  if (!p || lim <= 0) return make_float4(0.f, 0.f, 0.f, 0.f);
  if (lim >= 4 && (reinterpret_cast<uintptr_t>(p) & 15u) == 0) return *reinterpret_cast<const float4*>(p);
  float4 v;
  v.x = p[0];
  v.y = lim > 1 ? p[1] : 0.f;
  v.z = lim > 2 ? p[2] : 0.f;
  v.w = lim > 3 ? p[3] : 0.f;
  return v;
}

// TF32 hi/lo of one value into (row, k) of a swizzled stage.
__device__ __forceinline__ void store_split1(float* hi, float* lo, uint32_t row, uint32_t k, float x) {
  const float h = tf32_round(x);
  const uint32_t off = sw128_offset(row, k) >> 2;
  hi[off] = h;
  lo[off] = tf32_round(x - h);
}

// tile_product with either operand optionally supplied transposed.
//   TA = false: rowA(r) -> the K values of row r of A (16-byte aligned) or nullptr;
//   TA = true:  rowA(k) -> the values A(0 .. 127, k), contiguous, or nullptr
//               (k in [0, ceil32(K)); only the first alim are read).
// The same for B with BN rows (TB, blim).  negB: B enters negated.  acc0:
// add to the accumulator instead of overwriting it with the first chunk.
// A transposed chunk (32 values of K x 128 rows) is read by lane = k, so a
// warp's shared-memory stores fill one 128-byte row of the swizzled stage
// (conflict-free) while its global loads take 16 bytes from each of 32 rows.
template <int BN, bool TA, bool TB, int DEPTH = 2, class RA, class RB>
__device__ bool tile_product2(TcSmem<BN>& sm, TcPipe& p, uint32_t tmem, int K, RA rowA, RB rowB, int alim, int blim,
                              bool negB, bool acc0) {
  constexpr int NA = 128 * 8 / 256;
  constexpr int NB = (BN * 8 + 255) / 256;
  const int tid = threadIdx.x;
  const uint32_t idesc = idesc_tf32(128, BN);
  const int nchunk = (K + 31) / 32;
  float4 ra[DEPTH][NA], rb[DEPTH][NB];
  auto load = [&](int c, float4 (&xa)[NA], float4 (&xb)[NB]) {
    const int kc = c * 32;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int i = tid + 256 * j;
      if (TA) {
        const int kk = i & 31, r4 = i >> 5;
        const float* src = rowA(kc + kk);
        xa[j] = load4_lim(src ? src + r4 * 4 : nullptr, alim - r4 * 4);
      } else {
        const float* src = rowA(i >> 3);
        xa[j] = src ? *reinterpret_cast<const float4*>(src + kc + (i & 7) * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int i = tid + 256 * j;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < BN * 8) {
        if (TB) {
          const int kk = i & 31, c4 = i >> 5;
          const float* src = rowB(kc + kk);
          v = load4_lim(src ? src + c4 * 4 : nullptr, blim - c4 * 4);
        } else {
          const float* src = rowB(i >> 3);
          if (src) v = *reinterpret_cast<const float4*>(src + kc + (i & 7) * 4);
        }
      }
      if (negB) v = make_float4(-v.x, -v.y, -v.z, -v.w);
      xb[j] = v;
    }
  };
#pragma unroll
  for (int d = 0; d < DEPTH; ++d)
    if (d < nchunk) load(d, ra[d], rb[d]);
  for (int cb = 0; cb < nchunk; cb += DEPTH) {
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) {
      const int c = cb + d;
      if (c >= nchunk) break;
      const int s = c & 1;
      if (!tc_drain(sm, p, s)) return false;
      TcStage<BN>& S = sm.st[s];
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int i = tid + 256 * j;
        if (TA) {
          const int kk = i & 31, r = (i >> 5) * 4;
          store_split1(S.a_hi, S.a_lo, r + 0, kk, ra[d][j].x);
          store_split1(S.a_hi, S.a_lo, r + 1, kk, ra[d][j].y);
          store_split1(S.a_hi, S.a_lo, r + 2, kk, ra[d][j].z);
          store_split1(S.a_hi, S.a_lo, r + 3, kk, ra[d][j].w);
        } else {
          store_split4(S.a_hi, S.a_lo, i >> 3, (i & 7) * 4, ra[d][j]);
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int i = tid + 256 * j;
        if (i >= BN * 8) continue;
        if (TB) {
          const int kk = i & 31, r = (i >> 5) * 4;
          store_split1(S.b_hi, S.b_lo, r + 0, kk, rb[d][j].x);
          store_split1(S.b_hi, S.b_lo, r + 1, kk, rb[d][j].y);
          store_split1(S.b_hi, S.b_lo, r + 2, kk, rb[d][j].z);
          store_split1(S.b_hi, S.b_lo, r + 3, kk, rb[d][j].w);
        } else {
          store_split4(S.b_hi, S.b_lo, i >> 3, (i & 7) * 4, rb[d][j]);
        }
      }
      if (c + DEPTH < nchunk) load(c + DEPTH, ra[d], rb[d]);
      fence_async_smem();
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (tid < 32) {
        if (tid == 0) {
          const uint32_t ah = smem_addr(S.a_hi), al = smem_addr(S.a_lo);
          const uint32_t bh = smem_addr(S.b_hi), bl = smem_addr(S.b_lo);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t o = ks * 32;
            mma_tf32(tmem, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, (acc0 || c > 0 || ks > 0) ? 1u : 0u);
            mma_tf32(tmem, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
            mma_tf32(tmem, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
          }
          mma_commit(&sm.bar[s]);
        }
        __syncwarp();
      }
      p.cnt[s] += 1;
      p.pending[s] = true;
    }
  }
  bool ok = tc_drain(sm, p, 0);
  ok = tc_drain(sm, p, 1) && ok;
  fence_after_sync();
  return ok;
}

}  // namespace tc
}  // namespace lma

namespace lma {

// Sweep update of column panel kp on the tensor cores (mixed form).  CTA
// (window x, row tile y) owns rows [k0 + 128 y, k0 + 128 y + 128) of the
// window buffer: T = A_{rows, panel} - A_{rows, kb:k0} A_{panel, kb:k0}^T with
// the product on tcgen05 (3xTF32); columns [0, kb) were applied by the
// super-panel update (kb = 0 without one).  The diagonal 64x64 block (first
// rows of y = 0) is factorised in shared memory; every other row keeps T.
// The mixed sweep launches it for the row tile holding the diagonal block
// only (y = 0, K = 0: the first panel of a 128-column group); the rows
// below are solved by k_chol_panel2_tc.
__global__ void __launch_bounds__(256, 2) k_chol_step_tc(const Win* __restrict__ wins, float* __restrict__ buf,
                                                      float* __restrict__ dinv, int* __restrict__ info, int kp,
                                                      int kb, int* __restrict__ err) {
  grid_dep_wait();
  grid_dep_launch();
  using namespace tc;
  const Win w = wins[blockIdx.x];
  const int k0 = kp * TB;
  if (k0 >= w.npad) return;
  const int r0 = k0 + blockIdx.y * 128;
  if (r0 >= w.rows) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  TcSmem<64>& sm = tc_smem<64>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* A = buf + w.base;
  const int64_t ld = w.npad;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&sm.tmem, 64);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = sm.tmem;
  TcPipe pipe;
  bool ok = true;
  const int K = k0 - kb;
  if (K > 0) {
    auto rowA = [&](int r) -> const float* {
      const int row = r0 + r;
      return row < w.rows ? A + (int64_t)row * ld + kb : nullptr;
    };
    auto rowB = [&](int c) -> const float* { return A + (int64_t)(k0 + c) * ld + kb; };
    ok = tile_product<64>(sm, pipe, tmem, K, rowA, rowB);
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  const int q = warp & 3, half = warp >> 2;
  const int rl = q * 32 + lane;
  const int row = r0 + rl;
  float v[32];
  if (K > 0 && ok) {
    float t[16];
    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + half * 32, t);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = t[j];
    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + half * 32 + 16, t);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[16 + j] = t[j];
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = 0.f;
  }
  // all MMAs have completed (tile_product drained both stages): stage memory is free
  float* scratch = reinterpret_cast<float*>(&sm.st[0]);
  float(*Dm)[TB + 1] = reinterpret_cast<float(*)[TB + 1]>(scratch);
  const bool diag = (blockIdx.y == 0) && (rl < TB);
  if (row < w.rows) {
    float* dst = A + (int64_t)row * ld + k0 + half * 32;
    float4 av[8];  // all loads first: they are independent of the stores below
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) av[j4] = *reinterpret_cast<const float4*>(dst + 4 * j4);
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
      float4 a = av[j4];
      a.x -= v[4 * j4 + 0];
      a.y -= v[4 * j4 + 1];
      a.z -= v[4 * j4 + 2];
      a.w -= v[4 * j4 + 3];
      if (diag) {
        float* d = &Dm[rl][half * 32 + 4 * j4];
        d[0] = a.x;
        d[1] = a.y;
        d[2] = a.z;
        d[3] = a.w;
      } else {
        *reinterpret_cast<float4*>(dst + 4 * j4) = a;
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 64);
  if (blockIdx.y == 0)
    diag_factor<float>(Dm, A + (int64_t)k0 * ld + k0, ld, dinv + w.dinv + (int64_t)kp * TB * TB, info + blockIdx.x,
                       k0);
}

}  // namespace lma

namespace lma {
namespace tc {

// Warp-specialised tile product over a 128 x BN output tile: kWsProducers
// warps load 32-wide K chunks (two chunks ahead, in registers), split them
// into TF32 hi/lo and store them into an NS-stage ring; one thread of the
// last warp issues the MMAs of a stage as soon as its producers have
// arrived on full[s] and frees the stage with tcgen05.commit on empty[s].
// A kind::tf32 MMA instruction occupies the tensor pipe for the same time
// whatever its N up to 256, so wide tiles (BN = 256) are the efficient ones.
constexpr int kWsProducers = 8;
constexpr int kWsDepth = 2;  // K chunks each producer keeps in flight in registers (16 producers with 3 in flight ran 1.4x slower)
constexpr int kWsThreads = 32 * (kWsProducers + 1);

template <int NS, int BN>
struct WsSmem {
  TcStage<BN> st[NS];
  uint64_t full[NS], empty[NS], done;
  uint32_t tmem;
  int abort;
};

template <int NS, int BN>
__device__ __forceinline__ WsSmem<NS, BN>& ws_smem(unsigned char* raw) {
  uintptr_t p = reinterpret_cast<uintptr_t>(raw);
  p = (p + 1023) & ~uintptr_t(1023);
  return *reinterpret_cast<WsSmem<NS, BN>*>(p);
}

// Barrier set-up and tensor-memory allocation (BN columns, by the MMA warp).
template <int NS, int BN>
__device__ __forceinline__ void ws_setup(WsSmem<NS, BN>& sm) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&sm.full[s], kWsProducers);
      mbar_init(&sm.empty[s], 1);
    }
    mbar_init(&sm.done, 1);
    sm.abort = 0;
    mbar_fence_init();
  }
  if ((tid >> 5) == kWsProducers) tmem_alloc(&sm.tmem, BN);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

template <int NS, int BN>
__device__ __forceinline__ void ws_teardown(WsSmem<NS, BN>& sm) {
  fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == kWsProducers) tmem_dealloc(sm.tmem, BN);
}

// D (tensor memory, 128 lanes x BN FP32 columns) = sum_{k<K} A(r,k) B(c,k)
// (3xTF32), r < 128, c < BN, K % 32 == 0; rowA(r) / rowB(c) return a
// 16-byte-aligned pointer to the K values of that row or nullptr for a zero
// row.  Called by all kWsThreads threads; returns false (in every thread)
// when a wait timed out.  On return every MMA has completed.
template <int NS, int BN, class RA, class RB>
__device__ bool ws_product(WsSmem<NS, BN>& sm, int K, RA rowA, RB rowB) {
  constexpr int PT = 32 * kWsProducers, D = kWsDepth;
  constexpr int NA = 128 * 8 / PT, NB = BN * 8 / PT;  // float4 per producer thread per chunk
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nchunk = K / 32;
  volatile int* abort_flag = &sm.abort;
  if (warp < kWsProducers) {
    float4 ra[D][NA], rb[D][NB];
    auto load = [&](int c, float4 (&xa)[NA], float4 (&xb)[NB]) {
      const int k0 = c * 32;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int i = tid + PT * j, row = i >> 3, c4 = i & 7;
        const float* src = rowA(row);
        xa[j] = src ? *reinterpret_cast<const float4*>(src + k0 + c4 * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int i = tid + PT * j, row = i >> 3, c4 = i & 7;
        const float* src = rowB(row);
        xb[j] = src ? *reinterpret_cast<const float4*>(src + k0 + c4 * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
#pragma unroll
    for (int d = 0; d < D; ++d)
      if (d < nchunk) load(d, ra[d], rb[d]);
    bool run = true;
    for (int cb = 0; cb < nchunk && run; cb += D) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int c = cb + d;
        if (c >= nchunk || !run) break;
        const int s = c % NS, j = c / NS;
        if (c >= NS) {  // the MMAs that last read stage s have completed
          int okw = 1;
          if (lane == 0) okw = mbar_wait(&sm.empty[s], (j - 1) & 1) ? 1 : 0;
          okw = __shfl_sync(0xffffffffu, okw, 0);
          if (!okw) *abort_flag = 1;
        }
        if (*abort_flag) {
          run = false;
          break;
        }
        TcStage<BN>& S = sm.st[s];
#pragma unroll
        for (int q = 0; q < NA; ++q) {
          const int i = tid + PT * q;
          store_split4(S.a_hi, S.a_lo, i >> 3, (i & 7) * 4, ra[d][q]);
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const int i = tid + PT * q;
          store_split4(S.b_hi, S.b_lo, i >> 3, (i & 7) * 4, rb[d][q]);
        }
        if (c + D < nchunk) load(c + D, ra[d], rb[d]);
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.full[s]);
      }
    }
  } else {
    // the whole MMA warp runs this loop (a lane spinning on a barrier on a
    // divergent path would hold up the issuing lane); lane 0 issues
    const uint32_t idesc = idesc_tf32(128, BN);
    const uint32_t tmem = sm.tmem;
    for (int c = 0; c < nchunk; ++c) {
      const int s = c % NS, j = c / NS;
      if (*abort_flag) break;
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&sm.full[s], j & 1) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) {
        *abort_flag = 1;
        break;
      }
      fence_after_sync();
      if (lane == 0) {
        TcStage<BN>& S = sm.st[s];
        const uint32_t ah = smem_addr(S.a_hi), al = smem_addr(S.a_lo);
        const uint32_t bh = smem_addr(S.b_hi), bl = smem_addr(S.b_lo);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t o = ks * 32;
          mma_tf32(tmem, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, (c > 0 || ks > 0) ? 1u : 0u);
          mma_tf32(tmem, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
          mma_tf32(tmem, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
        }
        mma_commit(&sm.empty[s]);
      }
      __syncwarp();
    }
    if (lane == 0) mma_commit(&sm.done);  // arrives once every MMA issued above has completed
    __syncwarp();
  }
  const bool w = mbar_wait(&sm.done, 0);
  const bool ok = __syncthreads_and(w && !*abort_flag) != 0;
  fence_after_sync();
  return ok;
}

}  // namespace tc

// Panel-group update of the left-looking sweep (mixed form): for the BN
// columns [s0, s0 + BN) of every window (clipped to its order), every row
// r >= s0 gets A_{r,c} -= sum_{kfrom <= k < s0} L_{r,k} L_{c,k}, as one
// 128 x BN tensor-core tile per CTA (grid: x = window, y = 128-row tile).
// Only the lower triangle (c <= r) is written.  BN = 256 with kfrom = 0 is the
// super-panel update (all columns left of the super-panel); BN = 128 with
// kfrom = the super-panel's first column adds the super-panel's first 128
// columns to its last 128, so that the 64-wide panel steps only add the
// columns of their own 128-column half.
template <int BN>
__global__ void __launch_bounds__(tc::kWsThreads, 1) k_chol_wide(const Win* __restrict__ wins,
                                                                float* __restrict__ buf, int s0, int kfrom,
                                                                int* __restrict__ err) {
  grid_dep_wait();
  grid_dep_launch();
  using namespace tc;
  const Win w = wins[blockIdx.x];
  if (s0 >= w.npad) return;
  const int r0 = s0 + blockIdx.y * 128;
  if (r0 >= w.rows) return;
  const int ncol = min(BN, w.npad - s0);
  extern __shared__ __align__(16) unsigned char smraw[];
  WsSmem<2, BN>& sm = ws_smem<2, BN>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* A = buf + w.base;
  const int64_t ld = w.npad;
  ws_setup(sm);
  auto rowA = [&](int r) -> const float* {
    const int row = r0 + r;
    return row < w.rows ? A + (int64_t)row * ld + kfrom : nullptr;
  };
  auto rowB = [&](int c) -> const float* { return c < ncol ? A + (int64_t)(s0 + c) * ld + kfrom : nullptr; };
  const bool ok = ws_product(sm, s0 - kfrom, rowA, rowB);
  if (!ok && tid == 0) atomicExch(err, 1);
  if (ok && warp < kWsProducers) {
    constexpr int NPART = kWsProducers / 4, PW = BN / NPART;  // column groups of PW per producer warp
    const int q = warp & 3, part = warp >> 2;
    const int row = r0 + q * 32 + lane;
    float* dst = A + (int64_t)row * ld + s0;
    for (int g = 0; g < PW / 16; ++g) {
      const int c0 = part * PW + 16 * g;
      if (c0 >= ncol) break;  // warp-uniform
      float t[16];
      tmem_ld16(sm.tmem + ((uint32_t)(q * 32) << 16) + c0, t);
      if (row < w.rows) {
        float4 a[4];
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) a[j4] = *reinterpret_cast<const float4*>(dst + c0 + 4 * j4);
        if (s0 + c0 + 15 <= row) {
#pragma unroll
          for (int j4 = 0; j4 < 4; ++j4) {
            a[j4].x -= t[4 * j4];
            a[j4].y -= t[4 * j4 + 1];
            a[j4].z -= t[4 * j4 + 2];
            a[j4].w -= t[4 * j4 + 3];
            *reinterpret_cast<float4*>(dst + c0 + 4 * j4) = a[j4];
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (s0 + c0 + j <= row) dst[c0 + j] = reinterpret_cast<float*>(a)[j] - t[j];
        }
      }
    }
  }
  ws_teardown(sm);
}

}  // namespace lma

namespace lma {

// Update and solve of column panel kp in one pass (mixed form), for the rows
// below its diagonal block: CTA (row tile x, window y) owns rows
// [k0 + 64 + 128 x, ... + 128) and computes
//   T = A_{rows, panel} - A_{rows, kfrom:k0} A_{panel, kfrom:k0}^T   (skipped when kfrom = k0)
//   A_{rows, panel} <- T inv(L_kk)^T
// with both products on tcgen05 (3xTF32); columns [0, kfrom) were applied
// by the wider updates and inv(L_kk) is in dinv.  With `next`, row tile 0
// then also finishes panel kp + 1's diagonal block: its rows are the tile's
// first 64, whose panel-kp values it has just written, so
//   D = A_{kp+1, kp+1} - L_{kp+1, kp} L_{kp+1, kp}^T
// is the block with every column left of panel kp + 1 applied (those left of
// panel kp came from the wider updates), and the CTA factorises it into
// L_{kp+1, kp+1} and inv(L_{kp+1, kp+1}).  Row tile 0 of every window comes
// first in launch order, so the factorisations start in the first wave.
__global__ void __launch_bounds__(256, 2) k_chol_panel2_tc(const Win* __restrict__ wins, float* __restrict__ buf,
                                                        float* __restrict__ dinv, int* __restrict__ info, int kp,
                                                        int kfrom, int next, int* __restrict__ err) {
  grid_dep_wait();
  grid_dep_launch();
  using namespace tc;
  const Win w = wins[blockIdx.y];
  const int k0 = kp * TB;
  if (k0 >= w.npad) return;
  const int r0 = k0 + TB + blockIdx.x * 128;
  if (r0 >= w.rows) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  TcSmem<64>& sm = tc_smem<64>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* A = buf + w.base;
  const int64_t ld = w.npad;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&sm.tmem, 64);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = sm.tmem;
  TcPipe pipe;
  const int q = warp & 3, half = warp >> 2;
  const int rl = q * 32 + lane, row = r0 + rl;
  const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + half * 32;
  float* myrow = A + (int64_t)row * ld + k0 + half * 32;
  bool ok = true;
  const int K = k0 - kfrom;
  if (K > 0) {
    auto rowA = [&](int r) -> const float* {
      return r0 + r < w.rows ? A + (int64_t)(r0 + r) * ld + kfrom : nullptr;
    };
    auto rowB = [&](int c) -> const float* { return A + (int64_t)(k0 + c) * ld + kfrom; };
    ok = tile_product<64>(sm, pipe, tmem, K, rowA, rowB);
    if (ok) {
      float v[32], t[16];
      tmem_ld16(taddr, t);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = t[j];
      tmem_ld16(taddr + 16, t);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[16 + j] = t[j];
      if (row < w.rows) {
        float4 av[8];
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) av[j4] = *reinterpret_cast<const float4*>(myrow + 4 * j4);
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          float4 a = av[j4];
          a.x -= v[4 * j4 + 0];
          a.y -= v[4 * j4 + 1];
          a.z -= v[4 * j4 + 2];
          a.w -= v[4 * j4 + 3];
          *reinterpret_cast<float4*>(myrow + 4 * j4) = a;
        }
      }
    }
    fence_before_sync();
    __syncthreads();
  }
  if (ok) {
    const float* Dv = dinv + w.dinv + (int64_t)kp * TB * TB;
    auto rowT = [&](int r) -> const float* { return r0 + r < w.rows ? A + (int64_t)(r0 + r) * ld + k0 : nullptr; };
    auto rowD = [&](int c) -> const float* { return Dv + (int64_t)c * TB; };
    ok = tile_product<64>(sm, pipe, tmem, TB, rowT, rowD);
    if (ok) {
      float t[16];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        tmem_ld16(taddr + 16 * h, t);
        if (row < w.rows)
#pragma unroll
          for (int j4 = 0; j4 < 4; ++j4)
            *reinterpret_cast<float4*>(myrow + 16 * h + 4 * j4) =
                make_float4(t[4 * j4], t[4 * j4 + 1], t[4 * j4 + 2], t[4 * j4 + 3]);
      }
    }
    fence_before_sync();
    __syncthreads();
  }
  const bool diag = ok && next && blockIdx.x == 0 && k0 + TB < w.npad;
  if (diag) {
    // D = A_{kp+1, kp+1} - X X^T over the 64 panel-kp columns of rows [k0 + 64, k0 + 128)
    const int d0 = k0 + TB;
    auto rowX = [&](int r) -> const float* { return r < TB ? A + (int64_t)(d0 + r) * ld + k0 : nullptr; };
    auto rowY = [&](int c) -> const float* { return A + (int64_t)(d0 + c) * ld + k0; };
    ok = tile_product<64>(sm, pipe, tmem, TB, rowX, rowY);
  }
  float* scratch = reinterpret_cast<float*>(&sm.st[0]);
  float(*Dm)[TB + 1] = reinterpret_cast<float(*)[TB + 1]>(scratch);
  if (diag && ok) {
    float t[16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      tmem_ld16(taddr + 16 * h, t);  // whole warps; only rows < 64 are used
      if (rl < TB) {
        const float* src = A + (int64_t)(k0 + TB + rl) * ld + k0 + TB + half * 32 + 16 * h;
#pragma unroll
        for (int j = 0; j < 16; ++j) Dm[rl][half * 32 + 16 * h + j] = src[j] - t[j];
      }
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 64);
  if (diag && ok)
    diag_factor<float>(Dm, A + (int64_t)(k0 + TB) * ld + k0 + TB, ld, dinv + w.dinv + (int64_t)(kp + 1) * TB * TB,
                       info + blockIdx.y, k0 + TB);
}

// Forward solve of the prediction right-hand sides on the tensor cores: CTA
// (pair, 128 test rows) sweeps the window's column panels left to right,
//   T = P[:, panel] - P[:, 0:k0] L[panel, 0:k0]^T ;  P[:, panel] = T inv(L_kk)^T
// with both products on tcgen05 (3xTF32).  items: x = pair, y = 128-row tile.
__global__ void __launch_bounds__(256, 2) k_pred_sweep_tc(const Pair* __restrict__ pairs, const int2* __restrict__ items,
                                                       const Win* __restrict__ wins, const float* __restrict__ buf,
                                                       const float* __restrict__ dinv, float* __restrict__ P,
                                                       int* __restrict__ err) {
  using namespace tc;
  const int2 it = items[blockIdx.x];
  const Pair pr = pairs[it.x];
  const Win w = wins[pr.win];
  const int u0 = it.y * 128;
  extern __shared__ __align__(16) unsigned char smraw[];
  TcSmem<64>& sm = tc_smem<64>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* L = buf + w.base;
  const int64_t ld = w.npad;
  float* Pp = P + pr.pbase;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&sm.tmem, 64);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = sm.tmem;
  TcPipe pipe;
  const int q = warp & 3, half = warp >> 2;
  const int rl = q * 32 + lane;
  const bool live = (u0 + rl) < pr.nu;
  float* myrow = Pp + (int64_t)(u0 + rl) * ld;
  const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + half * 32;
  bool ok = true;
  const int npan = w.npad / TB;
  for (int kp = 0; kp < npan && ok; ++kp) {
    const int k0 = kp * TB;
    float v[32];
    if (k0 > 0) {
      auto rowA = [&](int r) -> const float* {
        return (u0 + r) < pr.nu ? Pp + (int64_t)(u0 + r) * ld : nullptr;
      };
      auto rowB = [&](int c) -> const float* { return L + (int64_t)(k0 + c) * ld; };
      ok = tile_product<64>(sm, pipe, tmem, k0, rowA, rowB);
      if (!ok) break;
      float t[16];
      tmem_ld16(taddr, t);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = t[j];
      tmem_ld16(taddr + 16, t);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[16 + j] = t[j];
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = 0.f;
    }
    if (live) {
      float* dst = myrow + k0 + half * 32;
      float4 av[8];  // all loads first: they are independent of the stores below
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
    fence_before_sync();
    __syncthreads();
    const float* Dv = dinv + w.dinv + (int64_t)kp * TB * TB;
    auto rowT = [&](int r) -> const float* { return (u0 + r) < pr.nu ? Pp + (int64_t)(u0 + r) * ld + k0 : nullptr; };
    auto rowD = [&](int c) -> const float* { return Dv + (int64_t)c * TB; };
    ok = tile_product<64>(sm, pipe, tmem, TB, rowT, rowD);
    if (!ok) break;
    float t[16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      tmem_ld16(taddr + 16 * h, t);
      if (live) {
        float* dst = myrow + k0 + half * 32 + 16 * h;
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4)
          *reinterpret_cast<float4*>(dst + 4 * j4) = make_float4(t[4 * j4], t[4 * j4 + 1], t[4 * j4 + 2], t[4 * j4 + 3]);
      }
    }
    fence_before_sync();
    __syncthreads();
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 64);
}

}  // namespace lma

namespace lma {

// Compensated tile product on the tensor cores over a 128 x BN tile:
// hi + lo = sum_{k<K} A(r,k) B(c,k) for worker thread t's row
// r = 32 (warp mod 4) + lane and its 32 columns c = 32 (warp / 4) + j.
// 4 BN worker threads (warps 0 .. BN/8 - 1) load each 32-wide K chunk one
// chunk ahead into registers, split it into TF32 hi/lo into stage c mod 2 and
// arrive on full[s]; the last warp issues the chunk's 12 MMAs into tensor-
// memory slot (c / 2) mod 2 (columns [BN slot, BN slot + BN)) and commits to
// done[s].  Before refilling stage s the workers wait for done[s] of chunk
// c - 2; when that chunk ends a pair (chunks 2p, 2p + 1) they drain the
// pair's slot into registers, adding its sums with TwoSum, so the slot is
// free before the MMAs of pair p + 2 start.  The tensor core's FP32
// accumulation is 24 MMA steps (64 values of K) deep, the cross-pair sum is
// compensated, and no CTA-wide barrier waits for the MMA issue.  (Draining
// after every chunk made the workers' TwoSum work, not the MMAs, the limit.)
template <int BN>
struct CompSmem {
  tc::TcStage<BN> st[2];
  uint64_t full[2], done[2], fin;
  uint32_t tmem;
  int abort;
};
template <int BN>
__device__ __forceinline__ CompSmem<BN>& comp_smem(unsigned char* raw) {
  uintptr_t p = reinterpret_cast<uintptr_t>(raw);
  p = (p + 1023) & ~uintptr_t(1023);
  return *reinterpret_cast<CompSmem<BN>*>(p);
}
template <int BN>
constexpr int comp_threads() { return 4 * BN + 32; }

// Barriers and tensor memory (2 BN columns, allocated by the MMA warp).
template <int BN>
__device__ __forceinline__ void comp_setup(CompSmem<BN>& sm) {
  using namespace tc;
  constexpr int NW = BN / 8;  // worker warps
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&sm.full[s], NW);
      mbar_init(&sm.done[s], 1);
    }
    mbar_init(&sm.fin, 1);
    sm.abort = 0;
    mbar_fence_init();
  }
  if ((threadIdx.x >> 5) == NW) tmem_alloc(&sm.tmem, 2 * BN);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}
template <int BN>
__device__ __forceinline__ void comp_teardown(CompSmem<BN>& sm) {
  using namespace tc;
  fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == BN / 8) tmem_dealloc(sm.tmem, 2 * BN);
}

// Chunk and call counters of a CTA's compensated products: a kernel may call
// comp_product several times (one K range each) and the barrier phases
// continue from one call to the next.
struct CompState {
  int chunks = 0;
  int calls = 0;
};

// Adds sum over k in [kbeg, kend) of A(r,k) B(c,k) to hi + lo (zeroed first
// unless ACC).  rowA(r) / rowB(c) return a 16-byte-aligned row pointer (or
// nullptr for a zero row) whose row holds at least kend rounded up to 4
// values; values outside [kbeg, kend) are masked.  MASK = false is for
// kbeg = 0 and kend a multiple of 32 (nothing to mask).  Returns false (in every
// thread) when a wait timed out.  hi / lo are only meaningful in workers.
template <int BN, bool ACC = false, bool MASK = true, class RA, class RB>
__device__ bool comp_product(CompSmem<BN>& sm, CompState& cs, int kbeg, int kend, RA rowA, RB rowB,
                             float (&hi)[32], float (&lo)[32]) {
  using namespace tc;
  constexpr int NW = BN / 8, NTHR = 4 * BN;
  constexpr int NA = 128 * 8 / NTHR, NB = BN * 8 / NTHR;  // float4 per worker per chunk
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kal = kbeg & ~3;
  const int nchunk = kend > kbeg ? (kend - kal + 31) / 32 : 0;
  const int g0 = cs.chunks;  // global index of this call's first chunk
  volatile int* abort_flag = &sm.abort;
  if (!ACC) {
#pragma unroll
    for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.f;
  }
  if (warp < NW) {
    const int q = warp & 3, half = warp >> 2;
    const uint32_t tlane = sm.tmem + ((uint32_t)(q * 32) << 16) + half * 32;
    auto wait_done = [&](int g) -> bool {  // MMAs of global chunk g have completed (warp-uniform result)
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&sm.done[g & 1], (g >> 1) & 1) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) *abort_flag = 1;
      return okw != 0;
    };
    auto drain = [&](int pair) {
      fence_after_sync();
      float t[16];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        tmem_ld16(tlane + BN * (pair & 1) + 16 * h, t);
#pragma unroll
        for (int j = 0; j < 16; ++j) two_sum(hi[16 * h + j], lo[16 * h + j], t[j]);
      }
      fence_before_sync();
    };
    float4 ra[NA], rb[NB];
    auto ld4 = [&](const float* src, int kk) -> float4 {
      if (!MASK) return src ? *reinterpret_cast<const float4*>(src + kk) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (!src || kk >= kend) return make_float4(0.f, 0.f, 0.f, 0.f);
      float4 v = *reinterpret_cast<const float4*>(src + kk);
      if (kk < kbeg || kk + 4 > kend) {
        v.x = (kk >= kbeg && kk < kend) ? v.x : 0.f;
        v.y = (kk + 1 >= kbeg && kk + 1 < kend) ? v.y : 0.f;
        v.z = (kk + 2 >= kbeg && kk + 2 < kend) ? v.z : 0.f;
        v.w = (kk + 3 >= kbeg && kk + 3 < kend) ? v.w : 0.f;
      }
      return v;
    };
    auto load = [&](int c) {
      const int k0 = kal + c * 32;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int i = tid + NTHR * j, row = i >> 3, c4 = i & 7;
        ra[j] = ld4(rowA(row), k0 + c4 * 4);
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int i = tid + NTHR * j, row = i >> 3, c4 = i & 7;
        rb[j] = ld4(rowB(row), k0 + c4 * 4);
      }
    };
    // chunk c of this call accumulates into tensor-memory slot (c / 2) mod 2;
    // a slot is drained once the last chunk of its pair has completed
    auto ends_pair = [&](int c) { return (c & 1) == 1 || c == nchunk - 1; };
    if (nchunk > 0) load(0);
    for (int c = 0; c < nchunk; ++c) {
      const int g = g0 + c, s = g & 1;
      if (c >= 2) {  // chunk c - 2 used stage s
        if (!wait_done(g - 2)) break;
        if (ends_pair(c - 2)) drain((c - 2) >> 1);
      }
      if (*abort_flag) break;
      TcStage<BN>& S = sm.st[s];
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int i = tid + NTHR * j;
        store_split4(S.a_hi, S.a_lo, i >> 3, (i & 7) * 4, ra[j]);
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int i = tid + NTHR * j;
        store_split4(S.b_hi, S.b_lo, i >> 3, (i & 7) * 4, rb[j]);
      }
      if (c + 1 < nchunk) load(c + 1);
      fence_async_smem();
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.full[s]);
    }
    for (int c = max(0, nchunk - 2); c < nchunk && !*abort_flag; ++c) {  // the last one or two chunks, in order
      if (!wait_done(g0 + c)) break;
      if (ends_pair(c)) drain(c >> 1);
    }
  } else {
    // MMA warp: the whole warp runs the loop, lane 0 issues
    const uint32_t idesc = idesc_tf32(128, BN);
    for (int c = 0; c < nchunk; ++c) {
      const int g = g0 + c, s = g & 1;
      if (*abort_flag) break;
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&sm.full[s], (g >> 1) & 1) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) {
        *abort_flag = 1;
        break;
      }
      fence_after_sync();
      if (lane == 0) {
        TcStage<BN>& S = sm.st[s];
        const uint32_t ah = smem_addr(S.a_hi), al = smem_addr(S.a_lo);
        const uint32_t bh = smem_addr(S.b_hi), bl = smem_addr(S.b_lo);
        const uint32_t dcol = sm.tmem + BN * ((c >> 1) & 1);
        const bool first = (c & 1) == 0;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t o = ks * 32;
          mma_tf32(dcol, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, (first && ks == 0) ? 0u : 1u);
          mma_tf32(dcol, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
          mma_tf32(dcol, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
        }
        mma_commit(&sm.done[s]);
      }
      __syncwarp();
    }
    if (lane == 0) mma_commit(&sm.fin);  // arrives once every MMA issued above has completed
    __syncwarp();
  }
  // every issued MMA has completed before anyone reads or frees tensor memory
  const bool w = mbar_wait(&sm.fin, cs.calls & 1);
  cs.chunks += nchunk;
  cs.calls += 1;
  return __syncthreads_and(w && !*abort_flag) != 0;
}

// ---------------------------------------------------------------------------
// Compensated product with pre-split operands fed by TMA.  The TF32 hi/lo
// halves of both operands are in global memory (k_split_tf32), so a
// 128 x 128 output tile costs no conversion work on the SM: one producer
// thread loads each 32-wide K chunk (four 128 x 32 boxes, 64 KB) into a ring
// of kSplitStages stages, one thread issues the chunk's 12 MMAs
// (hi.hi + hi.lo + lo.hi per 8-wide K step) into one of two tensor-memory
// accumulators, and 16 worker warps drain an accumulator into (hi, lo) with
// TwoSum every kSplitDrain chunks while the other one is being filled.
// Draining every 64 values of K instead of every 32 (comp_product) halves
// the SM's TwoSum work; the FP32 partial sums are twice as long, which moves
// the predictive mean by a few per cent of its error against the FP64 form
// (that error is dominated by the FP32 window factorisations).
constexpr int kSplitStages = 3;
constexpr int kSplitDrain = 2;
constexpr int kSplitWorkers = 16;                        // 4 lane quarters x 4 groups of 32 columns
constexpr int kSplitThreads = 32 * (kSplitWorkers + 2);  // + MMA warp + TMA warp
struct SplitSmem {
  tc::TcStage<128> st[kSplitStages];
  uint64_t full[kSplitStages], empty[kSplitStages], done[2], drained[2], fin;
  uint32_t tmem;
  int abort;
};
__device__ __forceinline__ SplitSmem& split_smem(unsigned char* raw) {
  uintptr_t p = reinterpret_cast<uintptr_t>(raw);
  p = (p + 1023) & ~uintptr_t(1023);
  return *reinterpret_cast<SplitSmem*>(p);
}

// TF32 hi/lo halves of a point-major FP32 matrix (n rows of ld values, ld a
// multiple of 4), rounded as store_split4 rounds them: hi = tf32(x),
// lo = tf32(x - hi).  reverse != 0 stores row p at row n - 1 - p: the rows
// of a window (training points in reverse) are then consecutive.
__global__ void k_split_tf32(const float* __restrict__ V, int64_t n, int ld, int reverse, float* __restrict__ hi,
                             float* __restrict__ lo) {
  const int l4 = ld >> 2;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n * l4) return;
  const int64_t p = q / l4, c = q - p * l4;
  const float4 v = reinterpret_cast<const float4*>(V)[q];
  float4 h, l;
  h.x = tc::tf32_round(v.x); l.x = tc::tf32_round(v.x - h.x);
  h.y = tc::tf32_round(v.y); l.y = tc::tf32_round(v.y - h.y);
  h.z = tc::tf32_round(v.z); l.z = tc::tf32_round(v.z - h.z);
  h.w = tc::tf32_round(v.w); l.w = tc::tf32_round(v.w - h.w);
  const int64_t o = (reverse ? n - 1 - p : p) * l4 + c;
  reinterpret_cast<float4*>(hi)[o] = h;
  reinterpret_cast<float4*>(lo)[o] = l;
}

__device__ __forceinline__ void split_setup(SplitSmem& sm) {
  using namespace tc;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSplitStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&sm.done[a], 1);
      mbar_init(&sm.drained[a], kSplitWorkers);
    }
    mbar_init(&sm.fin, 1);
    sm.abort = 0;
    mbar_fence_init();
  }
  if ((threadIdx.x >> 5) == kSplitWorkers) tmem_alloc(&sm.tmem, 256);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}
__device__ __forceinline__ void split_teardown(SplitSmem& sm) {
  using namespace tc;
  fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == kSplitWorkers) tmem_dealloc(sm.tmem, 256);
}

// Barrier of the kSplitWorkers worker warps only (id 1) that also ANDs a
// flag over them, so that all of them take the same branch after it.
__device__ __forceinline__ bool worker_sync_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(kSplitWorkers * 32)
      : "memory");
  return r != 0;
}

// Persistent loop over output tiles t = blockIdx.x, blockIdx.x + gridDim.x,
// ... < ntiles, each hi + lo = sum over its chunks c < chunks(t) of
// sum_{k < 32} A(ya + r, x + k) B(yb + c', x + k) with (x, ya, yb) =
// at(base, c) and base = coords(t) (computed once per tile by the producer):
// A from (ahi, alo), B from (bhi, blo); rows outside the maps read zero.  The
// producer and MMA warps run ahead into the next tile while the workers
// finish the current one: before(t) (shared-memory set-up of the epilogue,
// worker warps only, between two worker barriers), the drains, then
// after(t, hi, lo), where worker warp w holds row 32 (w mod 4) + lane,
// columns 32 (w / 4) + j in hi[j] + lo[j].  Barrier phases run on across
// tiles.  Every wait has an iteration limit: on a timeout all roles stop,
// no copy is left landing, and false is returned in every thread.
template <class Chunks, class Coords, class At, class Before, class After>
__device__ bool split_persistent(SplitSmem& sm, const CUtensorMap* ahi, const CUtensorMap* alo,
                                 const CUtensorMap* bhi, const CUtensorMap* blo, int ntiles, Chunks chunks,
                                 Coords coords, At at, Before before, After after) {
  using namespace tc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_flag = &sm.abort;
  if (warp < kSplitWorkers) {
    const int q = warp & 3, half = warp >> 2;
    const uint32_t tlane = sm.tmem + ((uint32_t)(q * 32) << 16) + half * 32;
    int G = 0;  // groups drained so far by this CTA
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      ok = worker_sync_and(ok && !*abort_flag);  // also: the previous epilogue is done with shared memory
      if (!ok) break;
      before(t);
      worker_sync_and(true);
      float hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.f;
      const int ngroup = (chunks(t) + kSplitDrain - 1) / kSplitDrain;
      for (int g = 0; g < ngroup && ok; ++g, ++G) {
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
        float tv[16];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tmem_ld16(tlane + 128 * a + 16 * h, tv);
#pragma unroll
          for (int j = 0; j < 16; ++j) two_sum(hi[16 * h + j], lo[16 * h + j], tv[j]);
        }
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.drained[a]);
      }
      ok = worker_sync_and(ok && !*abort_flag);
      if (!ok) break;
      after(t, hi, lo);
    }
  } else if (warp == kSplitWorkers) {
    // MMA warp: the whole warp runs the loops, lane 0 waits and issues
    const uint32_t idesc = idesc_tf32(128, 128);
    int C = 0, G = 0;  // chunks and groups issued so far by this CTA
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int nchunk = chunks(t);
      for (int c = 0; c < nchunk; ++c, ++C) {
        const int s = C % kSplitStages, a = G & 1;
        const bool first = (c % kSplitDrain) == 0, last = (c % kSplitDrain) == kSplitDrain - 1 || c == nchunk - 1;
        int okw = 1;
        if (lane == 0) {
          okw = mbar_wait(&sm.full[s], (C / kSplitStages) & 1) ? 1 : 0;
          if (okw && first && G >= 2) okw = mbar_wait(&sm.drained[a], ((G - 2) >> 1) & 1) ? 1 : 0;
        }
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw || *abort_flag) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        fence_after_sync();
        if (lane == 0) {
          TcStage<128>& S = sm.st[s];
          const uint32_t ah = smem_addr(S.a_hi), al = smem_addr(S.a_lo);
          const uint32_t bh = smem_addr(S.b_hi), bl = smem_addr(S.b_lo);
          const uint32_t dcol = sm.tmem + 128 * a;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t o = ks * 32;
            mma_tf32(dcol, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, (first && ks == 0) ? 0u : 1u);
            mma_tf32(dcol, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
            mma_tf32(dcol, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
          }
          mma_commit(&sm.empty[s]);           // the stage may be refilled
          if (last) mma_commit(&sm.done[a]);  // the accumulator may be drained
        }
        __syncwarp();
        if (last) ++G;
      }
    }
    if (lane == 0) mma_commit(&sm.fin);  // arrives once every MMA issued above has completed
    __syncwarp();
  } else {
    // TMA producer: the whole warp runs the loops, lane 0 waits and issues
    int C = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int4 base = coords(t);
      const int nchunk = chunks(t);
      for (int c = 0; c < nchunk; ++c, ++C) {
        const int s = C % kSplitStages;
        int okw = 1;
        if (lane == 0 && C >= kSplitStages) okw = mbar_wait(&sm.empty[s], (C / kSplitStages - 1) & 1) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw || *abort_flag) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        if (lane == 0) {
          TcStage<128>& S = sm.st[s];
          const int3 y = at(base, c);
          mbar_arrive_expect_tx(&sm.full[s], 4u * 128u * 32u * 4u);
          tma_load_2d(S.a_hi, ahi, y.x, y.y, &sm.full[s]);
          tma_load_2d(S.a_lo, alo, y.x, y.y, &sm.full[s]);
          tma_load_2d(S.b_hi, bhi, y.x, y.z, &sm.full[s]);
          tma_load_2d(S.b_lo, blo, y.x, y.z, &sm.full[s]);
        }
        __syncwarp();
      }
    }
    // no copy may still be landing in shared memory when the CTA leaves
    if (lane == 0)
      for (int c = C > kSplitStages ? C - kSplitStages : 0; c < C; ++c)
        mbar_wait(&sm.full[c % kSplitStages], (c / kSplitStages) & 1);
    __syncwarp();
  }
  // every issued MMA has completed before anyone frees tensor memory
  const bool w = mbar_wait(&sm.fin, 0);
  return __syncthreads_and(w && !*abort_flag) != 0;
}

// Residual tiles on the tensor cores (mixed form), one persistent CTA per SM
// walking the item list.  Item (window, I, J): rows [128 I, 128 I + 128) x
// columns [RB J, RB J + RB) of the window's residual
// R = K + sigma_n^2 I - Vt Vt^T, blanket-first, with the Vt Vt^T sum of
// split_persistent (RB = 128 columns).  (vhi, vlo): tensor maps of the TF32
// halves of V in reversed point order (row nrev - 1 - p holds point p), 32 x
// 128 boxes, 128-byte swizzle; nchunk = (row length of V) / 32.  Rows and
// columns past the window's order read other points' rows (or zeros): the
// epilogue writes the identity there and never reads those sums.
constexpr int RB = 128;

// Squared scaled distance |a - b|^2 over D (zero-padded) dimensions; b is a
// 16-byte-aligned shared-memory row read with broadcast vector loads.
template <int D>
__device__ __forceinline__ float dist2(const float (&a)[D], const float* b) {
  float d2 = 0.f;
#pragma unroll
  for (int t = 0; t < D; t += 4) {
    const float4 v = *reinterpret_cast<const float4*>(b + t);
    float u = a[t] - v.x;
    d2 = fmaf(u, u, d2);
    u = a[t + 1] - v.y;
    d2 = fmaf(u, u, d2);
    u = a[t + 2] - v.z;
    d2 = fmaf(u, u, d2);
    u = a[t + 3] - v.w;
    d2 = fmaf(u, u, d2);
  }
  return d2;
}
// Input dimension padded for the unrolled epilogues (a multiple of 4).
__host__ __device__ constexpr int pad_dim(int d) { return d <= 8 ? 8 : MAXD; }

template <int D>
__global__ void __launch_bounds__(kSplitThreads, 1) k_resid_tc(const int4* __restrict__ items, int nitems,
                                                  const Win* __restrict__ wins, const float* __restrict__ xs, int d,
                                                  const __grid_constant__ CUtensorMap vhi,
                                                  const __grid_constant__ CUtensorMap vlo, int nrev, int nchunk,
                                                  float ss2, float sn2, float* __restrict__ buf,
                                                  int* __restrict__ err) {
  using namespace tc;
  extern __shared__ __align__(16) unsigned char smraw[];
  SplitSmem& sm = split_smem(smraw);
  __shared__ __align__(16) float xc[RB][D];  // scaled inputs of the tile's columns, zero-padded
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  split_setup(sm);
  auto chunks = [&](int) { return nchunk; };
  auto coords = [&](int t) -> int4 {
    const int4 it = items[t];
    const int base = nrev - (int)wins[it.x].g_end;  // reversed row of the window's local row 0
    return make_int4(base + it.y * 128, base + it.z * RB, 0, 0);
  };
  auto at = [](int4 b, int c) { return make_int3(32 * c, b.x, b.y); };
  auto before = [&](int t) {
    const int4 it = items[t];
    const Win w = wins[it.x];
    const int c0 = it.z * RB;
    for (int e = tid; e < RB * D; e += kSplitWorkers * 32) {
      const int r = e / D, q = e % D;
      xc[r][q] = (c0 + r < w.n && q < d) ? xs[(w.g_end - 1 - (c0 + r)) * d + q] : 0.f;
    }
  };
  auto after = [&](int t, float(&hi)[32], float(&lo)[32]) {
    const int4 it = items[t];
    const Win w = wins[it.x];
    const int r0 = it.y * 128, c0 = it.z * RB;
    const int q = warp & 3, half = warp >> 2;
    const int i = r0 + q * 32 + lane;
    const int cg = c0 + half * 32;  // this thread's 32 columns (npad is a multiple of 64)
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
  const bool ok = split_persistent(sm, &vhi, &vlo, &vhi, &vlo, nitems, chunks, coords, at, before, after);
  if (!ok && tid == 0) atomicExch(err, 1);
  split_teardown(sm);
}

// Block-part summary rows of the owned windows, compacted and split for
// k_gram_split: window wi's extra rows e < se = s + 1, columns [nB, n) (its
// [z_m | Z_m]^T, Definition 1 whitened) go to rows wi se + e, columns
// [0, n - nB) of (hi, lo), row length kmax (a multiple of 32, zero pad).
__global__ void k_split_summary(const Win* __restrict__ wins, const float* __restrict__ buf, int se, int kmax,
                                float* __restrict__ hi, float* __restrict__ lo) {
  // block (x, window y): rows e = 4 x + threadIdx.y, four values per thread
  // and step (16-byte loads when the row's first value is aligned)
  const Win w = wins[blockIdx.y];
  const int e = blockIdx.x * blockDim.y + threadIdx.y;
  if (e >= se) return;
  const int nb = w.n - w.nB;
  const float* src = buf + w.base + (int64_t)(w.npad + e) * w.npad + w.nB;
  const bool al = (w.nB & 3) == 0;
  const int64_t o = ((int64_t)blockIdx.y * se + e) * kmax;
  for (int j = 4 * threadIdx.x; j < kmax; j += 4 * blockDim.x) {
    float4 x;
    if (al && j + 3 < nb) {
      x = *reinterpret_cast<const float4*>(src + j);
    } else {
      x.x = j < nb ? src[j] : 0.f;
      x.y = j + 1 < nb ? src[j + 1] : 0.f;
      x.z = j + 2 < nb ? src[j + 2] : 0.f;
      x.w = j + 3 < nb ? src[j + 3] : 0.f;
    }
    float4 h, l;
    h.x = tc::tf32_round(x.x); l.x = tc::tf32_round(x.x - h.x);
    h.y = tc::tf32_round(x.y); l.y = tc::tf32_round(x.y - h.y);
    h.z = tc::tf32_round(x.z); l.z = tc::tf32_round(x.z - h.z);
    h.w = tc::tf32_round(x.w); l.w = tc::tf32_round(x.w - h.w);
    *reinterpret_cast<float4*>(hi + o + j) = h;
    *reinterpret_cast<float4*>(lo + o + j) = l;
  }
}

// Gram of the local summaries on the tensor cores (mixed form), one
// persistent CTA per SM: item t = (tile (I, J) of the lower 128-tiles of G,
// window group g) adds sum over the windows of group g of
// [z_m | Z_m]^T [z_m | Z_m] with split_persistent, whose K runs window by
// window over the compacted rows of k_split_summary (kmax / 32 chunks each),
// and writes hi + lo as FP64 partial g, summed over groups by k_gram_reduce.
// Rows and columns past se read the next window's rows (or zeros) and are
// never written.
__global__ void __launch_bounds__(kSplitThreads, 1) k_gram_split(const int2* __restrict__ tiles, int ntile, int nwin,
                                                    int group, int se, int kmax,
                                                    const __grid_constant__ CUtensorMap shi,
                                                    const __grid_constant__ CUtensorMap slo,
                                                    double* __restrict__ partial, int* __restrict__ err) {
  using namespace tc;
  extern __shared__ __align__(16) unsigned char smraw[];
  SplitSmem& sm = split_smem(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cpw = kmax / 32;
  const int ngroup = (nwin + group - 1) / group;
  split_setup(sm);
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
    return make_int3(32 * (c % cpw), wi * se + b.x, wi * se + b.y);
  };
  auto before = [](int) {};
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
  const bool ok = split_persistent(sm, &shi, &slo, &shi, &slo, ntile * ngroup, chunks, coords, at, before, after);
  if (!ok && tid == 0) atomicExch(err, 1);
  split_teardown(sm);
}

// h[u][k] = sum over the pairs (n, m) of test block n of
// sum_{c in kept columns} P[u][c] X_{1+k}[c]  -  Vu[u][k]  on the tensor
// cores (mixed form): P rows are the swept right-hand sides, X_{1+k} the
// extra rows (L^-1 Vt_W)^T of window m, so the sum over a pair is a product
// with K over the window's kept columns [c0, c1).  Items: x = first pair of
// the test block, y = pair count, z = 128-row u tile, w = RB-wide s tile.
__global__ void __launch_bounds__(comp_threads<RB>(), 1) k_pred_accum_tc(const Pair* __restrict__ pairs,
                                                                       const int4* __restrict__ items,
                                                                       const Win* __restrict__ wins,
                                                                       const float* __restrict__ buf,
                                                                       const float* __restrict__ P,
                                                                       const float* __restrict__ Vu, int s,
                                                                       float* __restrict__ h, int* __restrict__ err) {
  using namespace tc;
  const int4 it = items[blockIdx.x];
  const int u0 = it.z * 128, k0 = it.w * RB;
  extern __shared__ __align__(16) unsigned char smraw[];
  CompSmem<RB>& sm = comp_smem<RB>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  comp_setup(sm);
  CompState cs;
  float hi[32], lo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.f;
  bool ok = true;
  for (int pi = 0; pi < it.y && ok; ++pi) {
    const Pair pr = pairs[it.x + pi];
    const Win w = wins[pr.win];
    const float* Pp = P + pr.pbase;
    const float* E = buf + w.base + (int64_t)w.npad * w.npad;
    const int64_t ld = w.npad;
    auto rowA = [&](int r) -> const float* { return (u0 + r < pr.nu) ? Pp + (int64_t)(u0 + r) * ld : nullptr; };
    auto rowB = [&](int c) -> const float* { return (k0 + c < s) ? E + (int64_t)(1 + k0 + c) * ld : nullptr; };
    ok = comp_product<RB, true>(sm, cs, pr.c0, pr.c1, rowA, rowB, hi, lo);
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  const Pair first = pairs[it.x];
  const int q = warp & 3, half = warp >> 2;
  const int uu = u0 + q * 32 + lane;
  const int kg = k0 + half * 32;
  if (ok && warp < RB / 8 && uu < first.nu) {
    const int64_t row = first.u0 + uu;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (kg + j < s) h[row * s + kg + j] = (hi[j] + lo[j]) - Vu[row * s + kg + j];
  }
  comp_teardown(sm);
}

// The h accumulation per window (mixed form): the test rows that use window m
// (the pairs (n, m), n = m .. m + B) share its extra rows X_{1+k} as the B
// operand, so one 128-row tile covers the test points of several blocks.
// Item x = first index into wp (the window's pairs, increasing n), y = pair
// count, z = 128-row tile of the window's test rows, w = RB-wide s tile; the
// partial hw[(prow + r) * s + k] = sum over the pair's kept columns of
// P[r][c] X_{1+k}[c] (block columns [nB, n) for every row, the blanket
// columns [0, nB) only for the rows of block m itself), where prow is the
// window's first partial row (wrow[item], one entry per item).  k_pred_hsum adds each test point's
// partials in window order.
__global__ void __launch_bounds__(comp_threads<RB>(), 1) k_pred_accum_win(const Pair* __restrict__ pairs,
                                                                        const int* __restrict__ wp,
                                                                        const int4* __restrict__ items,
                                                                        const int64_t* __restrict__ wrow,
                                                                        const Win* __restrict__ wins,
                                                                        const float* __restrict__ buf,
                                                                        const float* __restrict__ P, int s,
                                                                        float* __restrict__ hw, int* __restrict__ err) {
  using namespace tc;
  const int4 it = items[blockIdx.x];
  const int u0 = it.z * 128, k0 = it.w * RB;
  extern __shared__ __align__(16) unsigned char smraw[];
  CompSmem<RB>& sm = comp_smem<RB>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  comp_setup(sm);
  const Pair p0 = pairs[wp[it.x]];
  const Win w = wins[p0.win];
  const float* E = buf + w.base + (int64_t)w.npad * w.npad;
  const int64_t ld = w.npad;
  // row r of the tile -> pointer to its P row (nullptr past the window's test
  // rows) and whether it is a row of block m itself (kept blanket columns)
  __shared__ const float* rowp[128];
  __shared__ int rowown[128];
  __shared__ int s_rows;
  if (tid < 128) {
    int rr = u0 + tid;
    const float* ptr = nullptr;
    int own = 0;
    for (int j = 0; j < it.y; ++j) {
      const Pair pr = pairs[wp[it.x + j]];
      if (rr < pr.nu) {
        own = pr.c0 == 0;
        ptr = P + pr.pbase + (int64_t)rr * ld;
        break;
      }
      rr -= pr.nu;
    }
    rowp[tid] = ptr;
    rowown[tid] = own;
  }
  if (tid == 0) {
    int rows = 0;
    for (int j = 0; j < it.y; ++j) rows += pairs[wp[it.x + j]].nu;
    s_rows = rows;
  }
  __syncthreads();
  auto rowB = [&](int c) -> const float* { return (k0 + c < s) ? E + (int64_t)(1 + k0 + c) * ld : nullptr; };
  CompState cs;
  float hi[32], lo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.f;
  auto rowAll = [&](int r) -> const float* { return rowp[r]; };
  bool ok = comp_product<RB, true>(sm, cs, w.nB, w.n, rowAll, rowB, hi, lo);
  if (ok && w.nB > 0) {
    auto rowOwn = [&](int r) -> const float* { return rowown[r] ? rowp[r] : nullptr; };
    ok = comp_product<RB, true>(sm, cs, 0, w.nB, rowOwn, rowB, hi, lo);
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  const int rows = s_rows;
  const int q = warp & 3, half = warp >> 2;
  const int rr = u0 + q * 32 + lane;
  const int kg = k0 + half * 32;
  if (ok && warp < RB / 8 && rr < rows) {
    float* dst = hw + (wrow[blockIdx.x] + rr) * (int64_t)s;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (kg + j < s) dst[kg + j] = hi[j] + lo[j];
  }
  comp_teardown(sm);
}

// h[u][k] = sum over the pairs (n, m) of u's test block n, in window order, of
// hw[(prow of the pair + u - u0) * s + k] (added in FP64), minus Vu[u][k].
// Grid: y = test block (tb: x = its first pair, y = pair count, z = first test
// row, w = rows), x covers the block's rows x s elements; prow[pair] = the
// pair's first partial row.
__global__ void k_pred_hsum(const int4* __restrict__ tb, const int64_t* __restrict__ prow,
                            const float* __restrict__ hw, const float* __restrict__ Vu, int s,
                            float* __restrict__ h) {
  const int4 t = tb[blockIdx.y];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)t.w * s) return;
  const int64_t r = e / s;
  const int k = (int)(e - r * s);
  double acc = 0.0;
  for (int j = 0; j < t.y; ++j) acc += (double)hw[(prow[t.x + j] + r) * s + k];
  const int64_t o = (t.z + r) * (int64_t)s + k;
  h[o] = (float)(acc - (double)Vu[o]);
}

// Prediction right-hand sides on the tensor cores, one persistent CTA per SM
// walking the item list: item (pair, u tile of 128, column tile of RB):
// P[u][i] = K(xu_u, x_g(i)) - Vu[u] . Vt[g(i)] for the window of the pair,
// with split_persistent (the same cancellation as the residual).
// (uhi, ulo): tensor maps of the TF32 halves of Vu in test-point order;
// (vhi, vlo) those of Vt in reversed point order (row nrev - 1 - p holds
// point p); nchunk = (row length) / 32.  Test rows past the block and window
// columns past its order are never written from their sums.
template <int D>
__global__ void __launch_bounds__(kSplitThreads, 1) k_pred_rhs_tc(const Pair* __restrict__ pairs, const int4* __restrict__ items,
                                                     int nitems, const Win* __restrict__ wins,
                                                     const float* __restrict__ xs, const float* __restrict__ xu, int d,
                                                     const __grid_constant__ CUtensorMap uhi,
                                                     const __grid_constant__ CUtensorMap ulo,
                                                     const __grid_constant__ CUtensorMap vhi,
                                                     const __grid_constant__ CUtensorMap vlo, int nrev, int nchunk,
                                                     float ss2, float* __restrict__ P, int* __restrict__ err) {
  using namespace tc;
  extern __shared__ __align__(16) unsigned char smraw[];
  SplitSmem& sm = split_smem(smraw);
  __shared__ __align__(16) float xc[RB][D];  // scaled inputs of the tile's columns, zero-padded
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  split_setup(sm);
  auto chunks = [&](int) { return nchunk; };
  auto coords = [&](int t) -> int4 {
    const int4 it = items[t];
    const Pair pr = pairs[it.x];
    return make_int4(pr.u0 + it.y * 128, nrev - (int)wins[pr.win].g_end + it.z * RB, 0, 0);
  };
  auto at = [](int4 b, int c) { return make_int3(32 * c, b.x, b.y); };
  auto before = [&](int t) {
    const int4 it = items[t];
    const Win w = wins[pairs[it.x].win];
    const int c0 = it.z * RB;
    for (int e = tid; e < RB * D; e += kSplitWorkers * 32) {
      const int r = e / D, q = e % D;
      xc[r][q] = (c0 + r < w.n && q < d) ? xs[(w.g_end - 1 - (c0 + r)) * d + q] : 0.f;
    }
  };
  auto after = [&](int t, float(&hi)[32], float(&lo)[32]) {
    const int4 it = items[t];
    const Pair pr = pairs[it.x];
    const Win w = wins[pr.win];
    const int u0 = it.y * 128, c0 = it.z * RB;
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
  const bool ok = split_persistent(sm, &uhi, &ulo, &vhi, &vlo, nitems, chunks, coords, at, before, after);
  if (!ok && tid == 0) atomicExch(err, 1);
  split_teardown(sm);
}

}  // namespace lma
