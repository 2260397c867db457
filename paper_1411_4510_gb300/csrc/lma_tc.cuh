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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
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

// Diagonal block of column panel kp on the tensor cores (mixed form), one
// CTA per window (grid x = window, y = 1):
//   D = A_{kk} - A_{k, kb:k0} A_{k, kb:k0}^T   (3xTF32 on tcgen05; skipped when kb = k0)
// over the 64 rows of the block, then D = L_kk L_kk^T factorised in shared
// memory (L_kk and inv(L_kk) written; *info set if D is not positive
// definite).  Columns [0, kb) were applied by the wider updates; the rows
// below the block are left to the panel kernels.
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
      return (r < TB && row < w.rows) ? A + (int64_t)row * ld + kb : nullptr;
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
  if (row < w.rows && rl < TB) {  // the diagonal block's rows only; the rows below are left to the panel kernels
    const float* src = A + (int64_t)row * ld + k0 + half * 32;
    float4 av[8];
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) av[j4] = *reinterpret_cast<const float4*>(src + 4 * j4);
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
      float* d = &Dm[rl][half * 32 + 4 * j4];
      d[0] = av[j4].x - v[4 * j4 + 0];
      d[1] = av[j4].y - v[4 * j4 + 1];
      d[2] = av[j4].z - v[4 * j4 + 2];
      d[3] = av[j4].w - v[4 * j4 + 3];
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
    // Each producer warp subtracts the accumulator of 32 rows (its lane
    // quadrant q) x PW columns (its part).  Tensor memory gives a row per
    // lane; the rows go through the now idle stage ring (float4 slots
    // swizzled by the row, conflict-free both ways) so that global memory is
    // read and written coalesced, PW4 lanes per row.
    constexpr int NPART = kWsProducers / 4, PW = BN / NPART, PW4 = PW / 4, RPI = 32 / PW4;
    static_assert(PW4 == 16 || PW4 == 32, "a row part is 16 or 32 float4");
    const int q = warp & 3, part = warp >> 2;
    float4* xs = reinterpret_cast<float4*>(&sm.st[0]) + warp * 32 * PW4;
    auto slot = [&](int r, int c4) { return r * PW4 + (c4 ^ (r & (PW4 - 1))); };
    for (int g = 0; g < PW / 16; ++g) {
      const int c0 = part * PW + 16 * g;
      if (c0 >= ncol) break;  // warp-uniform
      float t[16];
      tmem_ld16(sm.tmem + ((uint32_t)(q * 32) << 16) + c0, t);
#pragma unroll
      for (int j4 = 0; j4 < 4; ++j4)
        xs[slot(lane, 4 * g + j4)] = make_float4(t[4 * j4], t[4 * j4 + 1], t[4 * j4 + 2], t[4 * j4 + 3]);
    }
    __syncwarp();
    const int cr = lane / PW4, cc = lane % PW4;
    const int col = part * PW + 4 * cc;  // local column of this lane's float4
    constexpr int NR = 32 / RPI, NL = 8;  // rows per lane, loaded NL at a time before any store
    for (int k0 = 0; k0 < NR; k0 += NL) {
      float4 a[NL];
#pragma unroll
      for (int k = 0; k < NL; ++k) {
        const int row = r0 + q * 32 + (k0 + k) * RPI + cr;
        a[k] = (row < w.rows && col < ncol) ? *reinterpret_cast<const float4*>(A + (int64_t)row * ld + s0 + col)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < NL; ++k) {
        const int r = (k0 + k) * RPI + cr, row = r0 + q * 32 + r;
        if (row < w.rows && col < ncol) {
          float* p = A + (int64_t)row * ld + s0 + col;
          const float4 b = xs[slot(r, cc)];
          a[k].x -= b.x;
          a[k].y -= b.y;
          a[k].z -= b.z;
          a[k].w -= b.w;
          if (s0 + col + 3 <= row) {
            *reinterpret_cast<float4*>(p) = a[k];
          } else {  // the diagonal: lower triangle only
            if (s0 + col <= row) p[0] = a[k].x;
            if (s0 + col + 1 <= row) p[1] = a[k].y;
            if (s0 + col + 2 <= row) p[2] = a[k].z;
          }
        }
      }
    }
  }
  ws_teardown(sm);
}

}  // namespace lma

namespace lma {

namespace tc {

// Persistent panel kernel (below): 8 producer warps, 1 MMA warp, 4 epilogue
// warps (13 warps: at most 4 on a scheduler, so 128 registers a thread).
// Operands are 64 values of K wide, stored as two 128-byte-swizzled 32-wide
// halves (TF32 hi and lo of each).
constexpr int kPtProducers = 8, kPtEpilogue = 4;
constexpr int kPtThreads = 32 * (kPtProducers + 1 + kPtEpilogue);

struct alignas(1024) PtTileA {  // 128 rows x 64
  float hi[2][128 * 32];
  float lo[2][128 * 32];
};
struct alignas(1024) PtTileB {  // 64 rows x 64
  float hi[2][64 * 32];
  float lo[2][64 * 32];
};
struct PtSmem {
  PtTileA a[2];     // per item in flight: the update's left operand, then T
  PtTileB b1, b2;   // per window: the update's right operand, inv(L_kk)
  float xo[128 * 64];  // epilogue: rows between tensor memory (a row a thread) and coalesced global access
  uint64_t full[2], tfull[2], empty[2], upd[2], sol[2], afree[2], bfull, bempty, done;
  uint32_t tmem;
  int abort;
};

// TF32 hi/lo of 4 K-consecutive values at (row, k), k < 64, of a 64-wide tile
template <class Tile>
__device__ __forceinline__ void pt_store(Tile& t, uint32_t row, uint32_t k, float4 v) {
  store_split4(t.hi[k >> 5], t.lo[k >> 5], row, k & 31u, v);
}

// 3xTF32 product of a 128 x 64 tile (a) with a 64 x 64 tile (b)^T into the
// 64 accumulator columns at d; `acc` = 0 starts from zero.
__device__ __forceinline__ void pt_mma(uint32_t d, const PtTileA& a, const PtTileB& b, uint32_t acc) {
  const uint32_t idesc = idesc_tf32(128, 64);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t ah = smem_addr(a.hi[h]), al = smem_addr(a.lo[h]);
    const uint32_t bh = smem_addr(b.hi[h]), bl = smem_addr(b.lo[h]);
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const uint32_t o = ks * 32;
      mma_tf32(d, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, (acc || h > 0 || ks > 0) ? 1u : 0u);
      mma_tf32(d, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
      mma_tf32(d, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
    }
  }
}

}  // namespace tc

// Column panel kp of every window, for the rows below its diagonal block, as
// a persistent kernel (one CTA per SM over a contiguous range of
// (window, 128-row tile) items, window-major):
//   T = A_{rows, panel} - A_{rows, kfrom:k0} A_{panel, kfrom:k0}^T   (K = k0 - kfrom, 0 or 64)
//   A_{rows, panel} <- T inv(L_kk)^T
// with both products on tcgen05 (3xTF32).  The diagonal block L_kk and its
// inverse come from k_chol_step_tc.  Warp roles:
//   producers (warps 0-7): per window, the right operands (A_{panel, kfrom:k0}
//     and inv(L_kk)) split into TF32 hi/lo; per item, the left operand
//     (A_{rows, kfrom:k0}, or A_{rows, panel} when K = 0), loaded two items
//     ahead into registers, split into one of two stages;
//   MMA warp (warp 8, lane 0 issues): the update into the item's
//     accumulator (one of two, 64 columns each), then the solve;
//   epilogue (4 warps, a quarter of the rows each): T = own rows - update,
//     written split into the item's stage as the solve's left operand; then
//     the solved rows are stored (coalesced through shared memory).
// Two items are in flight, so one item's loads overlap another's products
// and stores.  Every wait is bounded; on a timeout the CTA raises *err,
// every role leaves its loop and the MMA warp waits for its products before
// the tensor memory is freed.
__global__ void __maxnreg__(128) k_chol_panel_pt(const Win* __restrict__ wins, int nwin, float* __restrict__ buf,
                                                 const float* __restrict__ dinv, int kp, int kfrom, int ntile,
                                                 int* __restrict__ err) {
  grid_dep_wait();
  grid_dep_launch();
  using namespace tc;
  extern __shared__ __align__(16) unsigned char smraw[];
  PtSmem& sm = *reinterpret_cast<PtSmem*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k0 = kp * TB;
  const bool upd = kfrom < k0;  // K = 64
  const int64_t total = (int64_t)ntile * nwin;
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  const int64_t ibeg = (int64_t)blockIdx.x * per, iend = min(total, ibeg + per);
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&sm.full[s], kPtProducers);
      mbar_init(&sm.tfull[s], kPtEpilogue);
      mbar_init(&sm.empty[s], 1);
      mbar_init(&sm.upd[s], 1);
      mbar_init(&sm.sol[s], 1);
      mbar_init(&sm.afree[s], kPtEpilogue);
    }
    mbar_init(&sm.bfull, kPtProducers);
    mbar_init(&sm.bempty, 1);
    mbar_init(&sm.done, 1);
    sm.abort = 0;
    mbar_fence_init();
  }
  if (warp == kPtProducers) tmem_alloc(&sm.tmem, 128);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  volatile int* abort_flag = &sm.abort;
  // item i -> window and first row; false when the tile holds no rows of the window
  auto item = [&](int64_t i, int& wi, int& r0) -> bool {
    wi = (int)(i / ntile);
    const Win& w = wins[wi];
    r0 = k0 + TB + (int)(i % ntile) * 128;
    return k0 < w.npad && r0 < w.rows;
  };
  // bounded wait by lane 0, result shared with the warp
  auto wait_warp = [&](uint64_t* bar, uint32_t parity) -> bool {
    int ok = 1;
    if (lane == 0) ok = mbar_wait(bar, parity) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) *abort_flag = 1;
    return ok != 0;
  };

  if (warp < kPtProducers) {
    // ---------------- producers: two items' loads in flight ----------------
    constexpr int PT = 32 * kPtProducers, NA = 128 * 16 / PT, NB = 64 * 16 / PT;  // float4 per thread
    const int pt = tid;
    float4 ra[2][NA];
    auto load_a = [&](int wi, int r0, float4 (&x)[NA]) {
      const Win w = wins[wi];
      const float* A = buf + w.base;
      const int col = upd ? kfrom : k0;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int i = pt + PT * j, row = i >> 4, c4 = i & 15;
        x[j] = (r0 + row < w.rows) ? *reinterpret_cast<const float4*>(A + (int64_t)(r0 + row) * w.npad + col + 4 * c4)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto next_item = [&](int64_t from, int& wi, int& r0) -> int64_t {
      while (from < iend && !item(from, wi, r0)) ++from;
      return from;
    };
    int64_t cur[2];
    int wq[2] = {0, 0}, rq[2] = {0, 0};
    cur[0] = next_item(ibeg, wq[0], rq[0]);
    if (cur[0] < iend) load_a(wq[0], rq[0], ra[0]);
    cur[1] = cur[0] < iend ? next_item(cur[0] + 1, wq[1], rq[1]) : iend;
    if (cur[1] < iend) load_a(wq[1], rq[1], ra[1]);
    int t = 0, v = -1, wcur = -1;
    // one item from register set P: stage, then refill the set with the item two ahead
    auto step = [&](auto P) -> bool {
      constexpr int p = decltype(P)::value;
      const int wi = wq[p];
      const int s = t & 1, u = t >> 1;
      if (wi != wcur) {  // right operands of a new window
        ++v;
        wcur = wi;
        if (v >= 1 && !wait_warp(&sm.bempty, (v - 1) & 1)) return false;
        if (*abort_flag) return false;
        const Win w = wins[wi];
        const float* A = buf + w.base;
        const float* Dv = dinv + w.dinv + (int64_t)kp * TB * TB;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          const int i = pt + PT * j, row = i >> 4, c4 = i & 15;
          if (upd)
            pt_store(sm.b1, row, 4 * c4, *reinterpret_cast<const float4*>(A + (int64_t)(k0 + row) * w.npad + kfrom + 4 * c4));
          pt_store(sm.b2, row, 4 * c4, *reinterpret_cast<const float4*>(Dv + row * TB + 4 * c4));
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.bfull);
      }
      if (t >= 2 && !wait_warp(&sm.empty[s], (u - 1) & 1)) return false;
      if (*abort_flag) return false;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int i = pt + PT * j;
        pt_store(sm.a[s], i >> 4, 4 * (i & 15), ra[p][j]);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.full[s]);
      ++t;
      const int64_t after = cur[p ^ 1] < iend ? cur[p ^ 1] : iend;
      cur[p] = after < iend ? next_item(after + 1, wq[p], rq[p]) : iend;
      if (cur[p] < iend) load_a(wq[p], rq[p], ra[p]);
      return true;
    };
    while (cur[0] < iend) {
      if (!step(std::integral_constant<int, 0>{})) break;
      if (cur[1] >= iend) break;
      if (!step(std::integral_constant<int, 1>{})) break;
    }
  } else if (warp == kPtProducers) {
    // ---------------- MMA issue (whole warp loops, lane 0 issues) ----------------
    const uint32_t tmem = sm.tmem;
    int t = 0, v = -1, wcur = -1;
    int wi = 0, r0 = 0;
    int64_t i = ibeg;
    while (i < iend && !item(i, wi, r0)) ++i;
    while (i < iend) {
      int wn = 0, rn = 0;
      int64_t nx = i + 1;
      while (nx < iend && !item(nx, wn, rn)) ++nx;
      const bool last_of_window = nx >= iend || wn != wi;
      const int s = t & 1, u = t >> 1;
      const uint32_t d = tmem + 64u * (uint32_t)s;
      if (*abort_flag) break;
      if (wi != wcur) {
        ++v;
        wcur = wi;
        if (!wait_warp(&sm.bfull, v & 1)) break;
      }
      if (t >= 2 && !wait_warp(&sm.afree[s], (u - 1) & 1)) break;
      if (!wait_warp(&sm.full[s], u & 1)) break;
      fence_after_sync();
      if (upd) {
        if (lane == 0) {
          pt_mma(d, sm.a[s], sm.b1, 0u);
          mma_commit(&sm.upd[s]);
        }
        __syncwarp();
        if (!wait_warp(&sm.tfull[s], u & 1)) break;
        fence_after_sync();
      }
      if (lane == 0) {
        pt_mma(d, sm.a[s], sm.b2, 0u);
        mma_commit(&sm.sol[s]);
        mma_commit(&sm.empty[s]);
        if (last_of_window) mma_commit(&sm.bempty);
      }
      __syncwarp();
      ++t;
      i = nx;
      wi = wn;
      r0 = rn;
    }
    if (lane == 0) mma_commit(&sm.done);  // arrives once every MMA issued above has completed
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    // Tensor memory gives a row per thread; global memory is read and
    // written coalesced (lane L: row 2k + L/16 of the warp's 32, float4
    // L%16, k = 0..15), through the warp's 32 rows of xo (float4 slots
    // swizzled by the row, so that both access patterns are conflict-free).
    const int q = warp & 3;  // tensor-memory lane quadrant: rows 32q .. 32q + 31 of the item
    const uint32_t tl = sm.tmem + ((uint32_t)(q * 32) << 16);
    float4* xs = reinterpret_cast<float4*>(sm.xo) + q * 32 * 16;
    auto xs_at = [&](int r, int c4) -> float4& { return xs[r * 16 + (c4 ^ (r & 15))]; };
    const int cr = lane >> 4, cc = lane & 15;
    auto rows_to_xs = [&](int s) {  // the 64 accumulator columns of this lane's row into xo
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float x[16];
        tmem_ld16(tl + 64u * (uint32_t)s + 16u * (uint32_t)g, x);
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4)
          xs_at(lane, 4 * g + j4) = make_float4(x[4 * j4], x[4 * j4 + 1], x[4 * j4 + 2], x[4 * j4 + 3]);
      }
    };
    float4 own[16];  // the warp's rows of the current item's panel (update form), loaded one solve ahead
    auto load_own = [&](int64_t i) {
      int wi, r0;
      while (i < iend && !item(i, wi, r0)) ++i;
      if (i >= iend) return;
      const Win w = wins[wi];
      const float* src = buf + w.base + k0 + 4 * cc;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int row = r0 + 32 * q + 2 * k + cr;
        own[k] = row < w.rows ? *reinterpret_cast<const float4*>(src + (int64_t)row * w.npad)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    if (upd) load_own(ibeg);
    int t = 0;
    for (int64_t i = ibeg; i < iend; ++i) {
      int wi, r0;
      if (!item(i, wi, r0)) continue;
      const int s = t & 1, u = t >> 1;
      const Win w = wins[wi];
      if (*abort_flag) break;
      if (upd) {
        if (!wait_warp(&sm.upd[s], u & 1)) break;
        fence_after_sync();
        rows_to_xs(s);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int r = 2 * k + cr;
          const float4 b = xs_at(r, cc);
          float4 a = own[k];
          a.x -= b.x;
          a.y -= b.y;
          a.z -= b.z;
          a.w -= b.w;
          pt_store(sm.a[s], 32 * q + r, 4 * cc, a);
        }
        fence_async_smem();
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.tfull[s]);
        load_own(i + 1);  // the next item's rows, while this item is solved
      }
      if (!wait_warp(&sm.sol[s], u & 1)) break;
      fence_after_sync();
      rows_to_xs(s);
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.afree[s]);
      float* dst = buf + w.base + k0 + 4 * cc;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int r = 2 * k + cr, row = r0 + 32 * q + r;
        if (row < w.rows) *reinterpret_cast<float4*>(dst + (int64_t)row * w.npad) = xs_at(r, cc);
      }
      __syncwarp();  // xo is rewritten by the next item
      ++t;
    }
  }
  // every MMA this CTA issued has completed before its tensor memory is freed
  const bool okd = mbar_wait(&sm.done, 0);
  if ((!okd || *abort_flag) && tid == 0) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  if (warp == kPtProducers) tmem_dealloc(sm.tmem, 128);
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
// Worker warps of the persistent tensor-core products (4 lane quarters x 4
// groups of 32 columns of a 128 x 128 tile).
constexpr int kSplitWorkers = 16;

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

// Width of the 128 x RB output tiles of the compensated products.
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


}  // namespace lma
