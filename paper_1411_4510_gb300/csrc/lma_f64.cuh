// Right-looking blocked Cholesky of ONE FP64 matrix with appended rows, on
// 16 x 16 tiles: Sigma_SS (with identity rows appended, giving L^-T) and
// I + A of the global summary (identity rows and y appended, giving L_C^-T
// and L_C^-1 y).
//
// FP64 arithmetic is scarce on this part (under two FP64 FMAs per clock per
// SM, about 65 cycles of latency each), so the factorisation is a chain of
// small latency-bound steps.  Per column panel kp one launch does
//   * every trailing tile (i, j), kp < j <= i: solve L_ik = T_ik inv(L_kk)^T
//     and L_jk the same way in the CTA, then A_ij -= L_ik L_jk^T;  the CTA
//     of tile (kp + 1, kp + 1) then factorises it (the next diagonal factor);
//   * the in-place solve L_ik = T_ik inv(L_kk)^T of every tile of panel
//     kp - 1, deferred by one launch because the trailing update of panel
//     kp - 1 read T there; nobody reads column kp - 1 any more.
// A last launch (kp = npan) solves panel npan - 1.  The result is the
// factor L (zeros above the diagonal in the diagonal tiles), the appended
// rows (L^-1 Y)^T and the inverse diagonal tiles in dinv.
//
// Layout: row-major, leading dimension ld = npad (the padded order, a
// multiple of 16; padding rows/columns of the matrix hold the identity);
// rows [npad, rows) are appended rows.  The first nid appended rows are
// identity rows e_q^T: row tile e of them stays zero in every column panel
// k < e and is skipped there.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lma_kernels.cuh"

namespace lma {
namespace f64 {

constexpr int TS = 16;     // tile order
constexpr int NTH = 64;    // threads per CTA (4 TS, as diag_factor needs)

// True when row tile i (appended row tile e = i - npan) holds only identity
// rows that are still zero in column panel k.
__device__ __forceinline__ bool zero_identity_tile(int i, int npan, int k, int nid) {
  const int e = i - npan;
  return e > k && (e + 1) * TS <= nid;
}

// Loads a TS x TS tile (rows >= rows read as zero).
__device__ __forceinline__ void load_tile(double (*dst)[TS + 1], const double* buf, int64_t ld, int r0, int c0,
                                          int rows) {
  for (int q = threadIdx.x; q < TS * TS; q += NTH) {
    const int r = q / TS, c = q % TS;
    dst[r][c] = (r0 + r < rows) ? buf[(int64_t)(r0 + r) * ld + c0 + c] : 0.0;
  }
}

// out = T X^T for a TS x TS tile (X = inv(L_kk), lower); thread t computes
// row t / 4, columns (t mod 4) + 4 q.
__device__ __forceinline__ void solve_tile(double (*out)[TS + 1], const double (*T)[TS + 1],
                                           const double (*X)[TS + 1]) {
  const int r = threadIdx.x >> 2, p = threadIdx.x & 3;
  double acc[TS / 4] = {};
#pragma unroll
  for (int k = 0; k < TS; ++k) {
    const double a = T[r][k];
#pragma unroll
    for (int q = 0; q < TS / 4; ++q) acc[q] = fma(a, X[p + 4 * q][k], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < TS / 4; ++q) out[r][p + 4 * q] = acc[q];
}

// Factor of diagonal tile kp (the first panel; later diagonal tiles are
// factorised inside k_f64_panel).
__global__ void __launch_bounds__(NTH) k_f64_potrf(double* __restrict__ buf, int64_t ld, int kp,
                                                   double* __restrict__ dinv, int* __restrict__ info) {
  grid_dep_wait();
  grid_dep_launch();
  __shared__ double D[TS][TS + 1];
  double* A = buf + (int64_t)kp * TS * ld + kp * TS;
  load_tile(D, A, ld, 0, 0, TS);
  diag_factor<double, TS>(D, A, ld, dinv + (int64_t)kp * TS * TS, info, kp * TS);
}

// One launch per column panel kp (see the file comment).  Block order:
// [0, t1) matrix tiles (kp < j <= i < npan, block 0 = (kp + 1, kp + 1)),
// [t1, t2) appended-row tiles (i >= npan, kp < j < npan),
// [t2, t2 + nrt - kp) deferred solves of row tiles kp .. nrt - 1 of panel kp - 1.
__global__ void __launch_bounds__(NTH) k_f64_panel(double* __restrict__ buf, int64_t ld, int rows, int npan, int kp,
                                                   int nid, double* __restrict__ dinv, int* __restrict__ info) {
  grid_dep_wait();
  grid_dep_launch();
  const int nrt = (rows + TS - 1) / TS, napp = nrt - npan;
  const int m = npan - kp - 1;  // trailing panels (may be <= 0)
  const int t1 = m > 0 ? m * (m + 1) / 2 : 0;
  const int t2 = t1 + (m > 0 ? napp * m : 0);
  __shared__ double Ti[TS][TS + 1], Tj[TS][TS + 1], X[TS][TS + 1];
  __shared__ double Li[TS][TS + 1], Lj[TS][TS + 1];
  const int b = blockIdx.x;
  if (b >= t2) {  // deferred solve of tile (i, kp - 1)
    const int i = kp + (b - t2), k = kp - 1;
    if (k < 0 || zero_identity_tile(i, npan, k, nid)) return;
    load_tile(Ti, buf, ld, i * TS, k * TS, rows);
    load_tile(X, dinv + (int64_t)k * TS * TS, TS, 0, 0, TS);
    __syncthreads();
    solve_tile(Li, Ti, X);
    __syncthreads();
    for (int q = threadIdx.x; q < TS * TS; q += NTH) {
      const int r = q / TS, c = q % TS;
      if (i * TS + r < rows) buf[(int64_t)(i * TS + r) * ld + k * TS + c] = Li[r][c];
    }
    return;
  }
  int i, j;
  if (b < t1) {
    int I = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
    while (I * (I + 1) / 2 > b) --I;
    while ((I + 1) * (I + 2) / 2 <= b) ++I;
    i = kp + 1 + I;
    j = kp + 1 + (b - I * (I + 1) / 2);
  } else {
    const int q = b - t1;
    i = npan + q / m;
    j = kp + 1 + q % m;
  }
  const int r0 = i * TS, c0 = j * TS, k0 = kp * TS;
  if (zero_identity_tile(i, npan, kp, nid)) return;
  load_tile(Ti, buf, ld, r0, k0, rows);
  load_tile(X, dinv + (int64_t)kp * TS * TS, TS, 0, 0, TS);
  if (i != j) load_tile(Tj, buf, ld, c0, k0, rows);
  __syncthreads();
  solve_tile(Li, Ti, X);
  if (i != j) solve_tile(Lj, Tj, X);
  __syncthreads();
  const double(*LJ)[TS + 1] = (i != j) ? Lj : Li;
  const int r = threadIdx.x >> 2, p = threadIdx.x & 3;
  double acc[TS / 4] = {};
#pragma unroll
  for (int k = 0; k < TS; ++k) {
    const double a = Li[r][k];
#pragma unroll
    for (int q = 0; q < TS / 4; ++q) acc[q] = fma(a, LJ[p + 4 * q][k], acc[q]);
  }
  double* A = buf + (int64_t)r0 * ld + c0;
  if (b != 0) {
    if (r0 + r < rows)
#pragma unroll
      for (int q = 0; q < TS / 4; ++q) A[(int64_t)r * ld + p + 4 * q] -= acc[q];
    return;
  }
  // tile (kp + 1, kp + 1): update into shared memory, factorise, store
#pragma unroll
  for (int q = 0; q < TS / 4; ++q) Tj[r][p + 4 * q] = A[(int64_t)r * ld + p + 4 * q] - acc[q];
  diag_factor<double, TS>(Tj, A, ld, dinv + (int64_t)(kp + 1) * TS * TS, info, c0);
}

// Two-phase variant (two launches per column panel, no repeated solves):
// k_f64_solve2 solves every tile of panel kp below the diagonal in place,
// L_ik = T_ik inv(L_kk)^T (identity-row tiles that are still zero are
// skipped); k_f64_update2 then applies A_ij -= L_ik L_jk^T to every trailing
// tile (kp < j <= i < npan, and the appended-row tiles i >= npan, kp < j <
// npan) from the solved tiles, and its CTA 0 (tile (kp + 1, kp + 1))
// factorises that diagonal tile.  Each trailing tile thus does one product
// instead of two solves and a product, which pays at large orders.
__global__ void __launch_bounds__(NTH) k_f64_solve2(double* __restrict__ buf, int64_t ld, int rows, int npan, int kp,
                                                    int nid, const double* __restrict__ dinv) {
  grid_dep_wait();
  grid_dep_launch();
  const int i = kp + 1 + blockIdx.x;
  if (zero_identity_tile(i, npan, kp, nid)) return;
  __shared__ double Ti[TS][TS + 1], X[TS][TS + 1], Li[TS][TS + 1];
  load_tile(Ti, buf, ld, i * TS, kp * TS, rows);
  load_tile(X, dinv + (int64_t)kp * TS * TS, TS, 0, 0, TS);
  __syncthreads();
  solve_tile(Li, Ti, X);
  __syncthreads();
  for (int q = threadIdx.x; q < TS * TS; q += NTH) {
    const int r = q / TS, c = q % TS;
    if (i * TS + r < rows) buf[(int64_t)(i * TS + r) * ld + kp * TS + c] = Li[r][c];
  }
}

__global__ void __launch_bounds__(NTH) k_f64_update2(double* __restrict__ buf, int64_t ld, int rows, int npan,
                                                     int kp, int nid, double* __restrict__ dinv,
                                                     int* __restrict__ info) {
  grid_dep_wait();
  grid_dep_launch();
  const int napp = (rows + TS - 1) / TS - npan;
  const int m = npan - kp - 1;
  const int t1 = m * (m + 1) / 2;
  const int b = blockIdx.x;
  int i, j;
  if (b < t1) {
    int I = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
    while (I * (I + 1) / 2 > b) --I;
    while ((I + 1) * (I + 2) / 2 <= b) ++I;
    i = kp + 1 + I;
    j = kp + 1 + (b - I * (I + 1) / 2);
  } else {
    const int q = b - t1;
    if (q >= napp * m) return;
    i = npan + q / m;
    j = kp + 1 + q % m;
  }
  if (zero_identity_tile(i, npan, kp, nid)) return;
  __shared__ double Li[TS][TS + 1], Lj[TS][TS + 1], Tj[TS][TS + 1];
  const int r0 = i * TS, c0 = j * TS, k0 = kp * TS;
  load_tile(Li, buf, ld, r0, k0, rows);
  if (i != j) load_tile(Lj, buf, ld, c0, k0, rows);
  __syncthreads();
  const double(*LJ)[TS + 1] = (i != j) ? Lj : Li;
  const int r = threadIdx.x >> 2, p = threadIdx.x & 3;
  double acc[TS / 4] = {};
#pragma unroll
  for (int k = 0; k < TS; ++k) {
    const double a = Li[r][k];
#pragma unroll
    for (int qq = 0; qq < TS / 4; ++qq) acc[qq] = fma(a, LJ[p + 4 * qq][k], acc[qq]);
  }
  double* A = buf + (int64_t)r0 * ld + c0;
  if (b != 0) {
    if (r0 + r < rows)
#pragma unroll
      for (int qq = 0; qq < TS / 4; ++qq) A[(int64_t)r * ld + p + 4 * qq] -= acc[qq];
    return;
  }
#pragma unroll
  for (int qq = 0; qq < TS / 4; ++qq) Tj[r][p + 4 * qq] = A[(int64_t)r * ld + p + 4 * qq] - acc[qq];
  diag_factor<double, TS>(Tj, A, ld, dinv + (int64_t)(kp + 1) * TS * TS, info, c0);
}

// ---------------------------------------------------------------------------
// Persistent form: the whole right-looking factorisation in ONE cooperative
// launch (all CTAs resident), the launch boundaries of the two-phase form
// replaced by grid barriers.  At order 512 the two-phase form is 64 launches
// of a few microseconds of work each, so launch latency, not the FP64 pipe,
// set its time.  Per column panel kp:
//   solve phase   every tile (i, kp), i > kp, becomes T_ik inv(L_kk)^T;
//   barrier;
//   update phase  A_ij -= L_ik L_jk^T over the trailing tiles, CTA 0 taking
//                 tile (kp + 1, kp + 1) first and factorising it;
//   barrier.
// Tiles are dealt to CTAs round-robin.  Data written by other CTAs during
// the launch is read with ld.global.cg (L2), never through L1.

constexpr uint32_t kBarrierSpin = 1u << 22;  // polls before a grid barrier gives up

// Grid-wide barrier: *bar (zero before the launch) counts arrivals, barrier
// number g completes at g * gridDim.x.  Gives up after kBarrierSpin polls or
// once another CTA gave up (*err != 0), setting *err; returns false then.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& gen, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = ++gen * gridDim.x;
    __threadfence();
    atomicAdd(bar, 1u);
    int good = 1;
    for (uint32_t it = 0;; ++it) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (it >= kBarrierSpin || ((it & 1023u) == 1023u && *(volatile int*)err)) {
        good = 0;
        atomicExch(err, 1);
        break;
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// load_tile through L2 (the tile may have been written by another CTA).
__device__ __forceinline__ void load_tile_cg(double (*dst)[TS + 1], const double* buf, int64_t ld, int r0, int c0,
                                             int rows) {
  for (int q = threadIdx.x; q < TS * TS; q += NTH) {
    const int r = q / TS, c = q % TS;
    dst[r][c] = (r0 + r < rows) ? __ldcg(buf + (int64_t)(r0 + r) * ld + c0 + c) : 0.0;
  }
}

__global__ void __launch_bounds__(NTH) k_f64_coop(double* buf, int64_t ld, int rows, int npan, int nid,
                                                  double* dinv, int* info, unsigned* bar, int* err) {
  __shared__ double Ti[TS][TS + 1], X[TS][TS + 1], Li[TS][TS + 1], Lj[TS][TS + 1];
  const int G = gridDim.x, nrt = (rows + TS - 1) / TS, napp = nrt - npan;
  const int r = threadIdx.x >> 2, p = threadIdx.x & 3;
  unsigned gen = 0;
  if (blockIdx.x == 0) {
    load_tile_cg(Ti, buf, ld, 0, 0, rows);
    diag_factor<double, TS>(Ti, buf, ld, dinv, info, 0);
  }
  if (!grid_barrier(bar, gen, err)) return;
  for (int kp = 0; kp < npan; ++kp) {
    // solve phase
    for (int t = blockIdx.x; t < nrt - kp - 1; t += G) {
      const int i = kp + 1 + t;
      if (zero_identity_tile(i, npan, kp, nid)) continue;
      load_tile_cg(Ti, buf, ld, i * TS, kp * TS, rows);
      load_tile_cg(X, dinv + (int64_t)kp * TS * TS, TS, 0, 0, TS);
      __syncthreads();
      solve_tile(Li, Ti, X);
      __syncthreads();
      for (int q = threadIdx.x; q < TS * TS; q += NTH) {
        const int rr = q / TS, c = q % TS;
        if (i * TS + rr < rows) buf[(int64_t)(i * TS + rr) * ld + kp * TS + c] = Li[rr][c];
      }
      __syncthreads();
    }
    const int m = npan - kp - 1;
    if (m <= 0) break;
    if (!grid_barrier(bar, gen, err)) return;
    // update phase
    const int t1 = m * (m + 1) / 2, total = t1 + napp * m;
    for (int b = blockIdx.x; b < total; b += G) {
      int i, j;
      if (b < t1) {
        int I = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
        while (I * (I + 1) / 2 > b) --I;
        while ((I + 1) * (I + 2) / 2 <= b) ++I;
        i = kp + 1 + I;
        j = kp + 1 + (b - I * (I + 1) / 2);
      } else {
        const int q = b - t1;
        i = npan + q / m;
        j = kp + 1 + q % m;
      }
      if (zero_identity_tile(i, npan, kp, nid)) continue;
      const int r0 = i * TS, c0 = j * TS, k0 = kp * TS;
      load_tile_cg(Li, buf, ld, r0, k0, rows);
      if (i != j) load_tile_cg(Lj, buf, ld, c0, k0, rows);
      __syncthreads();
      const double(*LJ)[TS + 1] = (i != j) ? Lj : Li;
      double acc[TS / 4] = {};
#pragma unroll
      for (int k = 0; k < TS; ++k) {
        const double a = Li[r][k];
#pragma unroll
        for (int qq = 0; qq < TS / 4; ++qq) acc[qq] = fma(a, LJ[p + 4 * qq][k], acc[qq]);
      }
      double* A = buf + (int64_t)r0 * ld + c0;
      if (b != 0) {
        if (r0 + r < rows)
#pragma unroll
          for (int qq = 0; qq < TS / 4; ++qq) {
            double* a = A + (int64_t)r * ld + p + 4 * qq;
            *a = __ldcg(a) - acc[qq];
          }
      } else {
#pragma unroll
        for (int qq = 0; qq < TS / 4; ++qq) Ti[r][p + 4 * qq] = __ldcg(A + (int64_t)r * ld + p + 4 * qq) - acc[qq];
        diag_factor<double, TS>(Ti, A, ld, dinv + (int64_t)(kp + 1) * TS * TS, info, c0);
      }
      __syncthreads();
    }
    if (!grid_barrier(bar, gen, err)) return;
  }
}

// ---------------------------------------------------------------------------
// Dataflow form (one cooperative launch).  Tile (i, j) of the lower part,
// appended-row tiles included and identity-row tiles that stay zero left
// out, is owned by one CTA.  The owner applies A_ij -= L_ik L_jk^T for
// k = 0 .. j-1 as the tiles (i, k) and (j, k) become final (one flag per
// tile), then factorises the tile (i = j) or solves it against inv(L_jj)
// (i > j) and publishes it.  The tiles are listed column by column and a
// CTA takes its tiles in list order; every wait is for a tile earlier in the
// list, so with all CTAs resident every wait ends (by induction on the list
// position).  The critical path is the chain of diagonal factorisations and
// the solves and updates between them, not a launch per column panel.

// Waits (thread 0) until *f is set; false on timeout or once another CTA gave up.
__device__ __forceinline__ bool wait_flag(const unsigned* f, int* err) {
  for (uint32_t it = 0;; ++it) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    if (v) return true;
    if (it >= kBarrierSpin || ((it & 1023u) == 1023u && *(volatile int*)err)) {
      atomicExch(err, 1);
      return false;
    }
  }
}

__global__ void __launch_bounds__(NTH) k_f64_flow(double* buf, int64_t ld, int rows, int npan, int nid, double* dinv,
                                                  int* info, const int2* __restrict__ tiles, int ntiles,
                                                  unsigned* flags, int* err) {
  __shared__ double Li[TS][TS + 1], Lj[TS][TS + 1], Tm[TS][TS + 1];
  __shared__ int ok;
  const int r = threadIdx.x >> 2, p = threadIdx.x & 3;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i = tiles[t].x, j = tiles[t].y;
    const int r0 = i * TS, c0 = j * TS;
    double* A = buf + (int64_t)r0 * ld + c0;
    double acc[TS / 4];
#pragma unroll
    for (int q = 0; q < TS / 4; ++q) acc[q] = (r0 + r < rows) ? __ldcg(A + (int64_t)r * ld + p + 4 * q) : 0.0;
    for (int k = 0; k < j; ++k) {
      if (zero_identity_tile(i, npan, k, nid)) continue;  // L_ik is still zero
      if (threadIdx.x == 0) {
        bool w = wait_flag(flags + (int64_t)i * npan + k, err);
        if (w && i != j) w = wait_flag(flags + (int64_t)j * npan + k, err);
        __threadfence();
        ok = w;
      }
      __syncthreads();
      if (!ok) return;
      load_tile_cg(Li, buf, ld, r0, k * TS, rows);
      if (i != j) load_tile_cg(Lj, buf, ld, c0, k * TS, rows);
      __syncthreads();
      const double(*LJ)[TS + 1] = (i != j) ? Lj : Li;
#pragma unroll
      for (int kk = 0; kk < TS; ++kk) {
        const double a = Li[r][kk];
#pragma unroll
        for (int q = 0; q < TS / 4; ++q) acc[q] = fma(-a, LJ[p + 4 * q][kk], acc[q]);
      }
      __syncthreads();
    }
    if (i == j) {
#pragma unroll
      for (int q = 0; q < TS / 4; ++q) Tm[r][p + 4 * q] = acc[q];
      diag_factor<double, TS>(Tm, A, ld, dinv + (int64_t)j * TS * TS, info, c0);
    } else {
      if (threadIdx.x == 0) {
        const bool w = wait_flag(flags + (int64_t)j * npan + j, err);
        __threadfence();
        ok = w;
      }
#pragma unroll
      for (int q = 0; q < TS / 4; ++q) Tm[r][p + 4 * q] = acc[q];
      __syncthreads();
      if (!ok) return;
      load_tile_cg(Lj, dinv + (int64_t)j * TS * TS, TS, 0, 0, TS);
      __syncthreads();
      solve_tile(Li, Tm, Lj);
      __syncthreads();
      for (int q = threadIdx.x; q < TS * TS; q += NTH) {
        const int rr = q / TS, c = q % TS;
        if (r0 + rr < rows) A[(int64_t)rr * ld + c] = Li[rr][c];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flags + (int64_t)i * npan + j), "r"(1u) : "memory");
    }
  }
}

}  // namespace f64
}  // namespace lma
