// Right-looking blocked Cholesky of ONE FP64 matrix with appended rows, on
// 32 x 32 tiles: Sigma_SS (with identity rows appended, giving L^-T) and
// I + A of the global summary (identity rows and y appended, giving L_C^-T
// and L_C^-1 y).
//
// FP64 arithmetic is scarce on this part (a few FP64 FMAs per clock per SM),
// so a 64 x 64 x 64 FP64 tile product alone keeps one SM busy for tens of
// microseconds; 32-wide tiles cut the serial chain of diagonal factor ->
// panel solve -> trailing update by 8x per tile and spread the trailing
// update over 4x more SMs.  The diagonal tile of panel kp + 1 is factorised
// by the CTA that applies its last update (k_f64_trail), so every panel
// costs two launches.
//
// Layout: row-major, leading dimension ld = npad (the padded order, a
// multiple of 32; padding rows/columns of the matrix hold the identity);
// rows [npad, rows) are appended rows that ride along and end up as
// (L^-1 Y)^T.  The first nid appended rows are identity rows e_q^T: row
// tile e of them stays zero in every column panel k < e and is skipped there.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lma_kernels.cuh"

namespace lma {
namespace f64 {

constexpr int TS = 32;     // tile order
constexpr int NTH = 128;   // threads per CTA

struct TileSmem {
  double D[TS][TS + 1];
  double X[TS][TS + 1];
};

// True when row tile i (appended row tile e = i - npan) holds only identity
// rows that are still zero in column panel k.
__device__ __forceinline__ bool zero_identity_tile(int i, int npan, int k, int nid) {
  const int e = i - npan;
  return e > k && (e + 1) * TS <= nid;
}

// Factor of diagonal tile kp (used for the first panel; later diagonal
// tiles are factorised inside k_f64_trail).
__global__ void __launch_bounds__(NTH) k_f64_potrf(double* __restrict__ buf, int64_t ld, int kp,
                                                   double* __restrict__ dinv, int* __restrict__ info) {
  __shared__ TileSmem sm;
  double* A = buf + (int64_t)kp * TS * ld + kp * TS;
  for (int q = threadIdx.x; q < TS * TS; q += NTH) sm.D[q / TS][q % TS] = A[(int64_t)(q / TS) * ld + q % TS];
  diag_factor<double, TS>(sm.D, A, ld, dinv + (int64_t)kp * TS * TS, info, kp * TS);
}

// Panel solve: for row tiles i > kp (grid x = i - kp - 1), A[i, kp] <- A[i, kp] inv(L_kk)^T.
// Thread t computes row t / 4, columns (t mod 4) + 4 q.
__global__ void __launch_bounds__(NTH) k_f64_trsm(double* __restrict__ buf, int64_t ld, int rows, int npan, int kp,
                                                  int nid, const double* __restrict__ dinv) {
  const int i = kp + 1 + blockIdx.x;
  const int r0 = i * TS;
  if (r0 >= rows || zero_identity_tile(i, npan, kp, nid)) return;
  __shared__ double Ts[TS][TS + 1];
  __shared__ double Xs[TS][TS + 1];
  const double* Dv = dinv + (int64_t)kp * TS * TS;
  double* A = buf + (int64_t)r0 * ld + kp * TS;
  for (int q = threadIdx.x; q < TS * TS; q += NTH) {
    const int r = q / TS, c = q % TS;
    Ts[r][c] = (r0 + r < rows) ? A[(int64_t)r * ld + c] : 0.0;
    Xs[r][c] = Dv[q];
  }
  __syncthreads();
  const int r = threadIdx.x >> 2, p = threadIdx.x & 3;
  double acc[8] = {};
  for (int j = 0; j < TS; ++j) {
    const double a = Ts[r][j];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = fma(a, Xs[p + 4 * q][j], acc[q]);
  }
  if (r0 + r < rows)
#pragma unroll
    for (int q = 0; q < 8; ++q) A[(int64_t)r * ld + p + 4 * q] = acc[q];
}

// Trailing update after panel kp: tile (i, j), kp < j <= i < npan, and
// appended-row tiles (i >= npan, kp < j < npan): A_ij -= L_ik L_jk^T.  Block
// 0 is tile (kp + 1, kp + 1), which then factorises it (panel kp + 1's
// diagonal factor) and stores the factor and its inverse.
__global__ void __launch_bounds__(NTH) k_f64_trail(double* __restrict__ buf, int64_t ld, int rows, int npan, int kp,
                                                   int nid, double* __restrict__ dinv, int* __restrict__ info) {
  const int m = npan - kp - 1;
  const int t1 = m * (m + 1) / 2;
  int i, j;
  if ((int)blockIdx.x < t1) {
    int I = (int)((sqrtf(8.f * (float)blockIdx.x + 1.f) - 1.f) * 0.5f);
    while (I * (I + 1) / 2 > (int)blockIdx.x) --I;
    while ((I + 1) * (I + 2) / 2 <= (int)blockIdx.x) ++I;
    i = kp + 1 + I;
    j = kp + 1 + ((int)blockIdx.x - I * (I + 1) / 2);
  } else {
    const int q = blockIdx.x - t1;
    i = npan + q / m;
    j = kp + 1 + q % m;
  }
  const int r0 = i * TS, c0 = j * TS, k0 = kp * TS;
  if (r0 >= rows || zero_identity_tile(i, npan, kp, nid)) return;
  __shared__ TileSmem sm;   // D: L_ik, X: L_jk (then the factor's workspace)
  for (int q = threadIdx.x; q < TS * TS; q += NTH) {
    const int r = q / TS, c = q % TS;
    sm.D[r][c] = (r0 + r < rows) ? buf[(int64_t)(r0 + r) * ld + k0 + c] : 0.0;
    sm.X[r][c] = buf[(int64_t)(c0 + r) * ld + k0 + c];
  }
  __syncthreads();
  const int r = threadIdx.x >> 2, p = threadIdx.x & 3;
  double acc[8] = {};
  for (int k = 0; k < TS; ++k) {
    const double a = sm.D[r][k];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = fma(a, sm.X[p + 4 * q][k], acc[q]);
  }
  double* A = buf + (int64_t)r0 * ld + c0;
  if (blockIdx.x != 0) {
    if (r0 + r < rows)
#pragma unroll
      for (int q = 0; q < 8; ++q) A[(int64_t)r * ld + p + 4 * q] -= acc[q];
    return;
  }
  // tile (kp + 1, kp + 1): update into shared memory, factorise, store
  double v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = A[(int64_t)r * ld + p + 4 * q] - acc[q];
  __syncthreads();  // every thread has finished reading sm.D / sm.X
#pragma unroll
  for (int q = 0; q < 8; ++q) sm.D[r][p + 4 * q] = v[q];
  diag_factor<double, TS>(sm.D, A, ld, dinv + (int64_t)(kp + 1) * TS * TS, info, c0);
}

}  // namespace f64
}  // namespace lma
