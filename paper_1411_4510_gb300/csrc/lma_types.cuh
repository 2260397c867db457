// Shared constants and descriptors of the LMA kernels (host and device).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lma {

constexpr int TB = 64;     // tile edge (also the Cholesky panel width)
constexpr int NT = 256;    // threads per CTA
constexpr int KS = 16;     // K step of the SIMT tile product
constexpr int MAXD = 24;   // largest input dimension held in shared memory

// Programmatic dependent launch.  A kernel started with programmatic stream
// serialisation (launch_pdl) may become resident while the kernel before it
// in the stream is still running.  grid_dep_wait() returns once that kernel
// has completed and its writes are visible (at once when the launch had no
// such predecessor), so it must come before anything that reads or writes
// the predecessor's data; every kernel launched through launch_pdl calls it
// first.  grid_dep_launch() allows the next kernel in the stream to start
// launching; the dependent still waits in its own grid_dep_wait().
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// One factorisation problem ("window").  The window of block m is
// D_m u D^B_m (Section 3) stored in REVERSED row order: local row i is the
// global training row g_end-1-i, so the blanket D^B_m comes first and block
// m last.  Its buffer is a row-major matrix with leading dimension npad
// (n rounded up to 64):
//   rows [0, npad)          residual R (lower triangle; padding = identity)
//   rows [npad, rows)       extra rows that the sweep turns into (L^-1 Y)^T
struct Win {
  int64_t base;   // element offset of row 0 in the window buffer
  int64_t dinv;   // element offset of this window's inverted 64x64 diagonal tiles
  int64_t ew;     // element offset into the per-window vector buffer
  int64_t g_end;  // one past the last global training row of the window
  int n;          // true order of the window
  int npad;       // padded order, multiple of 64 (= leading dimension)
  int rows;       // npad + number of extra rows
  int nB;         // blanket size: block-m part is local rows [nB, n)
  int m;          // block index
  int pad_;
};

// A prediction pair (test block n, window m), m in [n-B, n].
struct Pair {
  int64_t pbase;  // element offset of this pair's RHS rows (nu x npad of window m)
  int win;        // window index m
  int u0;         // first test row of block n
  int nu;         // number of test rows in block n
  int c0, c1;     // kept window columns [c0, c1): block part for m < n, all for m == n
  int n;          // test block
};

// One requested block of the predictive covariance between test blocks n and
// n2 (Eq. vapvar on U_n x U_n2), written row-major at element `off` of the
// output.  In the band (|n - n2| <= B) the residual part sums the products of
// the right-hand sides of the pairs (n, m) and (n2, m) over the windows
// m = m_lo .. m_lo + nm - 1 (m_lo = max(0, max(n, n2) - B), up to min(n, n2));
// the pairs of one test block are consecutive in m, so pair index pa + j is
// (n, m_lo + j) and pb + j is (n2, m_lo + j).  Off the band nm = 0 and only
// the low-rank term remains.
struct CovReq {
  int64_t off;  // element offset of the block in the output
  int u0a, nua;  // test rows of block n
  int u0b, nub;  // test rows of block n2
  int pa, pb;    // pair indices of (n, m_lo) and (n2, m_lo)
  int nm;        // number of windows in the sum (0: off the band)
  int lo;        // min(n, n2): windows m < lo keep their block columns only
  int m_lo;      // first window of the sum
  int same;      // n == n2: noise on the diagonal
};

}  // namespace lma
