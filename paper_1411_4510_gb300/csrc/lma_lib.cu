// Fit / predict pipelines of the LMA hot path, instantiated for float (mixed
// form) and double (plain FP64 form).
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "lma_impl.cuh"
#include "lma_kernels.cuh"
#include "lma_grad.cuh"
#include "lma_tc.cuh"
#include "lma_grad_tc.cuh"
#include "lma_bf6.cuh"
#include "lma_f64.cuh"
#include "lma_tune.cuh"

namespace lma {

// ---------------------------------------------------------------------------
void make_windows(const std::vector<int64_t>& bptr, int64_t B, int64_t s, size_t /*elem*/, std::vector<Win>& wins,
                  int64_t& buf_elems, int64_t& dinv_elems, int64_t& ew_elems, int64_t m_begin, int64_t m_end,
                  const std::vector<int>* test_rows) {
  const int64_t M = (int64_t)bptr.size() - 1;
  if (m_end < 0) m_end = M;
  wins.resize(m_end - m_begin);
  buf_elems = dinv_elems = ew_elems = 0;
  for (int64_t m = m_begin; m < m_end; ++m) {
    const int64_t last = std::min(m + B, M - 1);
    Win w{};
    w.n = (int)(bptr[last + 1] - bptr[m]);
    w.nB = (int)(bptr[last + 1] - bptr[m + 1]);
    w.npad = (int)roundup(w.n, TB);
    w.rows = (int)(w.npad + s + 1) + (test_rows ? (*test_rows)[m] : 0);
    w.g_end = bptr[last + 1];
    w.m = (int)m;
    w.base = buf_elems;
    w.dinv = dinv_elems;
    w.ew = ew_elems;
    buf_elems += (int64_t)w.rows * w.npad;
    dinv_elems += (int64_t)(w.npad / TB) * TB * TB;
    ew_elems += w.npad;
    wins[m - m_begin] = w;
  }
}

void make_pairs(const std::vector<Win>& wins, int64_t w0, int64_t M, int64_t B, int64_t s, const int64_t* tptr,
                bool fused, std::vector<Pair>& pairs, std::vector<int4>& tb, int64_t* p_elems) {
  std::vector<int> used(wins.size(), 0);  // test rows already placed in each window (fused)
  int64_t pe = 0;
  for (int64_t nb = 0; nb < M; ++nb) {
    const int nu = (int)(tptr[nb + 1] - tptr[nb]);
    if (nu == 0) continue;
    const int first = (int)pairs.size();
    for (int64_t m = std::max<int64_t>(0, nb - B); m <= nb; ++m) {
      const Win& w = wins[m - w0];
      Pair p{};
      if (fused) {
        p.pbase = w.base + (int64_t)(w.npad + s + 1 + used[m - w0]) * w.npad;
        used[m - w0] += nu;
      } else {
        p.pbase = pe;
        pe += (int64_t)nu * w.npad;
      }
      p.win = (int)(m - w0);
      p.u0 = (int)tptr[nb];
      p.nu = nu;
      p.c0 = (m < nb) ? w.nB : 0;
      p.c1 = w.n;
      p.n = (int)nb;
      pairs.push_back(p);
    }
    tb.push_back(make_int4(first, (int)pairs.size() - first, (int)tptr[nb], nu));
  }
  if (p_elems) *p_elems = pe;
}

std::vector<int> fused_test_rows(int64_t M, int64_t B, const int64_t* tptr) {
  std::vector<int> rows(M, 0);
  for (int64_t nb = 0; nb < M; ++nb)
    for (int64_t m = std::max<int64_t>(0, nb - B); m <= nb; ++m) rows[m] += (int)(tptr[nb + 1] - tptr[nb]);
  return rows;
}

void* Staging::take(size_t bytes, cudaStream_t st) {
  (void)st;
  bytes = (bytes + 255) & ~size_t(255);
  if (used + bytes > cap) {
    if (hold) {
      // enqueued calls' uploads may still be in flight: every earlier upload
      // (of any stream of this thread) must have landed before reuse
      LMA_CK(cudaDeviceSynchronize());
      hold = false;
      reset();
    }
    if (used + bytes > cap) {
      // a larger buffer; the outgrown one stays until the next reset (its
      // uploads may still be in flight), so a call never waits for the GPU here
      if (base) retired.push_back(base);
      base = nullptr;
      cap = std::max<size_t>({bytes, 2 * cap, size_t(1) << 20});
      LMA_CK(cudaMallocHost((void**)&base, cap));
      used = 0;
    }
  }
  void* p = base + used;
  used += bytes;
  return p;
}

void Staging::reset() {
  if (hold) return;
  used = 0;
  for (char* b : retired) cudaFreeHost(b);
  retired.clear();
}

namespace {
struct FitWorkspace {
  void* p = nullptr;
  size_t cap = 0;
};
FitWorkspace& fit_ws() {
  static thread_local FitWorkspace ws[64];
  int dev = 0;
  LMA_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    fail(LMA_ERR_INTERNAL, "device index out of range");
    throw Fail{};
  }
  return ws[dev];
}
}  // namespace

void* fit_workspace(size_t bytes) {
  FitWorkspace& w = fit_ws();
  if (bytes > w.cap) {
    if (w.p) {
      LMA_CK(cudaDeviceSynchronize());  // the previous calls' work on it has completed anyway
      LMA_CK(cudaFree(w.p));
      w.p = nullptr;
      w.cap = 0;
    }
    if (cudaMalloc(&w.p, bytes) != cudaSuccess) {
      // the stream-ordered pool keeps freed memory (release threshold at
      // its maximum): hand it back and try once more
      cudaGetLastError();
      w.p = nullptr;
      int dev = 0;
      cudaMemPool_t pool;
      LMA_CK(cudaGetDevice(&dev));
      LMA_CK(cudaDeviceSynchronize());
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
      LMA_CK(cudaMalloc(&w.p, bytes));
    }
    w.cap = bytes;
  }
  return w.p;
}

void fit_workspace_release() {
  FitWorkspace& w = fit_ws();
  if (w.p) {
    LMA_CK(cudaDeviceSynchronize());
    LMA_CK(cudaFree(w.p));
  }
  w.p = nullptr;
  w.cap = 0;
}

Staging& staging() {
  static thread_local Staging s;
  return s;
}

static size_t tc_chol_smem() { return sizeof(tc::TcSmem<64>) + tc::kTcAlignSlack; }
static size_t pt_smem() { return sizeof(tc::PtSmem) + tc::kTcAlignSlack; }

template <int BN>
static size_t wide_smem() { return sizeof(tc::WsSmem<2, BN>) + tc::kTcAlignSlack; }
static size_t tc_resid_smem() { return sizeof(CompSmem<RB>) + tc::kTcAlignSlack; }

// Grid of a persistent kernel with one CTA per SM: min(items, SM count).
static unsigned persistent_grid(size_t items) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    LMA_CK(cudaGetDevice(&dev));
    LMA_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  return (unsigned)std::max<size_t>(1, std::min<size_t>(items, (size_t)nsm));
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of row-major bfloat16 planes (rows x cols, cols a multiple of
// 64, 16-byte-aligned base): 64 x 128 boxes, 128-byte swizzle; rows outside
// [0, rows) read zero.
static CUtensorMap bf16_tensor_map(const uint16_t* base, int64_t rows, int cols) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) {
    fail(LMA_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    throw Fail{};
  }
  CUtensorMap m;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)cols * sizeof(uint16_t)};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(base), gdim, gstride, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fail(LMA_ERR_CUDA, "cuTensorMapEncodeTiled (bfloat16) failed (" + std::to_string((int)r) + ")");
    throw Fail{};
  }
  return m;
}

// out[p][i] = sum_{k <= i} A[p][k] Linv[i][k] (p < nrows, i < s) on the tensor
// cores with the bf16x6 split (lma_bf6.cuh): A and Linv given as three
// bfloat16 planes (nrows and brows rows per plane, row length ldk).
static void proj_tc(cudaStream_t st, const char* name, const uint16_t* Ap, int64_t nrows, const uint16_t* Bp,
                    int brows, int s, int ldk, float* out, int64_t ldo, int* err) {
  if (nrows == 0) return;
  const CUtensorMap am = bf16_tensor_map(Ap, 3 * nrows, ldk), bm = bf16_tensor_map(Bp, 3 * (int64_t)brows, ldk);
  const int64_t nct = (s + 127) / 128, ntiles = ((nrows + 127) / 128) * nct;
  const int64_t nitems = (nct % 2) ? ntiles : ntiles / 2;  // tiles come in pairs when nct is even (k_proj_tc)
  launch(name, k_proj_tc, persistent_grid((size_t)nitems), bf6::NTHR, bf6::smem_bytes(), st, am, (int)nrows, bm,
         brows, nrows, s, out, ldo, err);
}

// Whitened support coordinates of npts points given by their scaled inputs
// xsP (npts x d): out[p][i] = (L_SS^-1 Sigma_{S p})_i, point-major with row
// length s (H3: V = L_SS^-1 Sigma_SD).  Mixed form on the tensor cores: the
// covariances are evaluated straight into bfloat16 planes and multiplied by
// the planes of L_SS^-1 (bf16x6); otherwise K_SD is formed and multiplied by
// ET = L_SS^-T on the CUDA cores.
template <typename T>
static void project(const ModelCore& mc, const T* xsP, int64_t npts, T* out, Arena& tmp, cudaStream_t st, int* err,
                    bool use_workspace = false) {
  const int64_t s = mc.s;
  const int d = (int)mc.d;
  if (npts == 0) return;
  if (sizeof(T) == 4 && mc.linv3) {
    const size_t nA = (size_t)3 * npts * mc.ldk;
    uint16_t* Ap = use_workspace ? (uint16_t*)fit_workspace(nA * sizeof(uint16_t)) : tmp.alloc<uint16_t>(nA);
    launch("k_kds_bf3", pad_dim(d) == 8 ? k_kds_bf3<8> : k_kds_bf3<MAXD>, dim3((unsigned)(mc.ldk / 64), nblk(npts, 32)),
           256, 0, st, (const float*)xsP, npts, d, (const float*)mc.ssT, (int)s, (float)mc.ss2, mc.ldk, Ap);
    proj_tc(st, "k_proj_tc", Ap, npts, mc.linv3, mc.brows, (int)s, mc.ldk, (float*)out, s, err);
    if (!use_workspace) tmp.free_one(Ap);
    return;
  }
  T* Kds = tmp.alloc<T>(npts * s);
  launch("k_kds", k_kds<T>, dim3(nblk(s, TB), nblk(npts, TB)), NT, 0, st, xsP, npts, d, (const T*)mc.ssT, (int)s,
         (T)mc.ss2, Kds);
  if (sizeof(T) == 4 && s % 4 == 0)
    launch("k_proj", k_proj128, dim3(nblk(s, 128), nblk(npts, 128)), NT, 0, st, (const float*)Kds, npts, (int)s,
           (const float*)mc.ET, (float*)out, (int)s);
  else
    launch("k_proj", k_proj<T>, dim3(nblk(s, TB), nblk(npts, TB)), NT, 0, st, (const T*)Kds, npts, (int)s,
           (const T*)mc.ET, out, (int)s);
  tmp.free_one(Kds);
}

// Three bfloat16 planes (k_split_bf3) of the point-major rows of V (n x s),
// row length ld (s rounded up to 64, zero pad), reversed or not.
static uint16_t* split_rows_bf3(cudaStream_t st, const float* V, int64_t n, int64_t s, int ld, bool reverse,
                                uint16_t* out) {
  launch("k_split_bf3", k_split_bf3, nblk(n * (ld / 8)), NT, 0, st, V, n, (int)s, (int64_t)s, ld, out,
         reverse ? 1 : 0);
  return out;
}

// Tensor cores for the mixed form's sweep; LMA_NO_TENSOR_CORES=1 selects the
// SIMT kernels instead (used to compare the two on the same build).
static bool use_tensor_cores() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("LMA_NO_TENSOR_CORES");
    v = (e && e[0] == '1') ? 0 : 1;
  }
  return v == 1;
}

template <typename T>
static void set_smem_attr() {
  cudaFuncSetAttribute(k_chol_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CholSmem<T>));
  cudaFuncSetAttribute(k_chol_trsm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrsmSmem<T>));
  cudaFuncSetAttribute(k_pred_sweep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CholSmem<T>));
  cudaFuncSetAttribute(k_bwd_sweep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CholSmem<T>));
}

template <typename T>
void Impl<T>::setup_attributes() {
  static bool done = false;
  if (!done) {
    set_smem_attr<T>();
    set_smem_attr<double>();
    cudaFuncSetAttribute(k_chol_step_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_chol_smem());
    cudaFuncSetAttribute(k_chol_panel_pt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pt_smem());
    cudaFuncSetAttribute(k_pred_sweep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_chol_smem());
    cudaFuncSetAttribute(k_gram_bf6, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bf6::smem_bytes());
    cudaFuncSetAttribute(k_resid_bf6<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bf6::smem_bytes());
    cudaFuncSetAttribute(k_resid_bf6<MAXD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bf6::smem_bytes());
    cudaFuncSetAttribute(k_pred_rhs_bf6<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bf6::smem_bytes());
    cudaFuncSetAttribute(k_pred_rhs_bf6<MAXD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bf6::smem_bytes());
    cudaFuncSetAttribute(k_pred_accum_win, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_resid_smem());
    cudaFuncSetAttribute(k_chol_wide<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wide_smem<256>());
    cudaFuncSetAttribute(k_chol_wide<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wide_smem<128>());
    cudaFuncSetAttribute(k_proj_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bf6::smem_bytes());
    cudaFuncSetAttribute(k_grad_rhs_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_chol_smem());
    cudaFuncSetAttribute(k_bwd_sweep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_chol_smem());
    cudaFuncSetAttribute(k_grad_G_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_chol_smem());
    cudaFuncSetAttribute(k_grad_gv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_chol_smem());
    done = true;
  }
}

// Left-looking sweep over all column panels.  batched: every window in
// each launch; otherwise one window per launch (the plain form).  With the
// tensor cores (tc_err != nullptr) the panels are grouped in super-panels of
// 256 columns: one wide update applies all columns left of the super-panel
// (N = 256 tiles), the 64-wide panel steps add the rest.
template <typename T>
void chol_sweep(cudaStream_t st, const std::vector<Win>& wins, Win* wins_d, T* buf, T* dinv, int* info, bool batched,
                int* tc_err) {
  if (wins.empty()) return;
  if (batched) {
    int maxpan = 0, maxrt = 0;
    for (const Win& w : wins) {
      maxpan = std::max(maxpan, w.npad / TB);
      maxrt = std::max(maxrt, (w.rows + TB - 1) / TB);
    }
    const unsigned nw = (unsigned)wins.size();
    int maxrows = 0;
    for (const Win& w : wins) maxrows = std::max(maxrows, w.rows);
    const bool tc = tc_err && sizeof(T) == 4;
    constexpr int SP = 256, HP = 128;
    for (int kp = 0; kp < maxpan; ++kp) {
      const int k0 = kp * TB;
      if (tc) {
        // columns [0, kb) of super-panel [kb, kb + 256) come from the 256-wide
        // update, [kb, kh) of its second half from the 128-wide one, and the
        // 64-wide panel step adds [kh, k0) (at most 64 columns)
        const int kb = (k0 / SP) * SP, kh = (k0 / HP) * HP;
        if (k0 == kb && kb > 0) {
          const unsigned gy = (unsigned)((maxrows - kb + 127) / 128);
          launch_pdl("k_chol_wide", k_chol_wide<256>, dim3(nw, gy), tc::kWsThreads, wide_smem<256>(), st, wins_d,
                     (float*)buf, kb, 0, tc_err);
        }
        if (k0 == kh && kh > kb) {
          const unsigned gy = (unsigned)((maxrows - kh + 127) / 128);
          launch_pdl("k_chol_mid", k_chol_wide<128>, dim3(nw, gy), tc::kWsThreads, wide_smem<128>(), st, wins_d,
                     (float*)buf, kh, kb, tc_err);
        }
        // every panel: its diagonal block (the first panel of a 128-column
        // group has every column to its left applied; the second adds the
        // first's 64 columns), then the persistent kernel updates the rows
        // below with the same columns and solves them
        launch_pdl("k_chol_step_tc", k_chol_step_tc, dim3(nw, 1), 256, tc_chol_smem(), st, wins_d, (float*)buf,
                   (float*)dinv, info, kp, kh, tc_err);
        if (maxrows - (kp + 1) * TB > 0) {
          const int ntile = (maxrows - (kp + 1) * TB + 127) / 128;
          launch_pdl("k_chol_panel_pt", k_chol_panel_pt, persistent_grid((size_t)ntile * nw), tc::kPtThreads,
                     pt_smem(), st, wins_d, (int)nw, (float*)buf, (const float*)dinv, kp, kh, ntile, tc_err);
        }
      } else {
        launch("k_chol_step", k_chol_step<T>, dim3(maxrt - kp, nw), NT, sizeof(CholSmem<T>), st, wins_d, buf, dinv,
               info, kp);
        if (maxrt - kp - 1 > 0)
          launch("k_chol_trsm", k_chol_trsm<T>, dim3(maxrt - kp - 1, nw), NT, sizeof(TrsmSmem<T>), st, wins_d, buf,
                 dinv, kp, 0);
      }
    }
  } else {
    for (size_t wi = 0; wi < wins.size(); ++wi) {
      const Win& w = wins[wi];
      const int npan = w.npad / TB, rt = (w.rows + TB - 1) / TB;
      for (int kp = 0; kp < npan; ++kp) {
        launch("k_chol_step", k_chol_step<T>, dim3(rt - kp, 1), NT, sizeof(CholSmem<T>), st, wins_d + wi, buf, dinv, info + wi, kp);
        if (rt - kp - 1 > 0) {
          launch("k_chol_trsm", k_chol_trsm<T>, dim3(rt - kp - 1, 1), NT, sizeof(TrsmSmem<T>), st, wins_d + wi, buf, dinv, kp,
                 0);
        }
      }
    }
  }
}

// Right-looking factorisation of one FP64 matrix on 16 x 16 tiles (see
// lma_f64.cuh).  nid: number of leading appended rows that are identity rows
// (0 = none).  wd is unused (kept for the window form's signature).
// variant 0: one launch per panel (trailing tiles solve their panel tiles
// themselves; fewest launches, for small orders where the chain is
// latency-bound); variant 1: a solve launch and an update launch per panel
// (each panel tile solved once; for large orders where the FP64 work counts).
// CTAs of a cooperative FP64 kernel that can be resident at once on this
// device (which = 0: k_f64_coop, 1: k_f64_flow).
static int coop_capacity(int which = 0) {
  static int cap[64][2] = {};
  int dev = 0;
  LMA_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return 0;
  if (!cap[dev][which]) {
    int nb = 0, sms = 0;
    if (which == 0)
      LMA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f64::k_f64_coop, f64::NTH, 0));
    else
      LMA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f64::k_f64_flow, f64::NTH, 0));
    LMA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cap[dev][which] = std::max(1, nb * sms);
  }
  return cap[dev][which];
}

// Tiles of the dataflow form, column by column (see k_f64_flow).
static std::vector<int2> flow_tiles(int npan, int nrt, int nid) {
  std::vector<int2> t;
  for (int j = 0; j < npan; ++j)
    for (int i = j; i < nrt; ++i) {
      const int e = i - npan;
      if (e > j && (e + 1) * f64::TS <= nid) continue;  // identity-row tile that stays zero
      t.push_back(make_int2(i, j));
    }
  return t;
}

// Launch variants: 0 one launch per panel (k_f64_panel), 1 two launches per
// panel (k_f64_solve2 + k_f64_update2), 2-4 one cooperative launch
// (k_f64_coop) with 1, 2 or 4 CTAs per SM, 5 the dataflow form (k_f64_flow,
// as many CTAs as fit).  `bar` (a zeroed counter for k_f64_coop; npan x nrt
// zeroed tile flags for k_f64_flow, whose tile list goes to `tl`) and `err`
// (set on a wait timeout) serve the cooperative forms.
static void right_looking_fp64(cudaStream_t st, const Win& w, Win* wd, double* buf, double* dv, int* info,
                               int nid = 0, int variant = 0, unsigned* bar = nullptr, int* err = nullptr,
                               int2* tl = nullptr) {
  (void)wd;
  using namespace f64;
  const int npan = w.npad / TS, nrt = (w.rows + TS - 1) / TS;
  const int64_t ld = w.npad;
  if (variant == 5) {
    const std::vector<int2> tiles = flow_tiles(npan, nrt, nid);
    const int G = std::max(1, std::min(coop_capacity(1), (int)tiles.size()));
    stage_copy(tl, tiles.data(), sizeof(int2) * tiles.size(), st);
    LMA_CK(cudaMemsetAsync(bar, 0, sizeof(unsigned) * (size_t)npan * nrt, st));
    launch_coop("k_f64_flow", k_f64_flow, (unsigned)G, NTH, 0, st, buf, ld, w.rows, npan, nid, dv, info,
                (const int2*)tl, (int)tiles.size(), bar, err);
    return;
  }
  if (variant >= 2) {
    int sms = 0, dev = 0;
    LMA_CK(cudaGetDevice(&dev));
    LMA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int m0 = npan - 1, work = std::max(m0 * (m0 + 1) / 2 + (nrt - npan) * m0, nrt);
    const int G = std::max(1, std::min({sms << (variant - 2), coop_capacity(), work}));
    LMA_CK(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    launch_coop("k_f64_coop", k_f64_coop, (unsigned)G, NTH, 0, st, buf, ld, w.rows, npan, nid, dv, info, bar, err);
    return;
  }
  launch_pdl("k_f64_potrf", k_f64_potrf, 1, NTH, 0, st, buf, ld, 0, dv, info);
  if (variant == 1) {
    for (int kp = 0; kp < npan; ++kp) {
      if (nrt - kp - 1 > 0)
        launch_pdl("k_f64_solve2", k_f64_solve2, (unsigned)(nrt - kp - 1), NTH, 0, st, buf, ld, w.rows, npan, kp,
                   nid, (const double*)dv);
      const int m = npan - kp - 1;
      if (m > 0)
        launch_pdl("k_f64_panel", k_f64_update2, (unsigned)(m * (m + 1) / 2 + (nrt - npan) * m), NTH, 0, st, buf,
                   ld, w.rows, npan, kp, nid, dv, info);
    }
    return;
  }
  for (int kp = 0; kp <= npan; ++kp) {
    const int m = npan - kp - 1;
    const int trail = m > 0 ? m * (m + 1) / 2 + (nrt - npan) * m : 0;
    const int solve = kp >= 1 ? nrt - kp : 0;
    if (trail + solve > 0)
      launch_pdl("k_f64_panel", k_f64_panel, (unsigned)(trail + solve), NTH, 0, st, buf, ld, w.rows, npan, kp, nid, dv,
             info);
  }
}

// Factorise one FP64 matrix already laid out in `buf` (order n, npad rows,
// `extra` extra rows); the first failing pivot (+1) goes to *info (device),
// which the caller checks after its next synchronisation; a grid-barrier
// timeout of the cooperative form sets *err.  The launch variant is a tuning
// site: all six are timed on a scratch copy of the matrix (the
// factorisation works in place), the model's default being the dataflow
// form.
static void factor_fp64_single(cudaStream_t st, Arena& tmp, double* buf, int n, int npad, int extra, int nid,
                               int* info, int* err) {
  Win w{};
  w.n = n;
  w.npad = npad;
  w.rows = npad + extra;
  double* dv = tmp.alloc<double>((size_t)npad * TB);
  const size_t nflag = (size_t)(npad / f64::TS) * ((w.rows + f64::TS - 1) / f64::TS);
  unsigned* bar = tmp.alloc<unsigned>(nflag);
  int2* tl = tmp.alloc<int2>(nflag);
  const size_t bytes = (size_t)w.rows * npad * sizeof(double);
  double* scratch = nullptr;
  int* sinfo = nullptr;
  auto run = [&](int v) {
    if (!scratch) {
      scratch = tmp.alloc<double>((size_t)w.rows * npad);
      sinfo = tmp.alloc<int>(1);
    }
    LMA_CK(cudaMemcpyAsync(scratch, buf, bytes, cudaMemcpyDeviceToDevice, st));
    LMA_CK(cudaMemsetAsync(sinfo, 0, sizeof(int), st));
    right_looking_fp64(st, w, nullptr, scratch, dv, sinfo, nid, v, bar, err, tl);
  };
  const std::string key = "fp64 factor n=" + std::to_string(n) + " rows=" + std::to_string(w.rows) +
                          " identity=" + std::to_string(nid);
  const int v = tune::pick(key, {0, 1, 2, 3, 4, 5}, 5, st, run);
  right_looking_fp64(st, w, nullptr, buf, dv, info, nid, v, bar, err, tl);
}

// ---------------------------------------------------------------------------
// One side stream and two events per host thread and device (created on
// first use): work that does not depend on the call stream's latest results
// runs there and is joined by an event.
struct Side {
  int dev = -1;
  cudaStream_t st = nullptr;
  cudaEvent_t local = nullptr, global = nullptr;
  void drop() {
    if (local) cudaEventDestroy(local);
    if (global) cudaEventDestroy(global);
    if (st) cudaStreamDestroy(st);
    st = nullptr;
    local = global = nullptr;
  }
  ~Side() { drop(); }
};

static Side& side_streams() {
  static thread_local Side side;
  int dev = 0;
  LMA_CK(cudaGetDevice(&dev));
  if (side.dev != dev) {
    side.drop();
    LMA_CK(cudaStreamCreateWithFlags(&side.st, cudaStreamNonBlocking));
    LMA_CK(cudaEventCreateWithFlags(&side.local, cudaEventDisableTiming));
    LMA_CK(cudaEventCreateWithFlags(&side.global, cudaEventDisableTiming));
    side.dev = dev;
  }
  return side;
}

template <typename T>
void Impl<T>::prepare(ModelCore& mc, const lma_problem* P, const lma_hyper* H, Arena& tmp, const double** X_d,
                      const double** y_d) {
  setup_attributes();
  cudaStream_t st = mc.st;
  const int64_t n = P->n, d = P->d, s = P->s;
  mc.n = n;
  mc.d = d;
  mc.M = P->m_blocks;
  mc.s = s;
  mc.B = P->markov_order;
  mc.mu = P->mean;
  mc.ss2 = exp(2.0 * H->log_sigma_s);
  mc.sn2 = exp(2.0 * H->log_sigma_n);
  mc.inv_ell.resize(d);
  for (int64_t q = 0; q < d; ++q) mc.inv_ell[q] = exp(-H->log_ell[q]);
  mc.bptr.assign(P->block_ptr, P->block_ptr + mc.M + 1);
  // inputs on the device
  const double *X = P->X, *y = P->y, *S = P->S;
  if (!P->inputs_on_device) {
    double* Xd = tmp.alloc<double>(n * d);
    double* yd = tmp.alloc<double>(n);
    double* Sd = tmp.alloc<double>(s * d);
    LMA_CK(cudaMemcpyAsync(Xd, X, sizeof(double) * n * d, cudaMemcpyHostToDevice, st));
    LMA_CK(cudaMemcpyAsync(yd, y, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    LMA_CK(cudaMemcpyAsync(Sd, S, sizeof(double) * s * d, cudaMemcpyHostToDevice, st));
    X = Xd;
    y = yd;
    S = Sd;
  }
  *X_d = X;
  *y_d = y;
  mc.inv_ell_d = mc.keep.alloc<double>(d);
  stage_copy(mc.inv_ell_d, mc.inv_ell.data(), sizeof(double) * d, st);
  T* xsT = mc.keep.alloc<T>(n * d);
  T* ssT = mc.keep.alloc<T>(s * d);
  double* ss64 = mc.keep.alloc<double>(s * d);
  mc.ss64 = ss64;
  launch("k_scale", k_scale<T>, nblk(n * d), NT, 0, st, X, n, (int)d, mc.inv_ell_d, nullptr, xsT);
  launch("k_scale", k_scale<T>, nblk(s * d), NT, 0, st, S, s, (int)d, mc.inv_ell_d, ss64, ssT);
  mc.xsT = xsT;
  mc.ssT = ssT;
  // Sigma_SS + jitter = L_SS L_SS^T, and L_SS^-T from the identity extra rows
  const int npS = (int)roundup(s, TB);
  double* kb = mc.keep.alloc<double>((size_t)(npS + s) * npS);
  mc.kss = kb;
  mc.npS = npS;
  launch("k_build_kss", k_build_kss, nblk((int64_t)(npS + s) * npS), NT, 0, st, ss64, (int)s, (int)d, mc.ss2, H->jitter, npS, kb);
  mc.flags = mc.keep.alloc<int>(4);
  LMA_CK(cudaMemsetAsync(mc.flags, 0, 4 * sizeof(int), st));
  T* ET = mc.keep.alloc<T>(s * s);
  T* Vt = mc.keep.alloc<T>(n * s);
  mc.ET = ET;
  mc.Vt = Vt;
  factor_fp64_single(st, tmp, kb, (int)s, npS, (int)s, (int)s, mc.flags + 0, mc.flags + 3);
  launch("k_copy_block", k_copy_block<T>, nblk(s * s), NT, 0, st, kb + (int64_t)npS * npS, npS, (int)s, ET);
  if (sizeof(T) == 4 && mc.prec == LMA_MIXED && use_tensor_cores()) {
    mc.ldk = (int)roundup(s, 64);
    mc.brows = (int)roundup(s, 128);
    mc.linv3 = mc.keep.alloc<uint16_t>((size_t)3 * mc.brows * mc.ldk);
    launch("k_linv_bf3", k_linv_bf3, nblk((int64_t)mc.brows * mc.ldk), NT, 0, st, (const double*)kb, (int64_t)npS,
           (int)s, mc.brows, mc.ldk, mc.linv3);
  }
  // V = L_SS^-1 Sigma_SD, point-major (the K_SD planes in the fit workspace)
  project<T>(mc, xsT, n, Vt, tmp, st, mc.flags + 2, true);
}

// Local part of a fit: windows of blocks [w_begin, own_end) are formed and
// factorised, and the Gram of the local summaries (Definition 1) of blocks
// [own_begin, own_end) goes to mc.G with their log-determinant sum in
// mc.logdetR.  A whole fit has w_begin = own_begin = 0, own_end = M.
template <typename T>
void Impl<T>::fit_local(ModelCore& mc, const lma_problem* P, const lma_hyper* H, int64_t w_begin,
                        int64_t own_begin, int64_t own_end, FusedTest* ft) {
  cudaStream_t st = mc.st;
  Arena tmp;
  tmp.st = st;
  try {
    const double *X_d, *y_d;
    prepare(mc, P, H, tmp, &X_d, &y_d);
    const bool batched = (mc.prec == LMA_MIXED);
    const int64_t n = mc.n, s = mc.s;
    const int d = (int)mc.d;
    T* rT = tmp.alloc<T>(n);
    launch("k_center", k_center<T>, nblk(n), NT, 0, st, y_d, n, mc.mu, rT);
    // windows
    int64_t bufe, dinve, ewe;
    std::vector<int> trows;
    if (ft) trows = fused_test_rows(mc.M, mc.B, ft->tptr);
    make_windows(mc.bptr, mc.B, s, sizeof(T), mc.wins, bufe, dinve, ewe, w_begin, own_end, ft ? &trows : nullptr);
    mc.w0 = w_begin;
    mc.own_b = own_begin;
    mc.own_e = own_end;
    const int64_t M = (int64_t)mc.wins.size();  // windows of this fit
    T* wbuf = mc.keep.alloc<T>(bufe);
    T* dinv = mc.keep.alloc<T>(dinve);
    T* ew = mc.keep.alloc<T>(ewe);
    Win* wd = mc.keep.alloc<Win>(M);
    int* info = mc.keep.alloc<int>(M);
    mc.winfo = info;
    mc.wbuf = wbuf;
    mc.dinv = dinv;
    mc.ew = ew;
    mc.wins_d = wd;
    stage_copy(wd, mc.wins.data(), sizeof(Win) * M, st);
    LMA_CK(cudaMemsetAsync(info, 0, sizeof(int) * M, st));
    int maxnt = 0;
    for (const Win& w : mc.wins) maxnt = std::max(maxnt, w.npad / TB);
    const T* Vt = (const T*)mc.Vt;
    const T* xsT = (const T*)mc.xsT;
    const unsigned et = nblk(s + 1, TB);
    if (batched && sizeof(T) == 4 && use_tensor_cores()) {
      // residual tiles on the tensor cores (bf16x6 products), fed by TMA from
      // the three bfloat16 planes of V (row length padded to 64) in reversed
      // point order
      const int sp = (int)roundup(s, 64);
      mc.ldvs = sp;
      mc.vb3 = split_rows_bf3(st, (const float*)Vt, n, s, sp, true, mc.keep.alloc<uint16_t>((size_t)3 * n * sp));
      const CUtensorMap vb = bf16_tensor_map(mc.vb3, 3 * n, sp);
      // tiles of window k inside its blanket's [0, L)^2 are copied from the
      // windows of the blanket's blocks afterwards (k_copy_shared_tiles)
      // instead of being recomputed; only where all those windows are in this fit
      std::vector<int> Ls((size_t)M, 0);
      int maxL = 0;
      for (int64_t k = 0; k < M; ++k) {
        const int64_t m = mc.wins[k].m, last = std::min<int64_t>(m + mc.B, mc.M - 1);
        if (last - w_begin >= M) continue;
        Ls[k] = (mc.wins[k].nB / 128) * 128;
        maxL = std::max(maxL, Ls[k]);
      }
      std::vector<int4> items;
      for (int64_t m = 0; m < M; ++m) {
        const int np = mc.wins[m].npad, Lt = Ls[m] / 128;
        for (int I = 0; I * 128 < np; ++I)
          for (int J = 0; J * RB < np && J * RB <= 128 * I + 127; ++J)
            if (!(I < Lt && J < Lt)) items.push_back(make_int4((int)m, I, J, 0));
      }
      int4* itd = tmp.alloc<int4>(items.size());
      int* rerr = mc.flags + 2;
      stage_copy(itd, items.data(), sizeof(int4) * items.size(), st);
      launch("k_resid_bf6", pad_dim(d) == 8 ? k_resid_bf6<8> : k_resid_bf6<MAXD>, persistent_grid(items.size()),
             bf6::NTHR, bf6::smem_bytes(), st, (const int4*)itd, (int)items.size(), (const Win*)wd, (const float*)xsT,
             d, vb, (int)n, sp / bf6::KC, (float)mc.ss2, (float)mc.sn2, (float*)wbuf, rerr);
      if (maxL > 0) {
        int* Lsd = tmp.alloc<int>((size_t)M);
        stage_copy(Lsd, Ls.data(), sizeof(int) * M, st);
        launch("k_copy_shared_tiles", k_copy_shared_tiles<float>, dim3((unsigned)maxL, (unsigned)M), NT, 0, st,
               (const Win*)wd, (int)M, (int)mc.B, (const int*)Lsd, (float*)wbuf);
      }
      launch("k_fill_ext", k_fill_ext4, dim3(maxnt, (unsigned)((s + 63) / 64 + 1), (unsigned)M), 256, 0, st,
             (const Win*)wd, (const float*)Vt, (const float*)rT, (int)s, (float*)wbuf);
    } else if (batched) {
      launch("k_resid", k_resid<T>, dim3(maxnt * (maxnt + 1) / 2, (unsigned)M), NT, 0, st, wd, xsT, d, Vt, (int)s, (T)mc.ss2,
                                                                          (T)mc.sn2, wbuf);
      launch("k_fill_ext", k_fill_ext<T>, dim3(maxnt, et, (unsigned)M), NT, 0, st, wd, Vt, rT, (int)s, wbuf);
    } else {
      for (int64_t m = 0; m < M; ++m) {
        const int nt = mc.wins[m].npad / TB;
        launch("k_resid", k_resid<T>, dim3(nt * (nt + 1) / 2, 1), NT, 0, st, wd + m, xsT, d, Vt, (int)s, (T)mc.ss2, (T)mc.sn2,
                                                               wbuf);
        launch("k_fill_ext", k_fill_ext<T>, dim3(nt, et, 1), NT, 0, st, wd + m, Vt, rT, (int)s, wbuf);
      }
    }
    int* tc_err = (batched && sizeof(T) == 4 && use_tensor_cores()) ? mc.flags + 2 : nullptr;
    if (ft) fused_rhs(mc, *ft, tmp);
    chol_sweep<T>(st, mc.wins, wd, wbuf, dinv, info, batched, tc_err);
    // Gram of the local summaries of the owned windows, reduced in a fixed order
    const int se = (int)s + 1;
    const int nte = (se + TB - 1) / TB;
    const int64_t nown = own_end - own_begin;
    const Win* wown = wd + (own_begin - w_begin);
    int nchunk = (int)std::min<int64_t>(nown, 32);
    int chunk = (int)((nown + nchunk - 1) / nchunk);
    std::vector<int2> tl;  // tensor cores: 128 x 128 tiles of the lower triangle
    double* partial = nullptr;
    int gtile = TB;
    if (tc_err) {
      gtile = 128;
      const int nt = (se + 127) / 128;
      for (int I = 0; I < nt; ++I)
        for (int J = 0; J <= I; ++J) tl.push_back(make_int2(I, J));
      int kmax = bf6::KC;
      for (int64_t m = own_begin; m < own_end; ++m) {
        const Win& w = mc.wins[m - w_begin];
        kmax = std::max(kmax, (int)roundup(w.n - w.nB, bf6::KC));
      }
      // the summary rows in three bfloat16 planes (bf16x6 products,
      // lma_bf6.cuh), in the fit workspace (the projection's planes in it
      // were consumed earlier on this stream)
      uint16_t* sb3 = (uint16_t*)fit_workspace(sizeof(uint16_t) * (size_t)3 * nown * se * kmax);
      launch("k_split_summary", k_split_summary_bf3, dim3((unsigned)((se + 7) / 8), (unsigned)nown), dim3(32, 8), 0,
             st, wown, (const float*)wbuf, se, (int)nown, kmax, sb3);
      const CUtensorMap sb = bf16_tensor_map(sb3, 3 * nown * se, kmax);
      int2* tld = tmp.alloc<int2>(tl.size());
      stage_copy(tld, tl.data(), sizeof(int2) * tl.size(), st);
      // Window groups: item (tile, group) sums the group's windows; the
      // groups' FP64 partials are added by k_gram_reduce.  Model: persistent
      // waves x windows per item (+ half a window of per-item overhead),
      // partials held to 1 GB; the tuner times the model's choice and its
      // neighbours.
      const int64_t nsm = persistent_grid(1u << 30);
      const int64_t gcap = std::max<int64_t>(1, std::min<int64_t>(nown, (int64_t)(1e9 / (8.0 * se * se))));
      auto groups_of = [&](int64_t g) { const int64_t c = (nown + g - 1) / g; return (nown + c - 1) / c; };
      auto cost = [&](int64_t g) {
        const int64_t c = (nown + g - 1) / g, G = (nown + c - 1) / c;
        return (double)((tl.size() * G + nsm - 1) / nsm) * ((double)c + 0.5);
      };
      int64_t gbest = 1;
      for (int64_t g = 1; g <= gcap; ++g)
        if (cost(g) < cost(gbest) - 1e-9) gbest = g;
      std::vector<int> cands;
      for (int64_t g : {gbest, gbest / 2, gbest * 2, gbest / 4, (int64_t)1})
        if (g >= 1 && g <= gcap && std::find(cands.begin(), cands.end(), (int)groups_of(g)) == cands.end())
          cands.push_back((int)groups_of(g));
      int64_t gmaxc = 1;
      for (int c : cands) gmaxc = std::max<int64_t>(gmaxc, c);
      partial = tmp.alloc<double>((size_t)gmaxc * se * se);
      auto run = [&](int g) {
        const int c = (int)((nown + g - 1) / g);
        launch("k_gram_bf6", k_gram_bf6, persistent_grid(tl.size() * g), bf6::NTHR, bf6::smem_bytes(), st,
               (const int2*)tld, (int)tl.size(), (int)nown, c, se, kmax, sb, (int)(nown * se), partial, tc_err);
      };
      const std::string key = "k_gram_bf6 se=" + std::to_string(se) + " windows=" + std::to_string(nown) +
                              " k=" + std::to_string(kmax) + " sm=" + std::to_string(nsm);
      const int g = tune::pick(key, cands, (int)groups_of(gbest), st, run);
      chunk = (int)((nown + g - 1) / g);
      nchunk = (int)((nown + chunk - 1) / chunk);
      run(g);
    } else {
      partial = tmp.alloc<double>((size_t)nchunk * se * se);
      launch("k_gram", k_gram<T>, dim3(nte * (nte + 1) / 2, nchunk), NT, 0, st, wown, (int)nown, chunk, (int)s, wbuf,
             partial);
    }
    mc.G = mc.keep.alloc<double>((size_t)se * se);
    launch("k_gram_reduce", k_gram_reduce, nblk((int64_t)se * se), NT, 0, st, partial, nchunk, se, mc.G, gtile);
    double* ldw = tmp.alloc<double>(nown);
    mc.ldR_d = mc.keep.alloc<double>(1);
    launch("k_logdet", k_logdet<T>, (unsigned)nown, NT, 0, st, wown, wbuf, ldw);
    launch("k_sum_ordered", k_sum_ordered, 1, 32, 0, st, ldw, (int)nown, mc.ldR_d);
    tmp.release();
  } catch (...) {
    tmp.release();
    throw;
  }
}

// Global part of a fit (Definition 2 and Eq. (pitck)) from the Gram in mc.G
// and mc.logdetR (local, or summed over the shards of a partitioned fit):
// C = I + A, L_C, beta = C^-1 y-ddot, L_C^-T, the per-window L^-1 e and the
// log-likelihood of n_total training points.
template <typename T>
void Impl<T>::fit_global(ModelCore& mc, int64_t n_total, cudaStream_t on) {
  cudaStream_t st = on ? on : mc.st;
  Arena tmp;
  tmp.st = st;
  const cudaStream_t keep_st = mc.keep.st;
  mc.keep.st = st;  // model buffers of the global step are ordered on its stream
  struct Restore {
    ModelCore& m;
    cudaStream_t s;
    ~Restore() { m.keep.st = s; }
  } restore{mc, keep_st};
  try {
    const int64_t s = mc.s, M = (int64_t)mc.wins.size();
    int maxnt = 0;
    for (const Win& w : mc.wins) maxnt = std::max(maxnt, w.npad / TB);
    // global step in FP64: C = I + A, L_C, w = L_C^-1 y, L_C^-T, beta = C^-1 y
    const int npC = (int)roundup(s, TB);
    double* cb = tmp.alloc<double>((size_t)(npC + 1 + s) * npC);
    launch("k_build_global", k_build_global, nblk((int64_t)(npC + 1 + s) * npC), NT, 0, st, mc.G, (int)s, npC, cb);
    factor_fp64_single(st, tmp, cb, (int)s, npC, (int)s + 1, (int)s, mc.flags + 1, mc.flags + 3);
    mc.beta = mc.keep.alloc<double>(s);
    mc.sc_d = mc.keep.alloc<double>(4);
    double* sc = mc.sc_d;
    launch("k_global_finish", k_global_finish, nblk(s, NT / 32), NT, 0, st, cb, mc.G, (int)s, npC, mc.beta, sc);
    T* LcT = mc.keep.alloc<T>(s * s);
    launch("k_copy_block", k_copy_block<T>, nblk(s * s), NT, 0, st, cb + (int64_t)npC * npC, npC, (int)s, LcT);
    mc.LcT = LcT;
    if (mc.linv3) {  // bfloat16 planes of L_C^-1 for the variance term on the tensor cores
      mc.lcinv3 = mc.keep.alloc<uint16_t>((size_t)3 * mc.brows * mc.ldk);
      launch("k_linv_bf3", k_linv_bf3, nblk((int64_t)mc.brows * mc.ldk), NT, 0, st, (const double*)cb, (int64_t)npC,
             (int)s, mc.brows, mc.ldk, mc.lcinv3);
    }
    if (sizeof(T) == 4) {
      float2* bs = tmp.alloc<float2>(s);
      launch("k_split_beta", k_split_beta, nblk(s), NT, 0, st, (const double*)mc.beta, (int)s, bs);
      launch("k_ew", k_ew_f32, dim3(nblk(maxnt * TB), (unsigned)M), NT, 0, st, mc.wins_d, (const float*)mc.wbuf,
             (const float2*)bs, (int)s, (float*)mc.ew);
    } else {
      launch("k_ew", k_ew<T>, dim3(nblk(maxnt * TB), (unsigned)M), NT, 0, st, mc.wins_d, (const T*)mc.wbuf, mc.beta,
             (int)s, (T*)mc.ew);
    }
    tmp.release();
  } catch (...) {
    tmp.release();
    throw;
  }
}

template <typename T>
void Impl<T>::check(ModelCore& mc, bool global, int64_t n_total, bool logdet_from_device) {
  cudaStream_t st = mc.st;
  int fl[4] = {0, 0, 0, 0};
  double hs[4] = {0, 0, 0, 0}, hr = 0;
  const int64_t nw = (int64_t)mc.wins.size();
  std::vector<int> wi((size_t)nw);
  LMA_CK(cudaMemcpyAsync(fl, mc.flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
  if (nw && mc.winfo) LMA_CK(cudaMemcpyAsync(wi.data(), mc.winfo, sizeof(int) * nw, cudaMemcpyDeviceToHost, st));
  if (logdet_from_device && mc.ldR_d) LMA_CK(cudaMemcpyAsync(&hr, mc.ldR_d, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (global) LMA_CK(cudaMemcpyAsync(hs, mc.sc_d, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
  LMA_CK(cudaStreamSynchronize(st));
  staging().reset();
  if (fl[0]) {
    fail(LMA_ERR_NOT_PD, "Sigma_SS + jitter is not positive definite", -1);
    throw Fail{};
  }
  if (fl[2]) {
    fail(LMA_ERR_TIMEOUT, "tensor-core pipeline wait timed out in the residual or window-sweep kernels");
    throw Fail{};
  }
  if (fl[3]) {
    fail(LMA_ERR_TIMEOUT, "grid barrier of the FP64 factorisation timed out");
    throw Fail{};
  }
  for (int64_t m = 0; m < nw; ++m)
    if (wi[m]) {
      fail(LMA_ERR_NOT_PD, "residual window of block " + std::to_string(mc.wins[m].m) +
                               " is not positive definite (pivot " + std::to_string(wi[m] - 1) + ")",
           mc.wins[m].m);
      throw Fail{};
    }
  if (logdet_from_device) mc.logdetR = hr;
  if (!global) return;
  if (fl[1]) {
    fail(LMA_ERR_NOT_PD, "global summary Sigma-ddot_SS is not positive definite", -2);
    throw Fail{};
  }
  mc.quad = hs[0];
  mc.wCw = hs[1];
  mc.logdetC = hs[2];
  mc.loglik = -0.5 * (mc.quad - mc.wCw) - 0.5 * (mc.logdetR + mc.logdetC) - 0.5 * (double)n_total * log(2.0 * M_PI);
  mc.have_global = true;
}

template <typename T>
void Impl<T>::fit(ModelCore& mc, const lma_problem* P, const lma_hyper* H) {
  fit_local(mc, P, H, 0, 0, P->m_blocks);
  fit_global(mc, mc.n);
  check(mc, true, mc.n, true);
}

// Fit and predict with the FP64 global step (Definition 2) on a second stream:
// the prediction's kernels that do not read its results (test-point support
// coordinates, right-hand sides, window sweeps, the h accumulation) overlap
// it, and the rest waits for its event.
template <typename T>
void Impl<T>::fit_predict(ModelCore& mc, const lma_problem* P, const lma_hyper* H, int64_t U, const double* XU,
                          const int64_t* tptr, int noisy, int on_device, double* mean, double* var) {
  Side& side = side_streams();
  // mixed form on the tensor cores: the test right-hand sides ride the fit's sweep
  FusedTest ft;
  FusedTest* ftp = nullptr;
  if (mc.prec == LMA_MIXED && sizeof(T) == 4 && use_tensor_cores() && U > 0) {
    ft.U = U;
    ft.XU = XU;
    ft.tptr = tptr;
    ft.on_device = on_device;
    ft.keep.st = mc.st;
    ftp = &ft;
  }
  try {
    fit_local(mc, P, H, 0, 0, P->m_blocks, ftp);
    LMA_CK(cudaEventRecord(side.local, mc.st));
    LMA_CK(cudaStreamWaitEvent(side.st, side.local, 0));
    try {
      fit_global(mc, mc.n, side.st);
      LMA_CK(cudaEventRecord(side.global, side.st));
      predict(mc, U, XU, tptr, noisy, on_device, mean, var, side.global, nullptr, ftp);
    } catch (...) {
      cudaStreamSynchronize(side.st);  // nothing of this call may still run on the side stream
      throw;
    }
  } catch (...) {
    ft.keep.release();
    throw;
  }
  ft.keep.release();
  LMA_CK(cudaStreamWaitEvent(mc.st, side.global, 0));
  check(mc, true, mc.n, true);
}

template <typename T>
void Impl<T>::fused_rhs(ModelCore& mc, FusedTest& ft, Arena& tmp) {
  if (sizeof(T) != 4 || !mc.vb3) {
    fail(LMA_ERR_INTERNAL, "appended test rows need the mixed form on the tensor cores");
    throw Fail{};
  }
  cudaStream_t st = mc.st;
  const int64_t s = mc.s, U = ft.U;
  const int d = (int)mc.d;
  ft.keep.st = st;
  const double* XUd = ft.XU;
  if (!ft.on_device) {
    double* t = tmp.alloc<double>(U * d);
    LMA_CK(cudaMemcpyAsync(t, ft.XU, sizeof(double) * U * d, cudaMemcpyHostToDevice, st));
    XUd = t;
  }
  float* xu = ft.keep.alloc<float>(U * d);
  launch("k_scale", k_scale<float>, nblk(U * d), NT, 0, st, XUd, U, d, mc.inv_ell_d, nullptr, xu);
  float* Vu = ft.keep.alloc<float>(U * s);
  project<float>(mc, (const float*)xu, U, Vu, tmp, st, mc.flags + 2);
  ft.xu = xu;
  ft.Vu = Vu;
  // One item row-range per window: its appended test rows are the test points
  // of blocks m .. m + B, consecutive both in the test order and in the
  // window buffer, so a 128-row tile covers the points of several blocks
  // (the right-hand sides R_{W_m u} of every pair (n, m) of the window).
  std::vector<Pair> pairs;
  const int64_t Mw = (int64_t)mc.wins.size();
  for (int64_t m = 0; m < Mw; ++m) {
    const Win& w = mc.wins[m];
    const int64_t last = std::min<int64_t>(m + mc.B, mc.M - 1);
    const int64_t u0 = ft.tptr[m], u1 = ft.tptr[last + 1];
    if (u1 <= u0) continue;
    Pair p{};
    p.pbase = w.base + (int64_t)(w.npad + s + 1) * w.npad;
    p.win = (int)m;
    p.u0 = (int)u0;
    p.nu = (int)(u1 - u0);
    p.c0 = 0;
    p.c1 = w.n;
    p.n = (int)m;
    pairs.push_back(p);
  }
  if (pairs.empty()) return;
  Pair* pd = tmp.alloc<Pair>(pairs.size());
  stage_copy(pd, pairs.data(), sizeof(Pair) * pairs.size(), st);
  const int sp = mc.ldvs;
  uint16_t* ub3 = split_rows_bf3(st, Vu, U, s, sp, false, tmp.alloc<uint16_t>((size_t)3 * U * sp));
  const CUtensorMap vb = bf16_tensor_map(mc.vb3, 3 * mc.n, sp), ub = bf16_tensor_map(ub3, 3 * U, sp);
  std::vector<int4> it_r;
  for (size_t pi = 0; pi < pairs.size(); ++pi) {
    const int nct = (mc.wins[pairs[pi].win].npad + 127) / 128;
    for (int ut = 0; ut < (pairs[pi].nu + 127) / 128; ++ut)
      for (int ct = 0; ct < nct; ++ct) it_r.push_back(make_int4((int)pi, ut, ct, 0));
  }
  int4* irr = tmp.alloc<int4>(it_r.size());
  stage_copy(irr, it_r.data(), sizeof(int4) * it_r.size(), st);
  launch("k_pred_rhs_bf6", pad_dim(d) == 8 ? k_pred_rhs_bf6<8> : k_pred_rhs_bf6<MAXD>, persistent_grid(it_r.size()),
         bf6::NTHR, bf6::smem_bytes(), st, (const Pair*)pd, (const int4*)irr, (int)it_r.size(),
         (const Win*)mc.wins_d, (const float*)mc.xsT, (const float*)xu, d, ub, (int)U, vb, (int)mc.n, sp / bf6::KC,
         (float)mc.ss2, (float*)mc.wbuf, mc.flags + 2);
}

template <typename T>
void Impl<T>::predict(const ModelCore& mc, int64_t U, const double* XU, const int64_t* tptr, int noisy, int on_device,
                      double* mean, double* var, cudaEvent_t global_done, double* cov, FusedTest* ft,
                      int* async_err, const int64_t* cov_pairs, int64_t n_cov_pairs) {
  cudaStream_t st = mc.st;
  Arena tmp;
  tmp.st = st;
  try {
    const int64_t s = mc.s, M = mc.M, B = mc.B;
    const int d = (int)mc.d;
    if (U == 0) {
      tmp.release();
      return;
    }
    int* perr = tmp.alloc<int>(1);  // tensor-core pipeline timeout, checked at the end
    LMA_CK(cudaMemsetAsync(perr, 0, sizeof(int), st));
    T* xu = nullptr;
    T* Vu = nullptr;
    if (ft) {  // test projections made before the fit's sweep
      xu = (T*)ft->xu;
      Vu = (T*)ft->Vu;
    } else {
      const double* XUd = XU;
      if (!on_device) {
        double* t = tmp.alloc<double>(U * d);
        LMA_CK(cudaMemcpyAsync(t, XU, sizeof(double) * U * d, cudaMemcpyHostToDevice, st));
        XUd = t;
      }
      xu = tmp.alloc<T>(U * d);
      launch("k_scale", k_scale<T>, nblk(U * d), NT, 0, st, XUd, U, d, mc.inv_ell_d, nullptr, xu);
      Vu = tmp.alloc<T>(U * s);
      project<T>(mc, (const T*)xu, U, Vu, tmp, st, perr);
    }
    // pairs (test block n, window m in [n-B, n])
    std::vector<Pair> pairs;
    std::vector<int4> tb;  // per test block: first pair, count, u0, nu
    int64_t pe = 0;
    make_pairs(mc.wins, mc.w0, M, B, s, tptr, ft != nullptr, pairs, tb, &pe);
    std::vector<int4> it_rhs, it_acc, it_t12;
    std::vector<int2> it_sw;
    for (size_t pi = 0; pi < pairs.size(); ++pi) {
      const Pair& p = pairs[pi];
      const int nut = (p.nu + TB - 1) / TB, nct = mc.wins[p.win].npad / TB;
      for (int ut = 0; ut < nut; ++ut) {
        it_sw.push_back(make_int2((int)pi, ut));
        for (int ct = 0; ct < nct; ++ct) it_rhs.push_back(make_int4((int)pi, ut, ct, 0));
      }
    }
    const int nst = (int)((s + TB - 1) / TB);
    for (const int4& t : tb) {
      const int nut = (t.w + TB - 1) / TB;
      for (int ut = 0; ut < nut; ++ut)
        for (int kt = 0; kt < nst; ++kt) it_acc.push_back(make_int4(t.x, t.y, ut, kt));
      for (int u = 0; u < t.w; ++u) it_t12.push_back(make_int4(t.x, t.y, u, 0));
    }
    Pair* pd = tmp.alloc<Pair>(pairs.size());
    int4* ird = tmp.alloc<int4>(it_rhs.size());
    int2* isd = tmp.alloc<int2>(it_sw.size());
    int4* iad = tmp.alloc<int4>(it_acc.size());
    int4* itd = tmp.alloc<int4>(it_t12.size());
    stage_copy(pd, pairs.data(), sizeof(Pair) * pairs.size(), st);
    stage_copy(ird, it_rhs.data(), sizeof(int4) * it_rhs.size(), st);
    stage_copy(isd, it_sw.data(), sizeof(int2) * it_sw.size(), st);
    stage_copy(iad, it_acc.data(), sizeof(int4) * it_acc.size(), st);
    stage_copy(itd, it_t12.data(), sizeof(int4) * it_t12.size(), st);
    T* Pbuf = ft ? (T*)mc.wbuf : tmp.alloc<T>(pe);
    const T* xs = (const T*)mc.xsT;
    const T* Vt = (const T*)mc.Vt;
    const T* wbuf = (const T*)mc.wbuf;
    if (ft) {
      // the right-hand sides were appended to the windows and solved by the fit's sweep
    } else if (mc.prec == LMA_MIXED) {
      const bool tc = (sizeof(T) == 4 && use_tensor_cores());
      if (tc) {
        // right-hand sides on the tensor cores (bf16x6 products), fed by TMA
        // from the bfloat16 planes of Vu (test order) and of Vt (reversed
        // point order)
        const int sp = (int)roundup(s, 64);
        const uint16_t* vb3 = mc.vb3;
        if (!vb3 || mc.ldvs != sp)
          vb3 = split_rows_bf3(st, (const float*)Vt, mc.n, s, sp, true, tmp.alloc<uint16_t>((size_t)3 * mc.n * sp));
        uint16_t* ub3 = split_rows_bf3(st, (const float*)Vu, U, s, sp, false, tmp.alloc<uint16_t>((size_t)3 * U * sp));
        const CUtensorMap vb = bf16_tensor_map(vb3, 3 * mc.n, sp), ub = bf16_tensor_map(ub3, 3 * U, sp);
        std::vector<int4> it_r;
        for (size_t pi = 0; pi < pairs.size(); ++pi) {
          const int nct = (mc.wins[pairs[pi].win].npad + 127) / 128;
          for (int ut = 0; ut < (pairs[pi].nu + 127) / 128; ++ut)
            for (int ct = 0; ct < nct; ++ct) it_r.push_back(make_int4((int)pi, ut, ct, 0));
        }
        int4* irr = tmp.alloc<int4>(it_r.size());
        stage_copy(irr, it_r.data(), sizeof(int4) * it_r.size(), st);
        launch("k_pred_rhs_bf6", pad_dim(d) == 8 ? k_pred_rhs_bf6<8> : k_pred_rhs_bf6<MAXD>,
               persistent_grid(it_r.size()), bf6::NTHR, bf6::smem_bytes(), st, (const Pair*)pd, (const int4*)irr,
               (int)it_r.size(), (const Win*)mc.wins_d, (const float*)xs, (const float*)xu, d, ub, (int)U, vb,
               (int)mc.n, sp / bf6::KC, (float)mc.ss2, (float*)Pbuf, perr);
      } else {
        launch("k_pred_rhs", k_pred_rhs<T>, (unsigned)it_rhs.size(), NT, 0, st, pd, ird, mc.wins_d, xs, xu, d, Vt, Vu,
               (int)s, (T)mc.ss2, Pbuf);
      }
      if (tc) {
        std::vector<int2> it_tc;
        for (size_t pi = 0; pi < pairs.size(); ++pi)
          for (int ut = 0; ut < (pairs[pi].nu + 127) / 128; ++ut) it_tc.push_back(make_int2((int)pi, ut));
        int2* itc = tmp.alloc<int2>(it_tc.size());
        stage_copy(itc, it_tc.data(), sizeof(int2) * it_tc.size(), st);
        launch("k_pred_sweep_tc", k_pred_sweep_tc, (unsigned)it_tc.size(), 256, tc_chol_smem(), st, pd,
               (const int2*)itc, mc.wins_d, (const float*)wbuf, (const float*)mc.dinv, (float*)Pbuf, perr);
      } else {
        launch("k_pred_sweep", k_pred_sweep<T>, (unsigned)it_sw.size(), NT, sizeof(CholSmem<T>), st, pd, isd,
               mc.wins_d, wbuf, (const T*)mc.dinv, Pbuf);
      }
    } else {
      // plain form: one pair per launch
      size_t a = 0, b = 0;
      for (size_t pi = 0; pi < pairs.size(); ++pi) {
        size_t a1 = a, b1 = b;
        while (a1 < it_rhs.size() && it_rhs[a1].x == (int)pi) ++a1;
        while (b1 < it_sw.size() && it_sw[b1].x == (int)pi) ++b1;
        launch("k_pred_rhs", k_pred_rhs<T>, (unsigned)(a1 - a), NT, 0, st, pd, ird + a, mc.wins_d, xs, xu, d, Vt, Vu, (int)s,
                                                         (T)mc.ss2, Pbuf);
        launch("k_pred_sweep", k_pred_sweep<T>, (unsigned)(b1 - b), NT, sizeof(CholSmem<T>), st, pd, isd + b, mc.wins_d, wbuf,
                                                                            (const T*)mc.dinv, Pbuf);
        a = a1;
        b = b1;
      }
    }
    T* h = tmp.alloc<T>(U * s);
    if (mc.prec == LMA_MIXED && sizeof(T) == 4 && use_tensor_cores()) {
      // per window: its pairs (n, m) in increasing n, their partial rows, items
      const int64_t nwin = (int64_t)mc.wins.size();
      std::vector<std::vector<int>> byw((size_t)nwin);
      for (size_t pi = 0; pi < pairs.size(); ++pi) byw[pairs[pi].win].push_back((int)pi);
      std::vector<int> wp;
      std::vector<int4> it_w;
      std::vector<int64_t> wrow, prow(pairs.size(), 0);
      int64_t hrows = 0;
      for (int64_t m = 0; m < nwin; ++m) {
        if (byw[m].empty()) continue;
        const int off = (int)wp.size();
        int rows = 0;
        for (int pi : byw[m]) {
          wp.push_back(pi);
          prow[pi] = hrows + rows;
          rows += pairs[pi].nu;
        }
        for (int ut = 0; ut < (rows + 127) / 128; ++ut)
          for (int kt = 0; kt < (s + RB - 1) / RB; ++kt) {
            it_w.push_back(make_int4(off, (int)byw[m].size(), ut, kt));
            wrow.push_back(hrows);
          }
        hrows += rows;
      }
      int* wpd = tmp.alloc<int>(wp.size());
      int4* iwd = tmp.alloc<int4>(it_w.size());
      int64_t* wrd = tmp.alloc<int64_t>(wrow.size());
      int64_t* prd = tmp.alloc<int64_t>(prow.size());
      int4* tbd = tmp.alloc<int4>(tb.size());
      stage_copy(wpd, wp.data(), sizeof(int) * wp.size(), st);
      stage_copy(iwd, it_w.data(), sizeof(int4) * it_w.size(), st);
      stage_copy(wrd, wrow.data(), sizeof(int64_t) * wrow.size(), st);
      stage_copy(prd, prow.data(), sizeof(int64_t) * prow.size(), st);
      stage_copy(tbd, tb.data(), sizeof(int4) * tb.size(), st);
      float* hw = tmp.alloc<float>((size_t)hrows * s);
      if (!it_w.empty())
        launch("k_pred_accum_tc", k_pred_accum_win, (unsigned)it_w.size(), comp_threads<RB>(), tc_resid_smem(), st, pd,
               (const int*)wpd, (const int4*)iwd, (const int64_t*)wrd, mc.wins_d, (const float*)wbuf,
               (const float*)Pbuf, (int)s, hw, perr);
      int maxnu = 1;
      for (const int4& t : tb) maxnu = std::max(maxnu, t.w);
      if (!tb.empty())
        launch("k_pred_hsum", k_pred_hsum, dim3(nblk((int64_t)maxnu * s), (unsigned)tb.size()), NT, 0, st,
               (const int4*)tbd, (const int64_t*)prd, (const float*)hw, (const float*)Vu, (int)s, (float*)h);
    } else {
      launch("k_pred_accum", k_pred_accum<T>, (unsigned)it_acc.size(), NT, 0, st, pd, iad, mc.wins_d, wbuf, Pbuf, Vu,
             (int)s, h);
    }
    double* t1 = tmp.alloc<double>(U);
    double* t2 = tmp.alloc<double>(U);
    // from here on the global step's results (beta, L^-1 e, L_C^-1) are read
    if (global_done) LMA_CK(cudaStreamWaitEvent(st, global_done, 0));
    launch("k_pred_t12", k_pred_t12<T>, nblk((int64_t)it_t12.size() * 32), NT, 0, st, pd, itd, (int)it_t12.size(), mc.wins_d, Pbuf,
                                                                    (const T*)mc.ew, t1, t2);
    double* part = tmp.alloc<double>((size_t)nst * U);
    int ntile_var = nst;
    if (sizeof(T) == 4 && mc.lcinv3) {  // L_C^-1 h on the tensor cores (bf16x6), then row norms
      uint16_t* hp = tmp.alloc<uint16_t>((size_t)3 * U * mc.ldk);
      launch("k_split_bf3", k_split_bf3, nblk(U * (mc.ldk / 8)), NT, 0, st, (const float*)h, U, (int)s, (int64_t)s,
             mc.ldk, hp, 0);
      float* g = tmp.alloc<float>((size_t)U * s);
      proj_tc(st, "k_var_gemm", hp, U, mc.lcinv3, mc.brows, (int)s, mc.ldk, g, s, perr);
      launch("k_row_sqnorm", k_row_sqnorm, nblk(U * 32), NT, 0, st, (const float*)g, U, (int)s, part);
      ntile_var = 1;
    } else if (sizeof(T) == 4 && s % 4 == 0) {  // L_C^-1 h with the 128 x 128 FP32 product, then row norms
      float* g = tmp.alloc<float>((size_t)U * s);
      launch("k_var_gemm", k_proj128, dim3(nblk(s, 128), nblk(U, 128)), NT, 0, st, (const float*)h, U, (int)s,
             (const float*)mc.LcT, g, (int)s);
      launch("k_row_sqnorm", k_row_sqnorm, nblk(U * 32), NT, 0, st, (const float*)g, U, (int)s, part);
      ntile_var = 1;
    } else {
      launch("k_var_gemm", k_var_gemm<T>, dim3(nst, nblk(U, TB)), NT, 0, st, h, U, (int)s, (const T*)mc.LcT, part);
    }
    double* md = mean;
    double* vd = var;
    if (!on_device) {
      md = tmp.alloc<double>(U);
      vd = tmp.alloc<double>(U);
    }
    const double prior = mc.ss2 + (noisy ? mc.sn2 : 0.0);
    launch("k_pred_final", k_pred_final<T>, nblk(U * 32), NT, 0, st, Vu, U, (int)s, mc.beta, t1, t2, part, ntile_var,
           mc.mu, prior, md, vd);
    if (cov) {
      // requested blocks of the covariance between test blocks (Eq. vapvar on
      // U_n x U_n2), packed row-major in request order; without a request
      // list, the block of every test block with itself, block after block
      std::vector<int> first(M, -1);  // first pair of each test block
      for (const int4& t : tb) first[pairs[t.x].n] = t.x;
      std::vector<int64_t> req;
      if (n_cov_pairs < 0) {
        for (int64_t nb = 0; nb < M; ++nb) {
          req.push_back(nb);
          req.push_back(nb);
        }
      } else {
        req.assign(cov_pairs, cov_pairs + 2 * n_cov_pairs);
      }
      std::vector<CovReq> rq;
      std::vector<int4> it_c;
      int64_t total = 0;
      for (size_t i = 0; i + 1 < req.size(); i += 2) {
        const int64_t n1 = req[i], n2 = req[i + 1];
        CovReq c{};
        c.off = total;
        c.u0a = (int)tptr[n1];
        c.nua = (int)(tptr[n1 + 1] - tptr[n1]);
        c.u0b = (int)tptr[n2];
        c.nub = (int)(tptr[n2 + 1] - tptr[n2]);
        total += (int64_t)c.nua * c.nub;
        if (c.nua == 0 || c.nub == 0) continue;
        c.lo = (int)std::min(n1, n2);
        const int64_t hi = std::max(n1, n2);
        c.same = n1 == n2;
        if (hi - c.lo <= B) {
          c.m_lo = (int)std::max<int64_t>(0, hi - B);
          c.nm = c.lo - c.m_lo + 1;
          c.pa = first[n1] + (int)(c.m_lo - std::max<int64_t>(0, n1 - B));
          c.pb = first[n2] + (int)(c.m_lo - std::max<int64_t>(0, n2 - B));
        }
        const int ri = (int)rq.size();
        rq.push_back(c);
        for (int a = 0; a < (c.nua + TB - 1) / TB; ++a)
          for (int b = 0; b < (c.nub + TB - 1) / TB; ++b) it_c.push_back(make_int4(ri, a, b, 0));
      }
      T* g = tmp.alloc<T>(U * s);
      launch("k_lc_apply", k_lc_apply<T>, dim3(nblk(s, TB), nblk(U, TB)), NT, 0, st, (const T*)h, U, (int)s,
             (const T*)mc.LcT, g);
      CovReq* rqd = tmp.alloc<CovReq>(rq.size());
      int4* icd = tmp.alloc<int4>(it_c.size());
      stage_copy(rqd, rq.data(), sizeof(CovReq) * rq.size(), st);
      stage_copy(icd, it_c.data(), sizeof(int4) * it_c.size(), st);
      double* cd = on_device ? cov : tmp.alloc<double>(total);
      if (!it_c.empty())
        launch("k_pred_xcov", k_pred_xcov<T>, (unsigned)it_c.size(), NT, 0, st, pd, (const CovReq*)rqd,
               (const int4*)icd, mc.wins_d, (const T*)xu, d, (const T*)Vu, (const T*)Pbuf, (const T*)g, (int)s,
               mc.ss2, noisy ? mc.sn2 : 0.0, cd);
      if (!on_device && total) LMA_CK(cudaMemcpyAsync(cov, cd, sizeof(double) * total, cudaMemcpyDeviceToHost, st));
    }
    if (!on_device) {
      LMA_CK(cudaMemcpyAsync(mean, md, sizeof(double) * U, cudaMemcpyDeviceToHost, st));
      LMA_CK(cudaMemcpyAsync(var, vd, sizeof(double) * U, cudaMemcpyDeviceToHost, st));
    }
    if (async_err) {  // enqueued: the status word is read by lma_model_wait, the staging kept
      launch("k_or_flag", k_or_flag, 1, 32, 0, st, (const int*)perr, async_err);
      tmp.release();
      staging().hold = true;
      return;
    }
    int herr = 0;
    LMA_CK(cudaMemcpyAsync(&herr, perr, sizeof(int), cudaMemcpyDeviceToHost, st));
    tmp.release();
    LMA_CK(cudaStreamSynchronize(st));
    staging().reset();
    if (herr) {
      fail(LMA_ERR_TIMEOUT, "tensor-core pipeline wait timed out in the prediction kernels");
      throw Fail{};
    }
  } catch (...) {
    tmp.release();
    throw;
  }
}

// residual window of block m in natural row order (host, n_w x n_w)
template <typename T>
void Impl<T>::window_residual(ModelCore& mc, const lma_problem* P, const lma_hyper* H, int64_t m, double* out) {
  cudaStream_t st = mc.st;
  Arena tmp;
  tmp.st = st;
  try {
    const double *X_d, *y_d;
    prepare(mc, P, H, tmp, &X_d, &y_d);
    int64_t bufe, dinve, ewe;
    std::vector<Win> all;
    make_windows(mc.bptr, mc.B, mc.s, sizeof(T), all, bufe, dinve, ewe);
    Win w = all[m];
    w.base = 0;
    Win* wd = tmp.alloc<Win>(1);
    stage_copy(wd, &w, sizeof(Win), st);
    T* buf = tmp.alloc<T>((size_t)w.npad * w.npad);
    const int nt = w.npad / TB;
    if (sizeof(T) == 4 && mc.prec == LMA_MIXED && use_tensor_cores()) {
      const int64_t s = mc.s, n = mc.n;
      const int sp = (int)roundup(s, 64);
      const uint16_t* vb3 = mc.vb3;
      if (!vb3 || mc.ldvs != sp)
        vb3 = split_rows_bf3(st, (const float*)mc.Vt, n, s, sp, true, tmp.alloc<uint16_t>((size_t)3 * n * sp));
      const CUtensorMap vb = bf16_tensor_map(vb3, 3 * n, sp);
      std::vector<int4> items;
      for (int I = 0; I * 128 < w.npad; ++I)
        for (int J = 0; J * RB < w.npad && J * RB <= 128 * I + 127; ++J) items.push_back(make_int4(0, I, J, 0));
      int4* itd = tmp.alloc<int4>(items.size());
      int* rerr = mc.flags + 2;
      stage_copy(itd, items.data(), sizeof(int4) * items.size(), st);
      launch("k_resid_bf6", pad_dim((int)mc.d) == 8 ? k_resid_bf6<8> : k_resid_bf6<MAXD>,
             persistent_grid(items.size()), bf6::NTHR, bf6::smem_bytes(), st, (const int4*)itd, (int)items.size(),
             (const Win*)wd, (const float*)mc.xsT, (int)mc.d, vb, (int)n, sp / bf6::KC, (float)mc.ss2, (float)mc.sn2,
             (float*)buf, rerr);
    } else {
      launch("k_resid", k_resid<T>, dim3(nt * (nt + 1) / 2, 1), NT, 0, st, wd, (const T*)mc.xsT, (int)mc.d,
             (const T*)mc.Vt, (int)mc.s, (T)mc.ss2, (T)mc.sn2, buf);
    }
    std::vector<T> h((size_t)w.npad * w.npad);
    LMA_CK(cudaMemcpyAsync(h.data(), buf, sizeof(T) * h.size(), cudaMemcpyDeviceToHost, st));
    check(mc, false, 0, false);
    const int n = w.n;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        int a = n - 1 - i, b = n - 1 - j;  // reversed storage, lower triangle valid
        if (b > a) std::swap(a, b);
        out[(int64_t)i * n + j] = (double)h[(size_t)a * w.npad + b];
      }
    tmp.release();
  } catch (...) {
    tmp.release();
    throw;
  }
}

template <typename T>
void Impl<T>::loglik_grad(ModelCore& mc, const lma_problem* P, const lma_hyper* H, double* ll, double* grad) {
  fit(mc, P, H);
  grad_windows(mc, 0, (int64_t)mc.wins.size(), grad);
  *ll = mc.loglik;
}

// The adjoint restricted to windows [k_lo, k_hi) of the model: their
// G_m terms and the chain of their Vt-bar contributions through K_DS and
// L_SS.  Every step after the window terms is linear in them, so the parts
// of a partition of the windows add up to the whole gradient.
template <typename T>
void Impl<T>::grad_windows(ModelCore& mc, int64_t k_lo, int64_t k_hi, double* grad) {
  cudaStream_t st = mc.st;
  Arena tmp;
  tmp.st = st;
  try {
    const int64_t n = mc.n, s = mc.s, M = k_hi - k_lo;
    const int d = (int)mc.d;
    const int si = (int)s;
    const Win* wk = mc.wins_d + k_lo;  // the windows of this gradient, indexed from 0
    // per-window backward layout
    std::vector<GWin> gw(M);
    int64_t qe = 0, ge = 0, gve = 0;
    int maxnt = 0, maxrows = 0;
    for (int64_t m = 0; m < M; ++m) {
      const Win& w = mc.wins[k_lo + m];
      GWin g{};
      g.nrows = 2 * (si + 1) + (w.n - w.nB);
      g.q = qe;
      g.g = ge;
      g.gv = gve;
      qe += (int64_t)g.nrows * w.npad;
      ge += (int64_t)w.npad * w.npad;
      gve += s * w.npad;
      gw[m] = g;
      maxnt = std::max(maxnt, w.npad / TB);
      maxrows = std::max(maxrows, g.nrows);
    }
    GWin* gwd = tmp.alloc<GWin>(M);
    stage_copy(gwd, gw.data(), sizeof(GWin) * M, st);
    T* Q = tmp.alloc<T>(qe);
    T* Gb = tmp.alloc<T>(ge);
    T* GV = tmp.alloc<T>(gve);
    const T* wbuf = (const T*)mc.wbuf;
    const int np2 = d + 2;
    // the window products on the tensor cores in the mixed form (3xTF32,
    // lma_grad_tc.cuh), on the SIMT kernels of lma_grad.cuh otherwise
    const bool tc = sizeof(T) == 4 && use_tensor_cores();
    int* tc_err = mc.flags + 2;
    LMA_CK(cudaMemsetAsync(tc_err, 0, sizeof(int), st));
    size_t n_g = 0;
    double* pG = nullptr;
    if (tc) {
      const unsigned st128 = nblk(s, 128);
      launch("k_grad_rhs_tc", k_grad_rhs_tc, dim3(maxnt, st128, (unsigned)M), 256, tc_chol_smem(), st, wk,
             gwd, (const float*)wbuf, (const float*)mc.LcT, si, (float*)Q, tc_err);
      launch("k_grad_rhs_fill", k_grad_rhs_fill<T>, dim3(64, (unsigned)M), NT, 0, st, wk, gwd,
             (const T*)mc.ew, si, Q);
      std::vector<int2> it_sw;
      std::vector<int4> it_g;
      for (int64_t m = 0; m < M; ++m) {
        const int nrt = (gw[m].nrows + 127) / 128;
        for (int ut = 0; ut < nrt; ++ut) it_sw.push_back(make_int2((int)m, ut));
        const int np = mc.wins[k_lo + m].npad;
        for (int I = 0; I * 128 < np; ++I)
          for (int J = 0; J * 64 < np && J * 64 <= 128 * I + 127; ++J) it_g.push_back(make_int4((int)m, I, J, 0));
      }
      int2* isw = tmp.alloc<int2>(it_sw.size());
      int4* ig = tmp.alloc<int4>(it_g.size());
      stage_copy(isw, it_sw.data(), sizeof(int2) * it_sw.size(), st);
      stage_copy(ig, it_g.data(), sizeof(int4) * it_g.size(), st);
      launch("k_bwd_sweep_tc", k_bwd_sweep_tc, dim3((unsigned)it_sw.size()), 256, tc_chol_smem(), st,
             (const int2*)isw, wk, gwd, (const float*)wbuf, (const float*)mc.dinv, (float*)Q, tc_err);
      n_g = it_g.size();
      pG = tmp.alloc<double>(n_g * np2);
      launch("k_grad_G_tc", k_grad_G_tc, dim3((unsigned)n_g), 256, tc_chol_smem(), st, (const int4*)ig, wk,
             gwd, (const float*)Q, (const float*)mc.xsT, d, si, (float)mc.ss2, mc.sn2, (float*)Gb, pG, tc_err);
      launch("k_grad_gv_tc", k_grad_gv_tc, dim3(maxnt, st128, (unsigned)M), 256, tc_chol_smem(), st, wk,
             gwd, (const float*)Gb, (const float*)mc.Vt, si, (float*)GV, tc_err);
    } else {
      launch("k_grad_rhs", k_grad_rhs<T>, dim3(maxnt, nblk(s, TB), (unsigned)M), NT, 0, st, wk, gwd, wbuf,
             (const T*)mc.LcT, si, Q);
      launch("k_grad_rhs_fill", k_grad_rhs_fill<T>, dim3(64, (unsigned)M), NT, 0, st, wk, gwd,
             (const T*)mc.ew, si, Q);
      std::vector<int2> it_sw, it_g;
      for (int64_t m = 0; m < M; ++m) {
        const int nrt = (gw[m].nrows + TB - 1) / TB;
        for (int ut = 0; ut < nrt; ++ut) it_sw.push_back(make_int2((int)m, ut));
        const int nt = mc.wins[k_lo + m].npad / TB;
        for (int t = 0; t < nt * (nt + 1) / 2; ++t) it_g.push_back(make_int2((int)m, t));
      }
      int2* isw = tmp.alloc<int2>(it_sw.size());
      int2* ig = tmp.alloc<int2>(it_g.size());
      stage_copy(isw, it_sw.data(), sizeof(int2) * it_sw.size(), st);
      stage_copy(ig, it_g.data(), sizeof(int2) * it_g.size(), st);
      launch("k_bwd_sweep", k_bwd_sweep<T>, dim3((unsigned)it_sw.size()), NT, sizeof(CholSmem<T>), st, isw,
             wk, gwd, wbuf, (const T*)mc.dinv, Q);
      n_g = it_g.size();
      pG = tmp.alloc<double>(n_g * np2);
      launch("k_grad_G", k_grad_G<T>, dim3((unsigned)n_g), NT, 0, st, ig, wk, gwd, (const T*)Q,
             (const T*)mc.xsT, d, si, mc.ss2, mc.sn2, Gb, pG);
      launch("k_grad_gv", k_grad_gv<T>, dim3(maxnt, nblk(s, TB), (unsigned)M), NT, 0, st, wk, gwd,
             (const T*)Gb, (const T*)mc.Vt, si, GV);
    }
    int64_t* bptr_d = tmp.alloc<int64_t>(mc.M + 1);
    stage_copy(bptr_d, mc.bptr.data(), sizeof(int64_t) * (mc.M + 1), st);
    T* PsiT = tmp.alloc<T>((s + 1) * n);
    T* GVT = tmp.alloc<T>(s * n);
    launch("k_grad_gather", k_grad_gather<T>, dim3(nblk(n), (unsigned)(2 * s + 1)), NT, 0, st, mc.wins_d, gwd,
           bptr_d, (int)mc.M, (int)mc.B, n, si, (const T*)Q, (const T*)GV, PsiT, GVT, (int)mc.w0, (int)k_lo,
           (int)k_hi);
    T* VbT = tmp.alloc<T>(s * n);
    launch("k_grad_vbar", k_grad_vbar<T>, dim3(nblk(n, TB), nblk(s, TB)), NT, 0, st, (const T*)PsiT,
           (const T*)GVT, (const T*)mc.LcT, mc.beta, n, si, VbT);
    const unsigned gx = nblk(n, TB), gy = nblk(s, TB);
    double* pK = tmp.alloc<double>((size_t)gx * gy * np2);
    launch("k_grad_kds", k_grad_kds<T>, dim3(gx, gy), NT, 0, st, (const T*)VbT, (const T*)mc.ET,
           (const T*)mc.xsT, (const T*)mc.ssT, d, n, si, mc.ss2, pK);
    // L_SS-bar = -L_SS^-T (Vt-bar^T Vt) and the Cholesky adjoint, in FP64
    const int nch = (int)std::min<int64_t>(64, (n + 8191) / 8192);
    const int64_t chunk = (n + nch - 1) / nch;
    double* pM = tmp.alloc<double>((size_t)nch * s * s);
    launch("k_grad_m1", k_grad_m1<T>, dim3(gy, gy, nch), NT, 0, st, (const T*)VbT, (const T*)mc.Vt, n, si, chunk,
           pM);
    double* M1 = tmp.alloc<double>(s * s);
    launch("k_sum_chunks", k_sum_chunks, nblk(s * s), NT, 0, st, (const double*)pM, nch, (int64_t)(s * s), M1);
    const double* ET64 = mc.kss + (int64_t)mc.npS * mc.npS;
    double* Lm = tmp.alloc<double>(s * s);   // L_SS with its upper triangle zeroed
    launch("k_copy_block", k_copy_block<double>, nblk(s * s), NT, 0, st, (const double*)mc.kss, (int64_t)mc.npS,
           si, Lm);
    launch("k_phi", k_phi, nblk(s * s), NT, 0, st, Lm, si);   // tril with halved diagonal ...
    launch("k_tril_fix", k_tril_fix, nblk(s * s), NT, 0, st, Lm, si);  // ... restore the diagonal
    double* Lbar = tmp.alloc<double>(s * s);
    double* X = tmp.alloc<double>(s * s);
    double* Y = tmp.alloc<double>(s * s);
    double* Sb = tmp.alloc<double>(s * s);
    const dim3 gg(gy, gy);
    launch("k_dgemm", k_dgemm<false, false>, gg, NT, 0, st, ET64, (int64_t)mc.npS, (const double*)M1, s, Lbar, s,
           si, -1.0);
    launch("k_dgemm", k_dgemm<true, false>, gg, NT, 0, st, (const double*)Lm, s, (const double*)Lbar, s, X, s, si,
           1.0);
    launch("k_phi", k_phi, nblk(s * s), NT, 0, st, X, si);
    launch("k_dgemm", k_dgemm<false, true>, gg, NT, 0, st, (const double*)X, s, ET64, (int64_t)mc.npS, Y, s, si,
           1.0);
    launch("k_dgemm", k_dgemm<false, false>, gg, NT, 0, st, ET64, (int64_t)mc.npS, (const double*)Y, s, Sb, s, si,
           1.0);
    double* pS = tmp.alloc<double>(s * np2);
    launch("k_grad_kss", k_grad_kss, (unsigned)s, NT, 0, st, (const double*)Sb, (const double*)mc.ss64, si, d,
           mc.ss2, pS);
    // ordered reduction of the partial sums on the host
    std::vector<double> h1(n_g * np2), h2((size_t)gx * gy * np2), h3(s * np2);
    int terr = 0;
    LMA_CK(cudaMemcpyAsync(h1.data(), pG, sizeof(double) * h1.size(), cudaMemcpyDeviceToHost, st));
    LMA_CK(cudaMemcpyAsync(h2.data(), pK, sizeof(double) * h2.size(), cudaMemcpyDeviceToHost, st));
    LMA_CK(cudaMemcpyAsync(h3.data(), pS, sizeof(double) * h3.size(), cudaMemcpyDeviceToHost, st));
    LMA_CK(cudaMemcpyAsync(&terr, tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMA_CK(cudaStreamSynchronize(st));
    if (terr) {
      fail(LMA_ERR_TIMEOUT, "tensor-core pipeline wait timed out in the gradient kernels");
      throw Fail{};
    }
    for (int q = 0; q < np2; ++q) grad[q] = 0.0;
    for (const auto* v : {&h1, &h2, &h3})
      for (size_t i = 0; i < v->size(); i += np2)
        for (int q = 0; q < np2; ++q) grad[q] += (*v)[i + q];
    tmp.release();
  } catch (...) {
    tmp.release();
    throw;
  }
}

// Tensor-core tile product self-check (see lma_tc_gemm_check in lma.h).
void tc_gemm_check(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
                   float* C, int64_t ldc, int tile_n, cudaStream_t st) {
  Arena tmp;
  tmp.st = st;
  try {
    int* err = tmp.alloc<int>(1);
    LMA_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    dim3 grid((unsigned)((N + tile_n - 1) / tile_n), (unsigned)((M + 127) / 128));
    if (tile_n == 64) {
      const size_t sm = sizeof(tc::TcSmem<64>) + tc::kTcAlignSlack;
      LMA_CK(cudaFuncSetAttribute(k_tc_gemm<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      launch("k_tc_gemm", k_tc_gemm<64>, grid, 256, sm, st, A, lda, B, ldb, C, ldc, (int)M, (int)N, (int)K, err);
    } else {
      const size_t sm = sizeof(tc::TcSmem<128>) + tc::kTcAlignSlack;
      LMA_CK(cudaFuncSetAttribute(k_tc_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      launch("k_tc_gemm", k_tc_gemm<128>, grid, 256, sm, st, A, lda, B, ldb, C, ldc, (int)M, (int)N, (int)K, err);
    }
    int h = 0;
    LMA_CK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMA_CK(cudaStreamSynchronize(st));
    if (h) {
      fail(LMA_ERR_TIMEOUT, "tensor-core pipeline wait timed out");
      throw Fail{};
    }
    tmp.release();
  } catch (...) {
    tmp.release();
    throw;
  }
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the global step.
//
// For callers that cannot allocate device memory themselves on the call
// path: a serving runtime or framework that pre-provisions all device memory
// and forbids allocation while it handles a request, or a pipeline whose
// device memory is owned by another allocator.  The kernels below need
// scratch (the (npad + 1 + s) x npad factorisation buffer, the inverted
// diagonal tiles, a window descriptor and a status flag); this variant keeps
// all of it in one file-scope device array of fixed size, so the call itself
// never allocates.  The array is part of the library's image: every GPU that
// loads the library holds it (about 17 MB) until the process exits.
constexpr int kNoAllocMaxS = 1024;
constexpr int64_t kNoAllocBuf = (int64_t)(2 * kNoAllocMaxS + 1) * kNoAllocMaxS;  // doubles
constexpr int64_t kNoAllocDinv = (int64_t)kNoAllocMaxS * TB;                      // doubles
constexpr int64_t kNoAllocMeta = 64;                                               // Win + flag
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocBuf + kNoAllocDinv + kNoAllocMeta];

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is fetched once
// per device (with that device current) and cached.
static double* noalloc_scratch() {
  static std::mutex mu;
  static double* addr[256] = {};
  int dev = 0;
  LMA_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    fail(LMA_ERR_INTERNAL, "device index out of range");
    throw Fail{};
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fail(LMA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      throw Fail{};
    }
    addr[dev] = static_cast<double*>(p);
  }
  return addr[dev];
}

static __global__ void k_noalloc_setup(Win* wslot, Win w, int* flag) {
  *wslot = w;
  *flag = 0;
}

// C = I + A (A: s x s, ld s) with s identity rows appended and then the row
// y, the layout of k_build_global: identity rows first, so that they stay
// 64-aligned and the factorisation skips their tiles while still zero.
static __global__ void k_noalloc_build(const double* __restrict__ A, const double* __restrict__ y, int s, int npad,
                                       double* __restrict__ buf) {
  int64_t total = (int64_t)(npad + 1 + s) * npad;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  int i = (int)(e / npad), j = (int)(e % npad);
  double v;
  if (i < npad) {
    if (i < s && j < s) v = A[(int64_t)i * s + j] + (i == j ? 1.0 : 0.0);
    else v = (i == j) ? 1.0 : 0.0;
  } else if (i < npad + s) {
    v = ((i - npad) == j) ? 1.0 : 0.0;
  } else {
    v = (j < s) ? y[j] : 0.0;
  }
  buf[e] = v;
}

// beta = L_C^-T w with w = L_C^-1 y (the appended y row of the factor), one
// warp per row k of L_C^-T over many CTAs (coalesced row reads, lane sums
// combined by shuffles); CTA 0 also writes out[0] = w^T w, out[1] =
// log|I + A| and out[2] = the log-likelihood.
static __global__ void __launch_bounds__(NT) k_noalloc_finish(const double* __restrict__ buf, int s, int npad,
                                                              double quad, double logdet_R, double n,
                                                              double* __restrict__ beta, double* __restrict__ out) {
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
    const double wCw = red[0][0], ldC = 2.0 * red[1][0];
    out[0] = wCw;
    out[1] = ldC;
    out[2] = -0.5 * (quad - wCw) - 0.5 * (logdet_R + ldC) - 0.5 * n * log(2.0 * M_PI);
  }
}

void global_step_noalloc(int64_t s, int64_t n, const double* A, const double* y, double quad, double logdet_R,
                         double* beta, double* scalars, cudaStream_t st) {
  if (s < 1 || s > kNoAllocMaxS) {
    fail(LMA_ERR_INVALID_ARG, "lma_global_step_noalloc: s must lie in [1, " + std::to_string(kNoAllocMaxS) +
                                  "] (fixed size of its device scratch array)");
    throw Fail{};
  }
  Impl<float>::setup_attributes();
  double* base = noalloc_scratch();
  double* buf = base;
  double* dv = base + kNoAllocBuf;
  Win* wslot = reinterpret_cast<Win*>(base + kNoAllocBuf + kNoAllocDinv);
  int* flag = reinterpret_cast<int*>(base + kNoAllocBuf + kNoAllocDinv + 32);
  const int npad = (int)roundup(s, TB);
  Win w{};
  w.n = (int)s;
  w.npad = npad;
  w.rows = npad + 1 + (int)s;
  launch("k_noalloc_setup", k_noalloc_setup, 1, 1, 0, st, wslot, w, flag);
  launch("k_noalloc_build", k_noalloc_build, nblk((int64_t)(npad + 1 + s) * npad), NT, 0, st, A, y, (int)s, npad,
         buf);
  right_looking_fp64(st, w, wslot, buf, dv, flag, (int)s);
  launch("k_noalloc_finish", k_noalloc_finish, nblk(s, NT / 32), NT, 0, st, (const double*)buf, (int)s, npad, quad,
         logdet_R, (double)n, beta, scalars);
  int h = 0;
  LMA_CK(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  LMA_CK(cudaStreamSynchronize(st));
  if (h) {
    fail(LMA_ERR_NOT_PD, "I + A is not positive definite", -2);
    throw Fail{};
  }
}

template struct Impl<float>;
template struct Impl<double>;

}  // namespace lma
