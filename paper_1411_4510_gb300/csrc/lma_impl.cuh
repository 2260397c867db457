// Host orchestration of the LMA hot path (fit, predict) for one precision.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/lma.h"

#include "lma_types.cuh"

namespace lma {

// ---- error state and bookkeeping -------------------------------------------
struct ErrState {
  lma_status status = LMA_OK;
  int64_t block = 0;
  std::string msg;
};
ErrState& err();
lma_status fail(lma_status st, const std::string& msg, int64_t block = 0);
void count_launch(int64_t n = 1);

struct Fail {};  // thrown inside the library only, caught at the ABI boundary

#define LMA_CK(call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      ::lma::fail(e_ == cudaErrorMemoryAllocation ? LMA_ERR_OOM : LMA_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
      throw ::lma::Fail{};                                                               \
    }                                                                                    \
  } while (0)

#define LMA_LAUNCHED()                                                                   \
  do {                                                                                   \
    ::lma::count_launch();                                                               \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess) {                                                             \
      ::lma::fail(LMA_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
      throw ::lma::Fail{};                                                               \
    }                                                                                    \
  } while (0)

// Stream-ordered device allocations released together.
struct Arena {
  cudaStream_t st = nullptr;
  std::vector<void*> ptrs;
  template <typename X> X* alloc(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    LMA_CK(cudaMallocAsync(&p, count * sizeof(X), st));
    ptrs.push_back(p);
    return static_cast<X*>(p);
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
  }
  // frees one buffer of this arena early (stream-ordered)
  void free_one(void* p) {
    for (size_t i = 0; i < ptrs.size(); ++i)
      if (ptrs[i] == p) {
        cudaFreeAsync(p, st);
        ptrs.erase(ptrs.begin() + (long)i);
        return;
      }
  }
};

// Optional launch profiler: when enabled, a CUDA event pair is recorded on the
// launching stream around every launch whose name matches the filter.
namespace prof {
bool active(const char* name);
void start(const char* name, cudaStream_t st);
void stop(cudaStream_t st);
}  // namespace prof

// Launch a kernel, count it, check the launch status and (optionally) time it.
template <typename... KArgs, typename... Args>
inline void launch(const char* name, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                   Args... args) {
  const bool p = prof::active(name);
  if (p) prof::start(name, st);
  kern<<<grid, block, smem, st>>>(static_cast<KArgs>(args)...);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (p) prof::stop(st);
  if (e != cudaSuccess) {
    fail(LMA_ERR_CUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
    throw Fail{};
  }
}

// launch() with programmatic stream serialisation: the kernel may become
// resident while its predecessor in the stream still runs, which hides the
// launch latency of long chains of short dependent launches (the panel steps
// of the factorisations).  Only for kernels that call grid_dep_wait() first.
template <typename... KArgs, typename... Args>
inline void launch_pdl(const char* name, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  const bool p = prof::active(name);
  if (p) prof::start(name, st);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
  count_launch();
  if (e == cudaSuccess) e = cudaGetLastError();
  if (p) prof::stop(st);
  if (e != cudaSuccess) {
    fail(LMA_ERR_CUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
    throw Fail{};
  }
}

// launch() as a cooperative launch: every CTA of the grid is resident at
// once, so the kernel's CTAs may wait on one another (grid barriers).
template <typename... KArgs, typename... Args>
inline void launch_coop(const char* name, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                        Args... args) {
  const bool p = prof::active(name);
  if (p) prof::start(name, st);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
  count_launch();
  if (e == cudaSuccess) e = cudaGetLastError();
  if (p) prof::stop(st);
  if (e != cudaSuccess) {
    fail(LMA_ERR_CUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
    throw Fail{};
  }
}

inline int64_t roundup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Page-locked staging for the small index tables a call uploads (window
// descriptors, work-item lists): from pinned memory cudaMemcpyAsync is a
// true asynchronous copy, while a pageable source can make the driver wait
// for the stream.  One buffer per host thread, handed out by a bump pointer;
// the entry points reset it after their final stream synchronisation.  If it
// fills up, the device is synchronised (every staged copy has landed) and the
// buffer grows.
struct Staging {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  bool hold = false;  // an enqueued call's uploads may still be in flight: no reuse before a device sync
  std::vector<char*> retired;  // outgrown buffers whose uploads may still be in flight
  void* take(size_t bytes, cudaStream_t st);
  // after the calling thread's work has completed: the buffer may be reused
  // from its start and the outgrown ones freed
  void reset();
};
Staging& staging();

// Device workspace for the two largest transient buffers of a fit (the
// bfloat16 planes of K_SD that the projection reads, then those of the
// summary rows that the Gram reads; about 25 GB each at N = 2M, |S| = 2,048),
// kept from call to call, one per host thread and device.  Taking buffers of
// that size from the stream-ordered pool cost 18-21 ms of host time in every
// call (the pool mapped them anew each time), during which the GPU went
// idle.  Only the synchronous fit entry points use it, in stream order, and
// their work has completed when they return, so calls never overlap on it.
// Grows (after a device synchronisation) when a larger one is asked for;
// lma_workspace_release frees it.
void* fit_workspace(size_t bytes);
void fit_workspace_release();

// Upload `bytes` of host data to device memory `dst` through the staging buffer.
inline void stage_copy(void* dst, const void* host, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return;
  void* h = staging().take(bytes, st);
  memcpy(h, host, bytes);
  LMA_CK(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, st));
}
inline unsigned nblk(int64_t n, int t = NT) { return (unsigned)((n + t - 1) / t); }

// Everything a fitted model keeps on the device.
struct ModelCore {
  lma_precision prec = LMA_MIXED;
  cudaStream_t st = nullptr;
  int64_t n = 0, d = 0, M = 0, s = 0, B = 0;
  double mu = 0, ss2 = 0, sn2 = 0;
  std::vector<double> inv_ell;
  std::vector<int64_t> bptr;
  std::vector<Win> wins;
  Arena keep;                 // buffers owned by the model
  double* inv_ell_d = nullptr;
  void* xsT = nullptr;        // n*d scaled inputs (T)
  void* ssT = nullptr;        // s*d scaled support inputs (T)
  void* ET = nullptr;         // s*s, ET[k][i] = (L_SS^-1)[i][k]   (T)
  void* Vt = nullptr;         // n*s whitened support coordinates  (T)
  uint16_t* vb3 = nullptr;    // three bfloat16 planes of Vt in reversed point order, row length
  int ldvs = 0;               //   ldvs (a multiple of 64; mixed form on the tensor cores only)
  void* wbuf = nullptr;       // window buffers (T)
  void* dinv = nullptr;       // inverted diagonal tiles (T)
  void* ew = nullptr;         // per-window L^-1 e (T)
  Win* wins_d = nullptr;
  double* G = nullptr;        // (s+1)^2 global Gram [quad, y; y, A]
  double* beta = nullptr;     // s
  void* LcT = nullptr;        // s*s, (L_C^-1)[i][k] at [k][i]   (T)
  double quad = 0, wCw = 0, logdetC = 0, logdetR = 0, loglik = 0;
  uint16_t* linv3 = nullptr;  // three bfloat16 planes of L_SS^-1 (mixed form on the tensor cores), brows x ldk each
  uint16_t* lcinv3 = nullptr; // the same for L_C^-1 (global step)
  int ldk = 0, brows = 0;     // plane row length (s rounded up to 64) and rows per plane (s rounded up to 128)
  double* kss = nullptr;      // Sigma_SS factor buffer: L_SS (rows < npS) and L_SS^-T rows (FP64)
  double* ss64 = nullptr;     // s*d scaled support inputs (FP64)
  int npS = 0;
  int64_t w0 = 0;             // block index of the first window (partitioned fits)
  int64_t own_b = 0, own_e = 0;  // blocks whose local summaries this model holds
  int* async_err = nullptr;   // device status word of the enqueued predictions (lma_predict_async)
  bool have_global = false;   // global step done (prediction possible)
  // device status words, checked once at the end of a call:
  // [0] Sigma_SS pivot failure (+1 column), [1] I + A pivot failure,
  // [2] tensor-core pipeline wait timed out
  int* flags = nullptr;
  int* winfo = nullptr;       // per-window pivot failure (+1 column), 0 = fine
  double* ldR_d = nullptr;    // device sum of log|R-dot_m^-1| over the owned windows
  double* sc_d = nullptr;     // device scalars of the global step
};

}  // namespace lma

struct lma_model {
  lma::ModelCore core;
};

namespace lma {

// Test points of lma_fit_predict whose right-hand sides R_{W_m u} are
// appended to the window buffers as extra rows, below the s + 1 rows of
// [r | Vt_W], so that the fit's own sweep turns them into (L_m^-1 R_{W_m u})^T
// (the rows the prediction's local route needs) and no separate prediction
// sweep runs.  Window m carries the test rows of blocks m .. m + B in block
// order.  xu / Vu (scaled test inputs, their whitened support coordinates)
// are kept in `keep` for the prediction.
struct FusedTest {
  int64_t U = 0;
  const double* XU = nullptr;
  const int64_t* tptr = nullptr;
  int on_device = 0;
  Arena keep;
  void* xu = nullptr;
  void* Vu = nullptr;
};

template <typename T>
struct Impl {
  // prepares inputs, Sigma_SS factor and Vt (shared by fit / residual / grad)
  static void prepare(ModelCore& mc, const lma_problem* P, const lma_hyper* H, Arena& tmp,
                      const double** X_d, const double** y_d);
  static void fit(ModelCore& mc, const lma_problem* P, const lma_hyper* H);
  static void fit_local(ModelCore& mc, const lma_problem* P, const lma_hyper* H, int64_t w_begin, int64_t own_begin,
                        int64_t own_end, FusedTest* ft = nullptr);
  // right-hand sides of ft's test points into the window buffers (before the sweep)
  static void fused_rhs(ModelCore& mc, FusedTest& ft, Arena& tmp);
  static void fit_global(ModelCore& mc, int64_t n_total, cudaStream_t on = nullptr);
  // waits for the stream and turns the status words into an error (if any);
  // global: also reads the global step's scalars and forms the loglik
  static void check(ModelCore& mc, bool global, int64_t n_total, bool logdet_from_device);
  static void predict(const ModelCore& mc, int64_t U, const double* XU, const int64_t* tptr, int noisy,
                      int on_device, double* mean, double* var, cudaEvent_t global_done = nullptr,
                      double* cov = nullptr, FusedTest* ft = nullptr, int* async_err = nullptr,
                      const int64_t* cov_pairs = nullptr, int64_t n_cov_pairs = -1);
  static void fit_predict(ModelCore& mc, const lma_problem* P, const lma_hyper* H, int64_t U, const double* XU,
                          const int64_t* tptr, int noisy, int on_device, double* mean, double* var);
  static void window_residual(ModelCore& mc, const lma_problem* P, const lma_hyper* H, int64_t m, double* out);
  static void loglik_grad(ModelCore& mc, const lma_problem* P, const lma_hyper* H, double* ll, double* grad);
  // gradient terms of windows [k_lo, k_hi) of a model with its global step done (d+2 doubles, host)
  static void grad_windows(ModelCore& mc, int64_t k_lo, int64_t k_hi, double* grad);
  static void setup_attributes();
};

void tc_gemm_check(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
                   float* C, int64_t ldc, int tile_n, cudaStream_t st);

void global_step_noalloc(int64_t s, int64_t n, const double* A, const double* y, double quad, double logdet_R,
                         double* beta, double* scalars, cudaStream_t st);

// builds the window descriptors of a partition (Section 3: W_m = D_m u D^B_m)
// for blocks [m_begin, m_end) (m_end < 0: all)
void make_windows(const std::vector<int64_t>& bptr, int64_t B, int64_t s, size_t elem, std::vector<Win>& wins,
                  int64_t& buf_elems, int64_t& dinv_elems, int64_t& ew_elems, int64_t m_begin = 0,
                  int64_t m_end = -1, const std::vector<int>* test_rows = nullptr);

// Prediction pairs (test block n, window m in [n - B, n]) and per test block
// (first pair, pair count, first test row, test rows).  fused: P rows of
// pair (n, m) are window m's appended test rows (FusedTest); otherwise they
// are packed in a separate buffer of *p_elems elements.
void make_pairs(const std::vector<Win>& wins, int64_t w0, int64_t M, int64_t B, int64_t s, const int64_t* tptr,
                bool fused, std::vector<Pair>& pairs, std::vector<int4>& tb, int64_t* p_elems);
// number of appended test rows of each window of a whole fit (FusedTest)
std::vector<int> fused_test_rows(int64_t M, int64_t B, const int64_t* tptr);

// sweep helpers (defined per precision)
template <typename T>
void chol_sweep(cudaStream_t st, const std::vector<Win>& wins, Win* wins_d, T* buf, T* dinv, int* info,
                bool batched, int* tc_err);

}  // namespace lma
