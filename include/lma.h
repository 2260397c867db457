/*
 * lma.h — C ABI of the GB300 LMA library (low-rank-cum-Markov approximation
 * of Gaussian-process regression; Low, Yu, Chen, Jaillet, AAAI 2015).
 *
 * Problem statement (Sections 2-3 of the paper): training inputs D with
 * outputs y_D, a partition of D into blocks D_1..D_M, a support set S, a
 * Markov order B, the SE-ARD covariance of Section 5 with hyperparameters
 * (l_1..l_d, sigma_s, sigma_n) and a constant prior mean mu.
 *
 * Conventions for every entry point:
 *  - The caller owns every input and output buffer; no call keeps a caller
 *    pointer after it returns.  The library owns an lma_model until
 *    lma_model_free.
 *  - All GPU work is ordered on options->cuda_stream (a cudaStream_t passed as
 *    void*, NULL = the legacy default stream).  Every call synchronises that
 *    stream before returning, so outputs are valid on return.
 *  - Errors come back as lma_status codes; nothing aborts and no C++
 *    exception crosses the ABI.  lma_last_error_info gives details of the
 *    calling thread's last failure.
 *  - Index arrays (block_ptr, test_block_ptr) and hyperparameter vectors are
 *    always HOST memory.  Point arrays are host or device memory as the
 *    *_on_device flag says; device pointers must be on the current device.
 *  - All matrices are row-major, doubles.
 */
#ifndef LMA_H
#define LMA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LMA_OK = 0,
  LMA_ERR_INVALID_ARG = 1,  /* a size, pointer or partition is inconsistent            */
  LMA_ERR_NOT_PD = 2,       /* a residual window or Sigma-ddot_SS lost positive definiteness;
                               lma_last_error_info reports the block index (-1: support set,
                               -2: global summary)                                       */
  LMA_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed               */
  LMA_ERR_OOM = 4,          /* device memory allocation failed                           */
  LMA_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                             */
  LMA_ERR_INTERNAL = 6      /* unexpected internal state                                 */
} lma_status;

typedef enum {
  LMA_FP64 = 0,   /* plain FP64 GPU form: every step in double, one window per launch   */
  LMA_MIXED = 1   /* FP32 covariance tiles / factorisations / solves, batched over all
                     windows; FP64 for Sigma_SS, the global summary and all reductions   */
} lma_precision;

typedef struct lma_model lma_model;

/* The data (D, y_D), its partition, the support set and the Markov order.
 * Section 3: D is partitioned into M disjoint blocks D_1..D_M; the Markov
 * blanket of block m is D^B_m = D_{m+1} u ... u D_{min(m+B, M)}.          */
typedef struct {
  int64_t n;            /* |D|                                                  */
  int64_t d;            /* input dimension, 1..24                               */
  int64_t m_blocks;     /* M >= 1                                               */
  int64_t s;            /* |S| >= 1                                             */
  int64_t markov_order; /* B in [0, M-1]                                        */
  const double* X;      /* n*d inputs, rows grouped by block                    */
  const double* y;      /* n outputs                                            */
  const int64_t* block_ptr; /* M+1 offsets (HOST): block m owns rows
                               [block_ptr[m], block_ptr[m+1]); block_ptr[0]=0,
                               block_ptr[M]=n, every block non-empty            */
  const double* S;      /* s*d support inputs                                   */
  double mean;          /* constant prior mean mu                               */
  int inputs_on_device; /* 1: X, y, S are device pointers; 0: host pointers     */
} lma_problem;

/* SE-ARD hyperparameters (Section 5):
 *   sigma_xx' = sigma_s^2 exp(-1/2 sum_i (x_i - x'_i)^2 / l_i^2) + sigma_n^2 delta_xx'.
 * The noise term is applied to the D-D diagonal only; Sigma_SS and the
 * cross-covariances with S are noise-free.  `jitter` (absolute, >= 0) is
 * added to the diagonal of Sigma_SS wherever it appears (in Q and in
 * Sigma-ddot_SS).                                                           */
typedef struct {
  const double* log_ell; /* d log length-scales (HOST)                          */
  double log_sigma_s;    /* log signal standard deviation                       */
  double log_sigma_n;    /* log noise standard deviation                        */
  double jitter;         /* absolute diagonal jitter on Sigma_SS                */
} lma_hyper;

typedef struct {
  lma_precision precision;
  int reserved;          /* must be 0                                           */
  void* cuda_stream;     /* cudaStream_t or NULL                                */
} lma_options;

/* Fit: the local summaries of Definition 1 for every block, reduced into the
 * global summary of Definition 2, then Sigma-ddot_SS^-1 y-ddot_S (Theorem 2).
 * Per block m the residual R (Section 3: R = Sigma - Q, Q_BB' =
 * Sigma_BS Sigma_SS^-1 Sigma_SB') over D_m u D^B_m is factorised blanket-first
 * so that its trailing factor is a square root of R-dot_m^-1 (Lemma 1).
 * *out receives a model owned by the library.  In the mixed form a window
 * whose FP32 factorisation loses positive definiteness makes the library
 * redo the fit in the FP64 form (same problem and hyperparameters, no added
 * jitter); the model is then an FP64 model (lma_model_precision).  The same
 * holds for lma_fit_local, lma_fit_predict, lma_loglik and lma_loglik_grad.
 * Returns LMA_ERR_NOT_PD when a window is not positive definite in FP64
 * either, or when Sigma_SS or I + A (factorised in FP64 in both forms) is
 * not.                                                                     */
lma_status lma_fit(const lma_problem* problem, const lma_hyper* hyper,
                   const lma_options* options, lma_model** out);

/* Predictive mean and variance of Theorem 2 (equivalently Eqs. vapmu/vapvar)
 * for u test inputs XU (u*d) partitioned like D: test block n owns rows
 * [test_block_ptr[n], test_block_ptr[n+1]) (HOST, M+1 entries, may be empty).
 * noisy=1 returns the variance of the noisy output (sigma_uu includes
 * sigma_n^2, the paper's convention), noisy=0 that of the latent function.
 * mean_out / var_out hold u doubles each, in host or device memory as
 * io_on_device says (XU likewise).                                         */
lma_status lma_predict(const lma_model* model, int64_t u, const double* XU,
                       const int64_t* test_block_ptr, int noisy, int io_on_device,
                       double* mean_out, double* var_out);

/* lma_predict, enqueued: the call returns once the prediction is queued on
 * the model's stream (the cuda_stream of its fit), without waiting for it.
 * XU, mean_out and var_out must be device memory and stay valid until the
 * stream has passed the work (a stream synchronisation or lma_model_wait).
 * Argument errors are returned at once (LMA_ERR_INVALID_ARG, also for host
 * buffers); an error found on the device (a bounded pipeline wait that gave
 * up) is recorded in a status word of the model and returned by the next
 * lma_model_wait.  Calls on one model are ordered by its stream.  The
 * paper has no counterpart.                                                 */
lma_status lma_predict_async(lma_model* model, int64_t u, const double* XU, const int64_t* test_block_ptr,
                             int noisy, double* mean_out, double* var_out);

/* Waits until the model's stream has finished everything queued on it and
 * returns the device status of the lma_predict_async calls since the last
 * wait (LMA_ERR_TIMEOUT if a bounded device wait gave up), clearing it.     */
lma_status lma_model_wait(lma_model* model);

/* lma_predict plus the predictive covariance of every test block: for the
 * test points of block n, Eq. (vapvar) restricted to U_n x U_n (these pairs
 * are in-band, so Sigma-bar_UU = Sigma_UU there), evaluated by the same local
 * route as the variance.  cov_out receives the blocks one after the other,
 * block n as a row-major |U_n| x |U_n| matrix, sum_n |U_n|^2 doubles in
 * total (host or device memory as io_on_device says, like mean_out and
 * var_out).  Errors as in lma_predict.                                     */
lma_status lma_predict_cov(const lma_model* model, int64_t u, const double* XU,
                           const int64_t* test_block_ptr, int noisy, int io_on_device,
                           double* mean_out, double* var_out, double* cov_out);

/* lma_predict plus chosen blocks of the predictive covariance between test
 * blocks: for each requested pair (n, n'), Eq. (vapvar) on U_n x U_n'
 * (Sigma-bar by Eqs. ares / acov, so off the band Sigma-bar_UU is the
 * approximation's, not Sigma_UU).  block_pairs (host memory) holds 2*n_pairs
 * block indices n_0, n'_0, n_1, n'_1, ..., each in [0, M); cov_out receives
 * the blocks in request order, block i as a row-major |U_n_i| x |U_n'_i|
 * matrix (host or device memory as io_on_device says), sum_i |U_n_i| |U_n'_i|
 * doubles in total; a pair with an empty test block contributes nothing.
 * Requesting every (n, n') gives the whole |U| x |U| covariance.  Evaluation:
 * the residual part R-bar_UU - R-bar_UD R-bar_DD^-1 R-bar_DU vanishes between
 * test blocks more than B apart (Eq. ares passes through the training
 * blankets only) and within the band is a sum of products of the local
 * route's window right-hand sides; the low-rank part is g_u . g_u' with
 * g = L_C^-1 h as in the variance.  noisy adds sigma_n^2 where a point meets
 * itself.  Errors as in lma_predict, and LMA_ERR_INVALID_ARG for a negative
 * n_pairs, a null block_pairs with n_pairs > 0 or a block index out of
 * range.                                                                    */
lma_status lma_predict_cov_blocks(const lma_model* model, int64_t u, const double* XU,
                                  const int64_t* test_block_ptr, int noisy, int io_on_device,
                                  int64_t n_pairs, const int64_t* block_pairs,
                                  double* mean_out, double* var_out, double* cov_out);

/* lma_fit followed by lma_predict in one call: the FP64 global step
 * (Definition 2) runs on a library-owned second stream while the
 * prediction's kernels that do not need its results run on cuda_stream, and
 * the rest of the prediction waits for it.  In the mixed form the test
 * points' right-hand sides R_{W_m u} are appended to the window buffers as
 * extra rows, so the fit's own sweep turns them into the rows
 * (L_m^-1 R_{W_m u})^T of the local route (Lemma 1) and no separate
 * prediction sweep runs: the results equal lma_fit + lma_predict to FP32
 * accuracy (the FP64 form's exactly).  Arguments as in lma_fit and
 * lma_predict; `out` may be NULL (the model is then freed) or receives the
 * model (free with lma_model_free).  Outputs are valid when the call
 * returns.  Errors as in lma_fit and lma_predict; on an error nothing is
 * returned in *out.                                                        */
lma_status lma_fit_predict(const lma_problem* problem, const lma_hyper* hyper,
                           const lma_options* options, int64_t u, const double* XU,
                           const int64_t* test_block_ptr, int noisy, int io_on_device,
                           double* mean_out, double* var_out, lma_model** out);

/* log N(y_D; mu, Sigma-bar_DD) of a fitted model (Sigma-bar by Eq. acov). */
lma_status lma_model_loglik(const lma_model* model, double* out);

/* Fit without keeping a model and return log N(y_D; mu, Sigma-bar_DD).     */
lma_status lma_loglik(const lma_problem* problem, const lma_hyper* hyper,
                      const lma_options* options, double* out);

/* Log-likelihood and its gradient with respect to
 * (log l_1..log l_d, log sigma_s, log sigma_n) (d+2 doubles, host memory),
 * by a hand-written adjoint that recomputes each window's residual and
 * factor instead of storing them.  The paper does not differentiate its
 * likelihood; jitter and the partition are held fixed.                    */
lma_status lma_loglik_grad(const lma_problem* problem, const lma_hyper* hyper,
                           const lma_options* options, double* loglik_out,
                           double* grad_out);

/* Global-summary diagnostics of a fitted model, in the whitened support
 * coordinates V = L_SS^-1 Sigma_SD (L_SS the Cholesky factor of Sigma_SS):
 *   A_out   (s*s, host): sum_m Sigma-dot^mT R-dot_m Sigma-dot^m whitened,
 *                        i.e. L_SS^-1 (Sigma-ddot_SS - Sigma_SS) L_SS^-T
 *   y_out   (s, host):   L_SS^-1 y-ddot_S
 *   scalars (4, host):   quad = sum_m y-dot_m^T R-dot_m y-dot_m,
 *                        log|R-bar_DD|, log|I + A|, loglik
 * Any output pointer may be NULL.                                          */
lma_status lma_model_summary(const lma_model* model, double* A_out, double* y_out,
                             double* scalars_out);

/* Partitioned fit (Remark 1: machines compute the local summaries of their
 * own blocks, Definition 1, and a master sums them into the global summary,
 * Definition 2).  Three calls per shard:
 *
 * lma_fit_local: windows D_m u D^B_m of blocks [win_begin, own_end) of
 *   `problem` are formed and factorised, and the local summaries of blocks
 *   [own_begin, own_end) are summed.  `problem` is normally a sub-problem
 *   holding the shard's blocks plus the B blocks after them (the blankets of
 *   its last blocks) and, for prediction, the B blocks before them (win_begin
 *   = own_begin - B, so that every window a test block of the shard needs is
 *   present).  0 <= win_begin <= own_begin < own_end <= m_blocks.  The model
 *   cannot predict or report a log-likelihood before lma_model_set_global.
 *
 * lma_model_local_summary: the shard's (s+1) x (s+1) FP64 Gram G, row-major,
 *   G[0][0] = sum y-dot_m^T R-dot_m y-dot_m, G[0][1+i] = G[1+i][0] =
 *   (L_SS^-1 y-ddot)_i, G[1+i][1+j] = A_ij (whitened, as in
 *   lma_model_summary), into G_out (device memory if on_device, else host),
 *   and the shard's sum of log|R-dot_m^-1| into *logdet_out (host).  The sum
 *   over shards of both is the whole fit's.
 *
 * lma_model_set_global: given the summed G (device or host) and log-det sum,
 *   and the total number of training points n_total, performs the global
 *   step (Definition 2, Eq. pitck) on this shard's model; afterwards
 *   lma_predict works for test blocks whose windows m in [n - B, n] lie in
 *   [win_begin, own_end), and lma_model_loglik returns the whole problem's
 *   log-likelihood.  Errors: LMA_ERR_INVALID_ARG for bad ranges or sizes,
 *   LMA_ERR_NOT_PD as in lma_fit.                                           */
lma_status lma_fit_local(const lma_problem* problem, const lma_hyper* hyper,
                         const lma_options* options, int64_t win_begin, int64_t own_begin,
                         int64_t own_end, lma_model** out);
lma_status lma_model_local_summary(const lma_model* model, double* G_out, double* logdet_out,
                                   int on_device);
lma_status lma_model_set_global(lma_model* model, const double* G, double logdet_R,
                                int64_t n_total, int on_device);

/* Gradient of the log-likelihood of a fitted model with respect to
 * (log l_1..log l_d, log sigma_s, log sigma_n) (d+2 doubles, host), by the
 * hand adjoint of lma_loglik_grad applied to the windows of the blocks whose
 * summaries the model holds: all of them for a model of lma_fit, blocks
 * [own_begin, own_end) for one of lma_fit_local whose global step is done
 * (lma_model_set_global).  Every step of the adjoint after the window terms
 * is linear in them, so the shards' results add up to the whole gradient:
 * a sharded gradient is one all-reduce of d+2 values (the paper does not
 * differentiate its likelihood; jitter and the partition are held fixed).
 * The model's stored window factors are reused.  LMA_ERR_INVALID_ARG before
 * the global step.                                                          */
lma_status lma_model_loglik_grad(lma_model* model, double* grad_out);

/* The residual R = Sigma - Q over the window D_m u D^B_m of block m, as an
 * n_w x n_w matrix in natural row order (host memory, n_w = number of rows
 * of D_m u D^B_m), evaluated by the selected precision's kernels before any
 * factorisation.  For parity tests of the residual-formation kernel.      */
lma_status lma_window_residual(const lma_problem* problem, const lma_hyper* hyper,
                               const lma_options* options, int64_t m, double* out);

/* Number of rows of the window D_m u D^B_m (0 on invalid arguments).      */
int64_t lma_window_rows(const lma_problem* problem, int64_t m);

void lma_model_free(lma_model* model);

/* The form a model was fitted in: the requested one, or LMA_FP64 after the
 * mixed form's FP64 retry (lma_fit).  LMA_FP64 for NULL.                   */
lma_precision lma_model_precision(const lma_model* model);

const char* lma_status_string(lma_status status);

/* Details of the calling thread's last failure: the block index for
 * LMA_ERR_NOT_PD (-1 = Sigma_SS, -2 = Sigma-ddot_SS, otherwise the block),
 * and a message that stays valid until the thread's next call.  Either
 * pointer may be NULL.                                                    */
lma_status lma_last_error_info(int64_t* failed_block, const char** message);

/* Number of kernels this library has launched in the calling process.     */
int64_t lma_kernel_launch_count(void);

/* Diagnostic (not part of the paper's method): C = A B^T computed by this
 * library's tensor-core tile product (tcgen05, FP32 operands split into TF32
 * hi/lo halves, three MMAs per product, FP32 accumulation in tensor memory),
 * for self-tests of that building block.  A is M x K, B is N x K, C is M x N,
 * all row-major FP32 DEVICE pointers with leading dimensions lda, ldb, ldc;
 * K must be a multiple of 32, lda and ldb multiples of 4, A and B 16-byte
 * aligned; tile_n is the tile width (64 or 128).  Returns LMA_ERR_TIMEOUT if
 * a bounded device wait gave up.                                         */
lma_status lma_tc_gemm_check(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                             const float* B, int64_t ldb, float* C, int64_t ldc, int tile_n,
                             void* cuda_stream);

/* Global step of the fit without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory on their call path (a serving runtime or framework that
 * pre-provisions all device memory and forbids allocation while handling a
 * request, or a caller whose device memory belongs to another allocator).
 *
 * From the whitened summaries of a fit (lma_model_summary: A is s x s, y has
 * s entries, quad and log|R-bar_DD| are scalars; n = |D|) it factorises
 * I + A in FP64 and returns beta = (I + A)^-1 y in beta_out (s doubles) and
 * scalars_out = { y^T (I + A)^-1 y, log|I + A|, log N(y_D; mu, Sigma-bar_DD) }
 * (3 doubles).  A, y, beta_out and scalars_out are DEVICE pointers owned by
 * the caller; the work is ordered on cuda_stream and synchronised before the
 * call returns.
 *
 * All scratch lives in one fixed device array inside the library, sized for
 * s <= 1024 (about 17 MB, held by every GPU that loads the library until the
 * process exits); larger s returns LMA_ERR_INVALID_ARG.  The call allocates
 * nothing.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the array and it keeps the last call's contents, so
 * calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them.  LMA_ERR_NOT_PD (block -2) if I + A is not positive
 * definite.                                                                */
lma_status lma_global_step_noalloc(int64_t s, int64_t n, const double* A, const double* y,
                                   double quad, double logdet_R, double* beta_out,
                                   double* scalars_out, void* cuda_stream);

/* Launch profiler (a single-threaded diagnostic, off by default; not part of
 * the paper's method).  lma_profile_start clears earlier records and, until
 * lma_profile_stop, brackets every launch whose kernel name contains
 * name_filter (NULL or "" = every launch) with a CUDA event pair recorded on
 * the launching stream.  lma_profile_stop waits for those events, writes the
 * distinct kernel names, newline-separated, into names (names_cap bytes,
 * NUL-terminated, may be NULL) and their summed milliseconds and launch
 * counts into total_ms / launches (cap entries each, may be NULL), and
 * returns the number of distinct names.                                   */
void lma_profile_start(const char* name_filter);
int lma_profile_stop(char* names, int names_cap, double* total_ms, int64_t* launches, int cap);

/* Per-launch trace of the records made since lma_profile_start (call before
 * lma_profile_stop, which discards them).  For record i < min(count, cap),
 * t0_ms[i] / t1_ms[i] are its start / end events' times in milliseconds
 * after the first record's start event (events on different streams of one
 * device share that clock), and names holds the records' kernel names in
 * order, newline-separated (names_cap bytes, NUL-terminated, may be NULL).
 * Waits for the recorded events; returns the number of records.           */
int lma_profile_trace(char* names, int names_cap, double* t0_ms, double* t1_ms, int cap);

/* Launch-shape autotuner (not part of the paper's method).  Some launches
 * have several valid shapes (the number of window groups of the summary
 * Gram, ...): the first call that meets a new shape class times each
 * candidate on its own data (CUDA events on the call's stream; only launches
 * that can be repeated without changing results) and keeps the fastest for
 * the rest of the process, per device; with the environment variable
 * LMA_TUNE_CACHE naming a file, choices are also appended there and read back
 * by later processes.  lma_autotune(0) (or LMA_AUTOTUNE=0 in the environment)
 * makes every launch take the shape its cost model predicts; lma_autotune(1)
 * turns timing back on (the default).  Results differ between shapes only by
 * the order of FP64 partial sums.                                          */
void lma_autotune(int enabled);

/* Frees the device workspace that the fit entry points (lma_fit,
 * lma_fit_predict, lma_fit_local, lma_loglik, lma_loglik_grad) of the calling
 * host thread keep on the current device from one call to the next: the
 * bfloat16 planes of K_SD read by the mixed form's projection, then those of
 * the summary rows read by its Gram (3 N rnd64(|S|) or 3 M (|S|+1) rnd64(b)
 * 16-bit values, whichever is larger; about 25 GB at N = 2M, |S| = 2,048).
 * Taking that much from the stream-ordered pool in every call cost tens of
 * milliseconds of host time while the GPU waited, so the library holds it;
 * the next fit allocates it again.  Waits for the device first.  Returns
 * LMA_OK, or a CUDA error status.                                          */
lma_status lma_workspace_release(void);

/* Pins the launch shape of every shape class whose key starts with `prefix`
 * (the keys are those of lma_autotune_report, e.g. "fp64 factor" for the
 * FP64 factorisations of Sigma_SS and I + A, whose choices are 0 one launch
 * per panel, 1 two launches per panel, 2-4 one cooperative launch with 1, 2
 * or 4 CTAs per SM, 5 the dataflow form with per-tile flags) to `choice`, on every device, ahead of timing, of the
 * cache file and of lma_autotune(0).  A choice that is not among a class's
 * candidates is ignored for that class; the latest matching pin wins.
 * prefix NULL removes every pin.                                            */
void lma_autotune_pin(const char* prefix, int choice);

/* Text report of the tuner's choices, one line per shape class:
 * "device | key | choice | candidate:ms ...", NUL-terminated into buf (cap
 * bytes, may be NULL).  Returns the full length of the report.            */
int lma_autotune_report(char* buf, int cap);

#ifdef __cplusplus
}
#endif

#endif /* LMA_H */
