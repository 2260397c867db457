// C ABI of the LMA library: argument checks, dispatch by precision, error
// reporting.  No C++ exception crosses this file's functions.
#include <math.h>

#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "lma_impl.cuh"

namespace lma {

ErrState& err() {
  static thread_local ErrState e;
  return e;
}

lma_status fail(lma_status st, const std::string& msg, int64_t block) {
  ErrState& e = err();
  e.status = st;
  e.block = block;
  e.msg = msg;
  return st;
}

namespace prof {
static bool g_on = false;
static std::string g_filter;
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_pool;

static cudaEvent_t take() {
  cudaEvent_t e = nullptr;
  if (!g_pool.empty()) {
    e = g_pool.back();
    g_pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  return e;
}
bool active(const char* name) { return g_on && (g_filter.empty() || strstr(name, g_filter.c_str()) != nullptr); }
void start(const char* name, cudaStream_t st) {
  Rec r{name, take(), take()};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
}
void stop(cudaStream_t st) { cudaEventRecord(g_recs.back().b, st); }
}  // namespace prof

static std::atomic<int64_t> g_launches{0};
void count_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static void init_pool() {
  static bool done = false;
  if (done) return;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  done = true;
}

static lma_status check_problem(const lma_problem* P, const lma_hyper* H, const lma_options* O) {
  if (!P || !H || !O) return fail(LMA_ERR_INVALID_ARG, "null problem, hyper or options");
  if (P->n < 1 || P->d < 1 || P->d > MAXD || P->s < 1 || P->m_blocks < 1)
    return fail(LMA_ERR_INVALID_ARG, "sizes out of range (n>=1, 1<=d<=24, s>=1, M>=1)");
  if (P->m_blocks > 65535) return fail(LMA_ERR_INVALID_ARG, "at most 65535 blocks");
  if (P->markov_order < 0 || P->markov_order > P->m_blocks - 1)
    return fail(LMA_ERR_INVALID_ARG, "Markov order B must lie in [0, M-1]");
  if (!P->X || !P->y || !P->S || !P->block_ptr || !H->log_ell)
    return fail(LMA_ERR_INVALID_ARG, "null data pointer");
  if (O->precision != LMA_FP64 && O->precision != LMA_MIXED) return fail(LMA_ERR_INVALID_ARG, "unknown precision");
  if (O->reserved != 0) return fail(LMA_ERR_INVALID_ARG, "options.reserved must be 0");
  if (P->block_ptr[0] != 0 || P->block_ptr[P->m_blocks] != P->n)
    return fail(LMA_ERR_INVALID_ARG, "block_ptr must start at 0 and end at n");
  int64_t maxwin = 0;
  for (int64_t m = 0; m < P->m_blocks; ++m) {
    if (P->block_ptr[m + 1] <= P->block_ptr[m])
      return fail(LMA_ERR_INVALID_ARG, "block " + std::to_string(m) + " is empty or block_ptr decreases", m);
    int64_t last = m + P->markov_order < P->m_blocks - 1 ? m + P->markov_order : P->m_blocks - 1;
    int64_t nw = P->block_ptr[last + 1] - P->block_ptr[m];
    if (nw > maxwin) maxwin = nw;
  }
  if (maxwin > (1 << 20)) return fail(LMA_ERR_INVALID_ARG, "window too large");
  for (int64_t q = 0; q < P->d; ++q)
    if (!isfinite(H->log_ell[q])) return fail(LMA_ERR_INVALID_ARG, "non-finite log length-scale");
  if (!isfinite(H->log_sigma_s) || !isfinite(H->log_sigma_n) || !isfinite(H->jitter) || H->jitter < 0)
    return fail(LMA_ERR_INVALID_ARG, "non-finite hyperparameter or negative jitter");
  if (!isfinite(P->mean)) return fail(LMA_ERR_INVALID_ARG, "non-finite mean");
  return LMA_OK;
}

template <class F>
static lma_status guarded(F f) {
  err().status = LMA_OK;
  err().msg.clear();
  err().block = 0;
  try {
    init_pool();
    f();
  } catch (const Fail&) {
    return err().status == LMA_OK ? LMA_ERR_INTERNAL : err().status;
  } catch (const std::bad_alloc&) {
    return fail(LMA_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(LMA_ERR_INTERNAL, "unexpected exception");
  }
  return LMA_OK;
}

// The mixed form factorises the windows in FP32, which can lose positive
// definiteness where FP64 does not (a residual whose smallest eigenvalue is
// below the FP32 rounding of its O(sigma_s^2) entries).  Such a fit is redone
// in the FP64 form with the same problem and hyperparameters (no jitter is
// added: that would change R); the model is then an FP64 model
// (lma_model_precision).  Sigma_SS and I + A (failed block -1 / -2) are
// factorised in FP64 in both forms and are not retried.
static bool retry_in_fp64(lma_status st, lma_precision prec) {
  return st == LMA_ERR_NOT_PD && prec == LMA_MIXED && err().block >= 0;
}

static void drop_model(lma_model* md) {
  md->core.keep.release();
  cudaStreamSynchronize(md->core.st);
  delete md;
}

// A fresh model on the caller's stream in the given form.
static lma_model* new_model(const lma_options* O, lma_precision prec) {
  lma_model* md = new (std::nothrow) lma_model();
  if (!md) return nullptr;
  md->core.prec = prec;
  md->core.st = (cudaStream_t)O->cuda_stream;
  md->core.keep.st = md->core.st;
  return md;
}

}  // namespace lma

using namespace lma;

extern "C" {

lma_status lma_fit(const lma_problem* P, const lma_hyper* H, const lma_options* O, lma_model** out) {
  if (!out) return fail(LMA_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  lma_status cs = check_problem(P, H, O);
  if (cs != LMA_OK) return cs;
  lma_model* md = new (std::nothrow) lma_model();
  if (!md) return fail(LMA_ERR_OOM, "host allocation failed");
  md->core.prec = O->precision;
  md->core.st = (cudaStream_t)O->cuda_stream;
  md->core.keep.st = md->core.st;
  lma_status st = guarded([&] {
    if (O->precision == LMA_MIXED)
      Impl<float>::fit(md->core, P, H);
    else
      Impl<double>::fit(md->core, P, H);
  });
  if (retry_in_fp64(st, O->precision)) {
    drop_model(md);
    md = new_model(O, LMA_FP64);
    if (!md) return fail(LMA_ERR_OOM, "host allocation failed");
    st = guarded([&] { Impl<double>::fit(md->core, P, H); });
  }
  if (st != LMA_OK) {
    drop_model(md);
    return st;
  }
  *out = md;
  return LMA_OK;
}

lma_status lma_fit_local(const lma_problem* P, const lma_hyper* H, const lma_options* O, int64_t win_begin,
                         int64_t own_begin, int64_t own_end, lma_model** out) {
  if (!out) return fail(LMA_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  lma_status cs = check_problem(P, H, O);
  if (cs != LMA_OK) return cs;
  if (win_begin < 0 || win_begin > own_begin || own_begin >= own_end || own_end > P->m_blocks)
    return fail(LMA_ERR_INVALID_ARG, "need 0 <= win_begin <= own_begin < own_end <= m_blocks");
  lma_model* md = new (std::nothrow) lma_model();
  if (!md) return fail(LMA_ERR_OOM, "host allocation failed");
  md->core.prec = O->precision;
  md->core.st = (cudaStream_t)O->cuda_stream;
  md->core.keep.st = md->core.st;
  lma_status st = guarded([&] {
    if (O->precision == LMA_MIXED) {
      Impl<float>::fit_local(md->core, P, H, win_begin, own_begin, own_end);
      Impl<float>::check(md->core, false, 0, true);
    } else {
      Impl<double>::fit_local(md->core, P, H, win_begin, own_begin, own_end);
      Impl<double>::check(md->core, false, 0, true);
    }
  });
  if (retry_in_fp64(st, O->precision)) {
    drop_model(md);
    md = new_model(O, LMA_FP64);
    if (!md) return fail(LMA_ERR_OOM, "host allocation failed");
    st = guarded([&] {
      Impl<double>::fit_local(md->core, P, H, win_begin, own_begin, own_end);
      Impl<double>::check(md->core, false, 0, true);
    });
  }
  if (st != LMA_OK) {
    drop_model(md);
    return st;
  }
  *out = md;
  return LMA_OK;
}

lma_status lma_model_local_summary(const lma_model* md, double* G_out, double* logdet_out, int on_device) {
  if (!md || !G_out || !logdet_out) return fail(LMA_ERR_INVALID_ARG, "null pointer");
  const ModelCore& mc = md->core;
  return guarded([&] {
    const int64_t se = mc.s + 1;
    LMA_CK(cudaMemcpyAsync(G_out, mc.G, sizeof(double) * se * se,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, mc.st));
    LMA_CK(cudaStreamSynchronize(mc.st));
    *logdet_out = mc.logdetR;
  });
}

lma_status lma_model_set_global(lma_model* md, const double* G, double logdet_R, int64_t n_total, int on_device) {
  if (!md || !G) return fail(LMA_ERR_INVALID_ARG, "null pointer");
  if (n_total < md->core.n || !isfinite(logdet_R)) return fail(LMA_ERR_INVALID_ARG, "bad n_total or logdet_R");
  ModelCore& mc = md->core;
  return guarded([&] {
    const int64_t se = mc.s + 1;
    LMA_CK(cudaMemcpyAsync(mc.G, G, sizeof(double) * se * se,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, mc.st));
    mc.logdetR = logdet_R;
    if (mc.prec == LMA_MIXED) {
      Impl<float>::fit_global(mc, n_total);
      Impl<float>::check(mc, true, n_total, false);
    } else {
      Impl<double>::fit_global(mc, n_total);
      Impl<double>::check(mc, true, n_total, false);
    }
  });
}

// Argument checks shared by lma_predict and lma_predict_async.
static lma_status lma_predict_checks(const lma_model* md, int64_t u, const double* XU, const int64_t* tptr,
                                     const double* mean_out, const double* var_out) {
  if (!md) return fail(LMA_ERR_INVALID_ARG, "null model");
  if (u < 0) return fail(LMA_ERR_INVALID_ARG, "negative test count");
  if (u > 0 && (!XU || !tptr || !mean_out || !var_out)) return fail(LMA_ERR_INVALID_ARG, "null pointer");
  const ModelCore& mc = md->core;
  if (!mc.have_global) return fail(LMA_ERR_INVALID_ARG, "model has no global step yet (lma_model_set_global)");
  if (u > 0) {
    if (tptr[0] != 0 || tptr[mc.M] != u) return fail(LMA_ERR_INVALID_ARG, "test_block_ptr must start at 0, end at u");
    const int64_t w1 = mc.w0 + (int64_t)mc.wins.size();
    for (int64_t m = 0; m < mc.M; ++m) {
      if (tptr[m + 1] < tptr[m]) return fail(LMA_ERR_INVALID_ARG, "test_block_ptr decreases", m);
      if (tptr[m + 1] > tptr[m] && (std::max<int64_t>(0, m - mc.B) < mc.w0 || m >= w1))
        return fail(LMA_ERR_INVALID_ARG, "test block outside the windows of this model", m);
    }
  }
  return LMA_OK;
}

lma_status lma_predict(const lma_model* md, int64_t u, const double* XU, const int64_t* tptr, int noisy,
                       int io_on_device, double* mean_out, double* var_out) {
  lma_status cst = lma_predict_checks(md, u, XU, tptr, mean_out, var_out);
  if (cst != LMA_OK) return cst;
  const ModelCore& mc = md->core;
  return guarded([&] {
    if (mc.prec == LMA_MIXED)
      Impl<float>::predict(mc, u, XU, tptr, noisy, io_on_device, mean_out, var_out);
    else
      Impl<double>::predict(mc, u, XU, tptr, noisy, io_on_device, mean_out, var_out);
  });
}

static bool on_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

lma_status lma_predict_async(lma_model* md, int64_t u, const double* XU, const int64_t* tptr, int noisy,
                             double* mean_out, double* var_out) {
  if (!md) return fail(LMA_ERR_INVALID_ARG, "null model");
  if (u > 0 && (!on_device_ptr(XU) || !on_device_ptr(mean_out) || !on_device_ptr(var_out)))
    return fail(LMA_ERR_INVALID_ARG, "lma_predict_async needs XU, mean_out and var_out in device memory");
  ModelCore& mc = md->core;
  lma_status st = lma_predict_checks(md, u, XU, tptr, mean_out, var_out);
  if (st != LMA_OK || u == 0) return st;
  return guarded([&] {
    if (!mc.async_err) {
      mc.async_err = mc.keep.alloc<int>(1);
      LMA_CK(cudaMemsetAsync(mc.async_err, 0, sizeof(int), mc.st));
    }
    if (mc.prec == LMA_MIXED)
      Impl<float>::predict(mc, u, XU, tptr, noisy, 1, mean_out, var_out, nullptr, nullptr, nullptr, mc.async_err);
    else
      Impl<double>::predict(mc, u, XU, tptr, noisy, 1, mean_out, var_out, nullptr, nullptr, nullptr, mc.async_err);
  });
}

lma_status lma_model_wait(lma_model* md) {
  if (!md) return fail(LMA_ERR_INVALID_ARG, "null model");
  ModelCore& mc = md->core;
  int herr = 0;
  lma_status st = guarded([&] {
    if (mc.async_err) {
      LMA_CK(cudaMemcpyAsync(&herr, mc.async_err, sizeof(int), cudaMemcpyDeviceToHost, mc.st));
      LMA_CK(cudaMemsetAsync(mc.async_err, 0, sizeof(int), mc.st));
    }
    LMA_CK(cudaStreamSynchronize(mc.st));
  });
  if (st != LMA_OK) return st;
  if (herr) return fail(LMA_ERR_TIMEOUT, "tensor-core pipeline wait timed out in an enqueued prediction");
  return LMA_OK;
}

lma_status lma_fit_predict(const lma_problem* P, const lma_hyper* H, const lma_options* O, int64_t u,
                           const double* XU, const int64_t* tptr, int noisy, int io_on_device, double* mean_out,
                           double* var_out, lma_model** out) {
  if (out) *out = nullptr;
  lma_status cs = check_problem(P, H, O);
  if (cs != LMA_OK) return cs;
  if (u < 0) return fail(LMA_ERR_INVALID_ARG, "negative test count");
  if (u > 0 && (!XU || !tptr || !mean_out || !var_out)) return fail(LMA_ERR_INVALID_ARG, "null pointer");
  if (u > 0) {
    if (tptr[0] != 0 || tptr[P->m_blocks] != u)
      return fail(LMA_ERR_INVALID_ARG, "test_block_ptr must start at 0, end at u");
    for (int64_t m = 0; m < P->m_blocks; ++m)
      if (tptr[m + 1] < tptr[m]) return fail(LMA_ERR_INVALID_ARG, "test_block_ptr decreases", m);
  }
  lma_model* md = new (std::nothrow) lma_model();
  if (!md) return fail(LMA_ERR_OOM, "host allocation failed");
  md->core.prec = O->precision;
  md->core.st = (cudaStream_t)O->cuda_stream;
  md->core.keep.st = md->core.st;
  lma_status st = guarded([&] {
    if (O->precision == LMA_MIXED)
      Impl<float>::fit_predict(md->core, P, H, u, XU, tptr, noisy, io_on_device, mean_out, var_out);
    else
      Impl<double>::fit_predict(md->core, P, H, u, XU, tptr, noisy, io_on_device, mean_out, var_out);
  });
  if (retry_in_fp64(st, O->precision)) {  // the outputs are written again by the FP64 run
    drop_model(md);
    md = new_model(O, LMA_FP64);
    if (!md) return fail(LMA_ERR_OOM, "host allocation failed");
    st = guarded([&] {
      Impl<double>::fit_predict(md->core, P, H, u, XU, tptr, noisy, io_on_device, mean_out, var_out);
    });
  }
  if (st != LMA_OK || !out) {
    drop_model(md);
    return st;
  }
  *out = md;
  return LMA_OK;
}

lma_status lma_predict_cov(const lma_model* md, int64_t u, const double* XU, const int64_t* tptr, int noisy,
                           int io_on_device, double* mean_out, double* var_out, double* cov_out) {
  lma_status cst = lma_predict_checks(md, u, XU, tptr, mean_out, var_out);
  if (cst != LMA_OK) return cst;
  if (u > 0 && !cov_out) return fail(LMA_ERR_INVALID_ARG, "null pointer");
  const ModelCore& mc = md->core;
  return guarded([&] {
    if (mc.prec == LMA_MIXED)
      Impl<float>::predict(mc, u, XU, tptr, noisy, io_on_device, mean_out, var_out, nullptr, cov_out);
    else
      Impl<double>::predict(mc, u, XU, tptr, noisy, io_on_device, mean_out, var_out, nullptr, cov_out);
  });
}

lma_status lma_predict_cov_blocks(const lma_model* md, int64_t u, const double* XU, const int64_t* tptr, int noisy,
                                  int io_on_device, int64_t n_pairs, const int64_t* block_pairs, double* mean_out,
                                  double* var_out, double* cov_out) {
  lma_status cst = lma_predict_checks(md, u, XU, tptr, mean_out, var_out);
  if (cst != LMA_OK) return cst;
  if (n_pairs < 0) return fail(LMA_ERR_INVALID_ARG, "negative pair count");
  if (n_pairs > 0 && !block_pairs) return fail(LMA_ERR_INVALID_ARG, "null block_pairs");
  const ModelCore& mc = md->core;
  int64_t total = 0;
  for (int64_t i = 0; i < 2 * n_pairs; ++i)
    if (block_pairs[i] < 0 || block_pairs[i] >= mc.M) return fail(LMA_ERR_INVALID_ARG, "block index out of range", i);
  if (u > 0)
    for (int64_t i = 0; i < n_pairs; ++i) {
      const int64_t a = block_pairs[2 * i], b = block_pairs[2 * i + 1];
      total += (tptr[a + 1] - tptr[a]) * (tptr[b + 1] - tptr[b]);
    }
  if (total > 0 && !cov_out) return fail(LMA_ERR_INVALID_ARG, "null cov_out");
  return guarded([&] {
    if (mc.prec == LMA_MIXED)
      Impl<float>::predict(mc, u, XU, tptr, noisy, io_on_device, mean_out, var_out, nullptr, cov_out, nullptr, nullptr,
                           block_pairs, n_pairs);
    else
      Impl<double>::predict(mc, u, XU, tptr, noisy, io_on_device, mean_out, var_out, nullptr, cov_out, nullptr,
                            nullptr, block_pairs, n_pairs);
  });
}

lma_status lma_model_loglik(const lma_model* md, double* out) {
  if (!md || !out) return fail(LMA_ERR_INVALID_ARG, "null pointer");
  if (!md->core.have_global) return fail(LMA_ERR_INVALID_ARG, "model has no global step yet (lma_model_set_global)");
  *out = md->core.loglik;
  return LMA_OK;
}

lma_status lma_loglik(const lma_problem* P, const lma_hyper* H, const lma_options* O, double* out) {
  if (!out) return fail(LMA_ERR_INVALID_ARG, "null output pointer");
  lma_model* md = nullptr;
  lma_status st = lma_fit(P, H, O, &md);
  if (st != LMA_OK) return st;
  *out = md->core.loglik;
  lma_model_free(md);
  return LMA_OK;
}

lma_status lma_loglik_grad(const lma_problem* P, const lma_hyper* H, const lma_options* O, double* ll,
                           double* grad) {
  if (!ll || !grad) return fail(LMA_ERR_INVALID_ARG, "null output pointer");
  lma_status cs = check_problem(P, H, O);
  if (cs != LMA_OK) return cs;
  ModelCore mc;
  mc.prec = O->precision;
  mc.st = (cudaStream_t)O->cuda_stream;
  mc.keep.st = mc.st;
  lma_status st = guarded([&] {
    if (O->precision == LMA_MIXED)
      Impl<float>::loglik_grad(mc, P, H, ll, grad);
    else
      Impl<double>::loglik_grad(mc, P, H, ll, grad);
  });
  mc.keep.release();
  cudaStreamSynchronize(mc.st);
  if (retry_in_fp64(st, O->precision)) {
    ModelCore m64;
    m64.prec = LMA_FP64;
    m64.st = mc.st;
    m64.keep.st = mc.st;
    st = guarded([&] { Impl<double>::loglik_grad(m64, P, H, ll, grad); });
    m64.keep.release();
    cudaStreamSynchronize(m64.st);
  }
  return st;
}

lma_status lma_model_loglik_grad(lma_model* md, double* grad) {
  if (!md || !grad) return fail(LMA_ERR_INVALID_ARG, "null pointer");
  ModelCore& mc = md->core;
  if (!mc.have_global) return fail(LMA_ERR_INVALID_ARG, "the model's global step is not done (lma_model_set_global)");
  return guarded([&] {
    const int64_t k_lo = mc.own_b - mc.w0, k_hi = mc.own_e - mc.w0;
    if (mc.prec == LMA_MIXED)
      Impl<float>::grad_windows(mc, k_lo, k_hi, grad);
    else
      Impl<double>::grad_windows(mc, k_lo, k_hi, grad);
  });
}

lma_precision lma_model_precision(const lma_model* md) { return md ? md->core.prec : LMA_FP64; }

lma_status lma_model_summary(const lma_model* md, double* A_out, double* y_out, double* sc) {
  if (!md) return fail(LMA_ERR_INVALID_ARG, "null model");
  const ModelCore& mc = md->core;
  return guarded([&] {
    const int64_t se = mc.s + 1;
    std::vector<double> G((size_t)(se * se));
    LMA_CK(cudaMemcpyAsync(G.data(), mc.G, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, mc.st));
    LMA_CK(cudaStreamSynchronize(mc.st));
    if (A_out)
      for (int64_t i = 0; i < mc.s; ++i)
        for (int64_t j = 0; j < mc.s; ++j) A_out[i * mc.s + j] = G[(size_t)((1 + i) * se + 1 + j)];
    if (y_out)
      for (int64_t i = 0; i < mc.s; ++i) y_out[i] = G[(size_t)((1 + i) * se)];
    if (sc) {
      sc[0] = mc.quad;
      sc[1] = mc.logdetR;
      sc[2] = mc.logdetC;
      sc[3] = mc.loglik;
    }
  });
}

int64_t lma_window_rows(const lma_problem* P, int64_t m) {
  if (!P || !P->block_ptr || m < 0 || m >= P->m_blocks || P->markov_order < 0) return 0;
  int64_t last = m + P->markov_order < P->m_blocks - 1 ? m + P->markov_order : P->m_blocks - 1;
  return P->block_ptr[last + 1] - P->block_ptr[m];
}

lma_status lma_window_residual(const lma_problem* P, const lma_hyper* H, const lma_options* O, int64_t m,
                               double* out) {
  lma_status cs = check_problem(P, H, O);
  if (cs != LMA_OK) return cs;
  if (m < 0 || m >= P->m_blocks || !out) return fail(LMA_ERR_INVALID_ARG, "bad block index or null output");
  ModelCore mc;
  mc.prec = O->precision;
  mc.st = (cudaStream_t)O->cuda_stream;
  mc.keep.st = mc.st;
  lma_status st = guarded([&] {
    if (O->precision == LMA_MIXED)
      Impl<float>::window_residual(mc, P, H, m, out);
    else
      Impl<double>::window_residual(mc, P, H, m, out);
  });
  mc.keep.release();
  cudaStreamSynchronize(mc.st);
  return st;
}

void lma_model_free(lma_model* md) {
  if (!md) return;
  md->core.keep.release();
  cudaStreamSynchronize(md->core.st);
  delete md;
}

const char* lma_status_string(lma_status s) {
  switch (s) {
    case LMA_OK: return "ok";
    case LMA_ERR_INVALID_ARG: return "invalid argument";
    case LMA_ERR_NOT_PD: return "matrix not positive definite";
    case LMA_ERR_CUDA: return "CUDA error";
    case LMA_ERR_OOM: return "out of device memory";
    case LMA_ERR_TIMEOUT: return "device wait timed out";
    case LMA_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

lma_status lma_last_error_info(int64_t* failed_block, const char** message) {
  ErrState& e = err();
  if (failed_block) *failed_block = e.block;
  if (message) *message = e.msg.c_str();
  return e.status;
}

int64_t lma_kernel_launch_count(void) { return g_launches.load(); }

lma_status lma_tc_gemm_check(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                             int64_t ldb, float* C, int64_t ldc, int tile_n, void* cuda_stream) {
  if (M < 1 || N < 1 || K < 32 || K % 32 || !A || !B || !C || lda % 4 || ldb % 4 || lda < K || ldb < K || ldc < N ||
      (tile_n != 64 && tile_n != 128) || M > (1ll << 30) || N > (1ll << 30) || K > (1ll << 30) ||
      ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
    return fail(LMA_ERR_INVALID_ARG, "tc_gemm_check: bad sizes, strides or alignment");
  return guarded([&] { tc_gemm_check(M, N, K, A, lda, B, ldb, C, ldc, tile_n, (cudaStream_t)cuda_stream); });
}

lma_status lma_global_step_noalloc(int64_t s, int64_t n, const double* A, const double* y, double quad,
                                   double logdet_R, double* beta_out, double* scalars_out, void* cuda_stream) {
  if (s < 1 || n < 1 || !A || !y || !beta_out || !scalars_out || !isfinite(quad) || !isfinite(logdet_R))
    return fail(LMA_ERR_INVALID_ARG, "lma_global_step_noalloc: bad sizes or null pointer");
  return guarded([&] { global_step_noalloc(s, n, A, y, quad, logdet_R, beta_out, scalars_out,
                                           (cudaStream_t)cuda_stream); });
}

void lma_profile_start(const char* name_filter) {
  prof::g_on = true;
  prof::g_filter = name_filter ? name_filter : "";
  for (auto& r : prof::g_recs) {
    prof::g_pool.push_back(r.a);
    prof::g_pool.push_back(r.b);
  }
  prof::g_recs.clear();
}

int lma_profile_trace(char* names, int names_cap, double* t0_ms, double* t1_ms, int cap) {
  std::string all;
  const int k = (int)prof::g_recs.size();
  for (int i = 0; i < k; ++i) {
    const prof::Rec& r = prof::g_recs[i];
    cudaEventSynchronize(r.b);
    if (i < cap) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, prof::g_recs[0].a, r.a);
      cudaEventElapsedTime(&b, prof::g_recs[0].a, r.b);
      if (t0_ms) t0_ms[i] = a;
      if (t1_ms) t1_ms[i] = b;
    }
    all += r.name;
    all += "\n";
  }
  if (names && names_cap > 0) {
    size_t n = all.size() < (size_t)(names_cap - 1) ? all.size() : (size_t)(names_cap - 1);
    memcpy(names, all.data(), n);
    names[n] = 0;
  }
  return k;
}

int lma_profile_stop(char* names, int names_cap, double* total_ms, int64_t* launches, int cap) {
  prof::g_on = false;
  std::map<std::string, std::pair<double, int64_t>> agg;
  std::vector<std::string> order;
  for (auto& r : prof::g_recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto it = agg.find(r.name);
    if (it == agg.end()) {
      order.push_back(r.name);
      agg[r.name] = {ms, 1};
    } else {
      it->second.first += ms;
      it->second.second += 1;
    }
    prof::g_pool.push_back(r.a);
    prof::g_pool.push_back(r.b);
  }
  prof::g_recs.clear();
  std::string all;
  int k = 0;
  for (const std::string& nm : order) {
    if (k < cap) {
      if (total_ms) total_ms[k] = agg[nm].first;
      if (launches) launches[k] = agg[nm].second;
    }
    all += nm;
    all += "\n";
    ++k;
  }
  if (names && names_cap > 0) {
    size_t n = all.size() < (size_t)(names_cap - 1) ? all.size() : (size_t)(names_cap - 1);
    memcpy(names, all.data(), n);
    names[n] = 0;
  }
  return k;
}

}  // extern "C"

// ---- launch-shape autotuner ------------------------------------------------
#include "lma_tune.cuh"

extern "C" void lma_autotune(int enabled) { lma::tune::set_enabled(enabled != 0); }

extern "C" void lma_autotune_pin(const char* prefix, int choice) { lma::tune::pin(prefix, choice); }

extern "C" lma_status lma_workspace_release(void) {
  return guarded([] { lma::fit_workspace_release(); });
}

extern "C" int lma_autotune_report(char* buf, int cap) {
  const std::string r = lma::tune::report();
  if (buf && cap > 0) {
    const size_t n = std::min<size_t>(r.size(), (size_t)cap - 1);
    memcpy(buf, r.data(), n);
    buf[n] = '\0';
  }
  return (int)r.size();
}
