"""Python binding of the LMA C ABI with the same entry-point names.

Argument marshalling only: arrays are converted to contiguous float64 (numpy
on the host, torch tensors on the host or the current CUDA device) and their
pointers are handed to the library; every step of the computation runs in
the CUDA library.  Device tensors are passed as device pointers together with
torch's current stream.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _abi

try:
    import torch
except Exception:  # pragma: no cover - torch is expected but not required for host use
    torch = None

FP64 = _abi.LMA_FP64
MIXED = _abi.LMA_MIXED


def _is_cuda_tensor(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor) and a.is_cuda


def _f64(a, keep):
    """(pointer, on_device) of a contiguous float64 view of `a`; `keep` holds references."""
    if _is_cuda_tensor(a):
        t = a.detach().to(torch.float64).contiguous()
        keep.append(t)
        return t.data_ptr(), True
    if torch is not None and isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    keep.append(arr)
    return arr.ctypes.data, False


def _i64(a, keep):
    if torch is not None and isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    keep.append(arr)
    return arr.ctypes.data


def _stream(stream):
    if stream is not None:
        return stream
    if torch is not None and torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return None


def _structs(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter, mean, precision, stream, keep):
    n, d = int(X.shape[0]), int(X.shape[1])
    s = int(S.shape[0])
    M = int(len(block_ptr) - 1)
    xp, xdev = _f64(X, keep)
    yp, ydev = _f64(y, keep)
    sp, sdev = _f64(S, keep)
    if not (xdev == ydev == sdev):
        raise ValueError("X, y and S must all be on the host or all on the device")
    prob = _abi.lma_problem(n, d, M, s, int(B), xp, yp, _i64(block_ptr, keep), sp, float(mean), int(xdev))
    le = np.ascontiguousarray(np.broadcast_to(np.asarray(log_ell, dtype=np.float64), (d,)))
    keep.append(le)
    hyp = _abi.lma_hyper(le.ctypes.data, float(log_sigma_s), float(log_sigma_n), float(jitter))
    opt = _abi.lma_options(int(precision), 0, _stream(stream))
    return prob, hyp, opt


@dataclass
class Model:
    """A fitted model owned by the library (freed with lma_model_free)."""
    handle: int
    n_blocks: int
    s: int
    d: int = 0

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                _abi.load().lma_model_free(self.handle)
            except Exception:
                pass
            self.handle = None


def lma_fit(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter=1e-6, mean=0.0,
            precision=MIXED, stream=None) -> Model:
    lib = _abi.load()
    keep = []
    prob, hyp, opt = _structs(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter, mean,
                              precision, stream, keep)
    h = C.c_void_p()
    _abi.check(lib.lma_fit(C.byref(prob), C.byref(hyp), C.byref(opt), C.byref(h)))
    return Model(h.value, prob.m_blocks, prob.s, prob.d)


def lma_predict(model: Model, XU, test_block_ptr, noisy: bool = True, out=None):
    """Returns (mean, var): numpy arrays for host input, torch CUDA tensors for device input."""
    lib = _abi.load()
    keep = []
    u = int(XU.shape[0])
    xp, dev = _f64(XU, keep)
    tp = _i64(test_block_ptr, keep)
    if dev:
        mean = torch.empty(u, dtype=torch.float64, device=XU.device) if out is None else out[0]
        var = torch.empty(u, dtype=torch.float64, device=XU.device) if out is None else out[1]
        mp, vp = mean.data_ptr(), var.data_ptr()
    else:
        mean = np.empty(u) if out is None else out[0]
        var = np.empty(u) if out is None else out[1]
        mp, vp = mean.ctypes.data, var.ctypes.data
    _abi.check(lib.lma_predict(model.handle, u, xp, tp, int(bool(noisy)), int(dev), mp, vp))
    return mean, var


def lma_predict_async(model: Model, XU, test_block_ptr, noisy: bool = True):
    """lma_predict queued on the model's stream, without waiting (see
    lma_predict_async in lma.h).  XU must be a contiguous float64 CUDA tensor
    and stay alive until lma_model_wait(model) (or a synchronisation of the
    model's stream); returns the (mean, var) CUDA tensors that the queued work
    fills."""
    if not (isinstance(XU, torch.Tensor) and XU.is_cuda and XU.dtype == torch.float64 and XU.is_contiguous()):
        raise ValueError("lma_predict_async needs XU as a contiguous float64 CUDA tensor")
    keep = []
    u = int(XU.shape[0])
    mean = torch.empty(u, dtype=torch.float64, device=XU.device)
    var = torch.empty(u, dtype=torch.float64, device=XU.device)
    tp = _i64(test_block_ptr, keep)
    _abi.check(_abi.load().lma_predict_async(model.handle, u, XU.data_ptr(), tp, int(bool(noisy)), mean.data_ptr(),
                                             var.data_ptr()))
    return mean, var


def lma_model_wait(model: Model) -> None:
    """Wait for the model's stream; raises the status of the queued predictions."""
    _abi.check(_abi.load().lma_model_wait(model.handle))


def lma_predict_cov(model: Model, XU, test_block_ptr, noisy: bool = True):
    """(mean, var, covs): covs[n] is the |U_n| x |U_n| predictive covariance of
    test block n (None for empty blocks); numpy for host input, torch CUDA
    tensors for device input."""
    lib = _abi.load()
    keep = []
    u = int(XU.shape[0])
    xp, dev = _f64(XU, keep)
    tp = np.asarray(test_block_ptr, dtype=np.int64)
    tpp = _i64(tp, keep)
    sizes = np.diff(tp)
    total = int(np.sum(sizes * sizes))
    if dev:
        mean = torch.empty(u, dtype=torch.float64, device=XU.device)
        var = torch.empty(u, dtype=torch.float64, device=XU.device)
        cov = torch.empty(max(total, 1), dtype=torch.float64, device=XU.device)
        ptrs = mean.data_ptr(), var.data_ptr(), cov.data_ptr()
    else:
        mean, var, cov = np.empty(u), np.empty(u), np.empty(max(total, 1))
        ptrs = mean.ctypes.data, var.ctypes.data, cov.ctypes.data
    _abi.check(lib.lma_predict_cov(model.handle, u, xp, tpp, int(bool(noisy)), int(dev), *ptrs))
    covs, off = [], 0
    for k in sizes:
        k = int(k)
        covs.append(cov[off:off + k * k].reshape(k, k) if k else None)
        off += k * k
    return mean, var, covs


def lma_predict_cov_blocks(model: Model, XU, test_block_ptr, block_pairs, noisy: bool = True):
    """(mean, var, blocks): blocks[i] is the |U_n| x |U_n'| predictive
    covariance between test blocks n and n' for the i-th requested pair
    (n, n') of block_pairs (Eq. vapvar); numpy for host input, torch CUDA
    tensors for device input."""
    lib = _abi.load()
    keep = []
    u = int(XU.shape[0])
    xp, dev = _f64(XU, keep)
    tp = np.asarray(test_block_ptr, dtype=np.int64)
    tpp = _i64(tp, keep)
    bp = np.ascontiguousarray(np.asarray(block_pairs, dtype=np.int64).reshape(-1, 2))
    sizes = np.diff(tp)
    size = lambda n: int(sizes[n]) if 0 <= n < sizes.size else 0   # noqa: E731  (the library rejects bad indices)
    shapes = [(size(a), size(b)) for a, b in bp]
    total = sum(a * b for a, b in shapes)
    if dev:
        mean = torch.empty(u, dtype=torch.float64, device=XU.device)
        var = torch.empty(u, dtype=torch.float64, device=XU.device)
        cov = torch.empty(max(total, 1), dtype=torch.float64, device=XU.device)
        ptrs = mean.data_ptr(), var.data_ptr(), cov.data_ptr()
    else:
        mean, var, cov = np.empty(u), np.empty(u), np.empty(max(total, 1))
        ptrs = mean.ctypes.data, var.ctypes.data, cov.ctypes.data
    _abi.check(lib.lma_predict_cov_blocks(model.handle, u, xp, tpp, int(bool(noisy)), int(dev), len(bp),
                                          bp.ctypes.data, *ptrs))
    blocks, off = [], 0
    for a, b in shapes:
        blocks.append(cov[off:off + a * b].reshape(a, b))
        off += a * b
    return mean, var, blocks


def lma_predict_cov_full(model: Model, XU, test_block_ptr, noisy: bool = True):
    """(mean, var, cov): the whole |U| x |U| predictive covariance (every
    block pair through lma_predict_cov_blocks), numpy or torch like XU."""
    tp = np.asarray(test_block_ptr, dtype=np.int64)
    M = len(tp) - 1
    nz = [n for n in range(M) if tp[n + 1] > tp[n]]
    pairs = [(a, b) for a in nz for b in nz]
    mean, var, blocks = lma_predict_cov_blocks(model, XU, tp, pairs, noisy)
    u = int(XU.shape[0])
    if isinstance(mean, np.ndarray):
        cov = np.empty((u, u))
    else:
        cov = torch.empty((u, u), dtype=torch.float64, device=mean.device)
    for (a, b), C in zip(pairs, blocks):
        cov[tp[a]:tp[a + 1], tp[b]:tp[b + 1]] = C
    return mean, var, cov


def lma_fit_predict(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, XU, test_block_ptr, jitter=1e-6,
                    mean=0.0, precision=MIXED, noisy: bool = True, stream=None, keep_model: bool = False):
    """lma_fit + lma_predict in one call (the global step overlaps the
    prediction; in the mixed form the test right-hand sides ride the fit's
    sweep as extra window rows).  Returns (mean, var) or (mean, var, model)
    with keep_model."""
    lib = _abi.load()
    keep = []
    prob, hyp, opt = _structs(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter, mean,
                              precision, stream, keep)
    u = int(XU.shape[0])
    xp, dev = _f64(XU, keep)
    tp = _i64(test_block_ptr, keep)
    if dev:
        m = torch.empty(u, dtype=torch.float64, device=XU.device)
        v = torch.empty(u, dtype=torch.float64, device=XU.device)
        mp, vp = m.data_ptr(), v.data_ptr()
    else:
        m, v = np.empty(u), np.empty(u)
        mp, vp = m.ctypes.data, v.ctypes.data
    h = C.c_void_p()
    _abi.check(lib.lma_fit_predict(C.byref(prob), C.byref(hyp), C.byref(opt), u, xp, tp, int(bool(noisy)), int(dev),
                                   mp, vp, C.byref(h) if keep_model else None))
    if keep_model:
        return m, v, Model(h.value, prob.m_blocks, prob.s, prob.d)
    return m, v


def lma_model_loglik(model: Model) -> float:
    out = C.c_double()
    _abi.check(_abi.load().lma_model_loglik(model.handle, C.byref(out)))
    return out.value


def lma_model_loglik_grad(model: Model) -> np.ndarray:
    """Gradient of the model's log-likelihood over (log l_1..d, log sigma_s,
    log sigma_n) from the windows of its own blocks (all of them for lma_fit;
    a shard's part, which sums over the shards, for lma_fit_local after
    lma_model_set_global).  See lma_model_loglik_grad in lma.h."""
    g = np.empty(model.d + 2)
    _abi.check(_abi.load().lma_model_loglik_grad(model.handle, g.ctypes.data))
    return g


def lma_model_summary(model: Model):
    s = model.s
    A = np.empty((s, s))
    yv = np.empty(s)
    sc = np.empty(4)
    _abi.check(_abi.load().lma_model_summary(model.handle, A.ctypes.data, yv.ctypes.data, sc.ctypes.data))
    return dict(A=A, y=yv, quad=sc[0], logdet_R=sc[1], logdet_C=sc[2], loglik=sc[3])


def lma_fit_local(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, win_begin, own_begin, own_end,
                  jitter=1e-6, mean=0.0, precision=MIXED, stream=None) -> Model:
    """Shard part of a partitioned fit (windows of blocks [win_begin, own_end),
    local summaries of blocks [own_begin, own_end)); see lma_model_set_global."""
    lib = _abi.load()
    keep = []
    prob, hyp, opt = _structs(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter, mean,
                              precision, stream, keep)
    h = C.c_void_p()
    _abi.check(lib.lma_fit_local(C.byref(prob), C.byref(hyp), C.byref(opt), int(win_begin), int(own_begin),
                                 int(own_end), C.byref(h)))
    return Model(h.value, prob.m_blocks, prob.s, prob.d)


def lma_model_local_summary(model: Model, device=None):
    """(G, logdet): the shard's (s+1) x (s+1) Gram of local summaries and its
    log-determinant sum.  G is a CUDA tensor on `device` if given, else numpy."""
    lib = _abi.load()
    se = model.s + 1
    ld = C.c_double()
    if device is not None:
        G = torch.empty((se, se), dtype=torch.float64, device=device)
        _abi.check(lib.lma_model_local_summary(model.handle, G.data_ptr(), C.byref(ld), 1))
    else:
        G = np.empty((se, se))
        _abi.check(lib.lma_model_local_summary(model.handle, G.ctypes.data, C.byref(ld), 0))
    return G, ld.value


def lma_model_set_global(model: Model, G, logdet_R: float, n_total: int) -> None:
    """Global step of a partitioned fit from the summed Gram and log-det sum."""
    keep = []
    gp, dev = _f64(G, keep)
    _abi.check(_abi.load().lma_model_set_global(model.handle, gp, float(logdet_R), int(n_total), int(dev)))


def lma_loglik(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter=1e-6, mean=0.0,
               precision=MIXED, stream=None) -> float:
    lib = _abi.load()
    keep = []
    prob, hyp, opt = _structs(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter, mean,
                              precision, stream, keep)
    out = C.c_double()
    _abi.check(lib.lma_loglik(C.byref(prob), C.byref(hyp), C.byref(opt), C.byref(out)))
    return out.value


def lma_loglik_grad(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter=1e-6, mean=0.0,
                    precision=MIXED, stream=None):
    """(loglik, grad) with grad ordered (log l_1..d, log sigma_s, log sigma_n)."""
    lib = _abi.load()
    keep = []
    prob, hyp, opt = _structs(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter, mean,
                              precision, stream, keep)
    out = C.c_double()
    g = np.empty(prob.d + 2)
    _abi.check(lib.lma_loglik_grad(C.byref(prob), C.byref(hyp), C.byref(opt), C.byref(out), g.ctypes.data))
    return out.value, g


def lma_window_residual(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, m, jitter=1e-6, mean=0.0,
                        precision=MIXED, stream=None):
    lib = _abi.load()
    keep = []
    prob, hyp, opt = _structs(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, jitter, mean,
                              precision, stream, keep)
    nw = lib.lma_window_rows(C.byref(prob), int(m))
    out = np.empty((nw, nw))
    _abi.check(lib.lma_window_residual(C.byref(prob), C.byref(hyp), C.byref(opt), int(m), out.ctypes.data))
    return out


def lma_kernel_launch_count() -> int:
    return int(_abi.load().lma_kernel_launch_count())


def problem_args(p, B=None):
    """Positional/keyword arguments of lma_fit for a workloads.Problem."""
    return dict(X=p.X, y=p.y, block_ptr=p.block_ptr, S=p.S, B=p.B if B is None else B, log_ell=p.log_ell,
                log_sigma_s=p.log_sigma_s, log_sigma_n=p.log_sigma_n, jitter=p.jitter, mean=p.mean)


if torch is not None:
    class LMALogLik(torch.autograd.Function):
        """log N(y; mu, Sigma-bar_DD) as a function of (log l, log sigma_s, log sigma_n);
        forward and the hand-written adjoint both run in the CUDA library."""

        @staticmethod
        def forward(ctx, log_ell, log_sigma_s, log_sigma_n, data):
            ll, g = lma_loglik_grad(log_ell=log_ell.detach().cpu().numpy(), log_sigma_s=float(log_sigma_s),
                                    log_sigma_n=float(log_sigma_n), **data)
            gt = torch.as_tensor(g, dtype=torch.float64)
            ctx.save_for_backward(gt)
            ctx.d = int(log_ell.numel())
            return torch.tensor(ll, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            g = g * gout.detach().cpu().to(torch.float64)
            d = ctx.d
            return g[:d].reshape(-1), g[d], g[d + 1], None

    def lma_loglik_autograd(log_ell, log_sigma_s, log_sigma_n, data):
        """Differentiable log-likelihood; `data` holds the remaining lma_loglik_grad keywords."""
        return LMALogLik.apply(log_ell, log_sigma_s, log_sigma_n, data)


def lma_model_precision(model) -> int:
    """FP64 or MIXED: the form the model was fitted in (FP64 after the mixed
    form's FP64 retry of a window that lost positive definiteness in FP32)."""
    return int(_abi.load().lma_model_precision(model.handle))


def lma_autotune(enabled: bool) -> None:
    """Turn the launch-shape autotuner's timing on or off (see lma_autotune in lma.h)."""
    _abi.load().lma_autotune(int(bool(enabled)))


def lma_workspace_release() -> None:
    """Frees the device workspace the fits of this thread keep between calls
    (see lma_workspace_release in lma.h)."""
    _abi.check(_abi.load().lma_workspace_release())


def lma_autotune_pin(prefix, choice: int = 0) -> None:
    """Pin the launch shape of every tuner key starting with `prefix` to
    `choice`; prefix None removes every pin (see lma_autotune_pin in lma.h)."""
    _abi.load().lma_autotune_pin(None if prefix is None else prefix.encode(), int(choice))


def lma_autotune_report() -> list:
    """[(device, key, choice, {candidate: ms})] of the tuner's cached choices."""
    lib = _abi.load()
    n = lib.lma_autotune_report(None, 0)
    buf = C.create_string_buffer(n + 1)
    lib.lma_autotune_report(buf, n + 1)
    out = []
    for line in buf.value.decode().splitlines():
        parts = [x.strip() for x in line.split("|")]
        if len(parts) < 4:
            continue
        ms = {}
        for tok in parts[3].split():
            c, _, v = tok.partition(":")
            ms[int(c)] = float(v)
        out.append((parts[0], parts[1], int(parts[2]), ms))
    return out


def profile_start(name_filter: str = "") -> None:
    """Bracket matching kernel launches with CUDA events (see lma_profile_start)."""
    _abi.load().lma_profile_start(name_filter.encode())


def profile_trace(cap: int = 4096) -> list:
    """[(kernel name, start ms, end ms)] of every launch recorded since
    profile_start, relative to the first one (call before profile_stop)."""
    lib = _abi.load()
    names = C.create_string_buffer(64 * cap)
    t0 = np.zeros(cap)
    t1 = np.zeros(cap)
    k = lib.lma_profile_trace(names, 64 * cap, t0.ctypes.data, t1.ctypes.data, cap)
    keys = names.value.decode().split("\n")
    return [(keys[i], float(t0[i]), float(t1[i])) for i in range(min(k, cap, len(keys)))]


def profile_stop() -> dict:
    """{kernel name: (total milliseconds, launches)} since profile_start."""
    lib = _abi.load()
    cap = 64
    names = C.create_string_buffer(8192)
    ms = np.zeros(cap)
    cnt = np.zeros(cap, dtype=np.int64)
    k = lib.lma_profile_stop(names, 8192, ms.ctypes.data, cnt.ctypes.data, cap)
    keys = names.value.decode().split("\n")[:k]
    return {nm: (float(ms[i]), int(cnt[i])) for i, nm in enumerate(keys)}
