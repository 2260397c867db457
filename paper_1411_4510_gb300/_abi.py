"""ctypes declarations of the C ABI in include/lma.h (no arithmetic here)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblma_gb300.so")

LMA_OK, LMA_ERR_INVALID_ARG, LMA_ERR_NOT_PD, LMA_ERR_CUDA, LMA_ERR_OOM, LMA_ERR_TIMEOUT, LMA_ERR_INTERNAL = range(7)
LMA_FP64, LMA_MIXED = 0, 1

EXPORTED = (
    "lma_fit", "lma_predict", "lma_predict_async", "lma_model_wait", "lma_model_loglik", "lma_model_loglik_grad", "lma_loglik", "lma_loglik_grad", "lma_model_summary",
    "lma_window_residual", "lma_window_rows", "lma_model_free", "lma_status_string", "lma_last_error_info",
    "lma_kernel_launch_count", "lma_profile_start", "lma_profile_stop", "lma_profile_trace", "lma_tc_gemm_check",
    "lma_global_step_noalloc", "lma_fit_local", "lma_model_local_summary", "lma_model_set_global",
    "lma_fit_predict", "lma_predict_cov", "lma_predict_cov_blocks", "lma_model_precision", "lma_autotune", "lma_autotune_pin", "lma_autotune_report", "lma_workspace_release",
)


class lma_problem(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("d", C.c_int64), ("m_blocks", C.c_int64), ("s", C.c_int64),
        ("markov_order", C.c_int64), ("X", C.c_void_p), ("y", C.c_void_p), ("block_ptr", C.c_void_p),
        ("S", C.c_void_p), ("mean", C.c_double), ("inputs_on_device", C.c_int),
    ]


class lma_hyper(C.Structure):
    _fields_ = [("log_ell", C.c_void_p), ("log_sigma_s", C.c_double), ("log_sigma_n", C.c_double),
                ("jitter", C.c_double)]


class lma_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("reserved", C.c_int), ("cuda_stream", C.c_void_p)]


_lib = None


class LMAError(RuntimeError):
    def __init__(self, status: int, message: str, block: int):
        super().__init__(f"LMA status {status}: {message}" + (f" (block {block})" if status == LMA_ERR_NOT_PD else ""))
        self.status = status
        self.block = block


def load(path: str | None = None):
    """Load the shared library (building is done by paper_1411_4510_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"LMA CUDA library not built: {p} is missing (run __graft_entry__.build())")
    lib = C.CDLL(p)
    P, H, O = C.POINTER(lma_problem), C.POINTER(lma_hyper), C.POINTER(lma_options)
    vp = C.c_void_p
    lib.lma_fit.argtypes = [P, H, O, C.POINTER(vp)]
    lib.lma_fit.restype = C.c_int
    lib.lma_predict.argtypes = [vp, C.c_int64, vp, vp, C.c_int, C.c_int, vp, vp]
    lib.lma_predict.restype = C.c_int
    lib.lma_model_loglik.argtypes = [vp, C.POINTER(C.c_double)]
    lib.lma_model_loglik.restype = C.c_int
    lib.lma_model_loglik_grad.argtypes = [vp, vp]
    lib.lma_model_loglik_grad.restype = C.c_int
    lib.lma_predict_async.argtypes = [vp, C.c_int64, vp, vp, C.c_int, vp, vp]
    lib.lma_predict_async.restype = C.c_int
    lib.lma_model_wait.argtypes = [vp]
    lib.lma_model_wait.restype = C.c_int
    lib.lma_loglik.argtypes = [P, H, O, C.POINTER(C.c_double)]
    lib.lma_loglik.restype = C.c_int
    lib.lma_loglik_grad.argtypes = [P, H, O, C.POINTER(C.c_double), vp]
    lib.lma_loglik_grad.restype = C.c_int
    lib.lma_model_summary.argtypes = [vp, vp, vp, vp]
    lib.lma_model_summary.restype = C.c_int
    lib.lma_window_residual.argtypes = [P, H, O, C.c_int64, vp]
    lib.lma_window_residual.restype = C.c_int
    lib.lma_window_rows.argtypes = [P, C.c_int64]
    lib.lma_window_rows.restype = C.c_int64
    lib.lma_model_free.argtypes = [vp]
    lib.lma_model_free.restype = None
    lib.lma_status_string.argtypes = [C.c_int]
    lib.lma_status_string.restype = C.c_char_p
    lib.lma_last_error_info.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_char_p)]
    lib.lma_last_error_info.restype = C.c_int
    lib.lma_kernel_launch_count.argtypes = []
    lib.lma_kernel_launch_count.restype = C.c_int64
    lib.lma_tc_gemm_check.argtypes = [C.c_int64, C.c_int64, C.c_int64, vp, C.c_int64, vp, C.c_int64, vp,
                                      C.c_int64, C.c_int, vp]
    lib.lma_tc_gemm_check.restype = C.c_int
    lib.lma_global_step_noalloc.argtypes = [C.c_int64, C.c_int64, vp, vp, C.c_double, C.c_double, vp, vp, vp]
    lib.lma_global_step_noalloc.restype = C.c_int
    lib.lma_fit_local.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, C.c_int64, C.POINTER(vp)]
    lib.lma_fit_local.restype = C.c_int
    lib.lma_model_local_summary.argtypes = [vp, vp, C.POINTER(C.c_double), C.c_int]
    lib.lma_model_local_summary.restype = C.c_int
    lib.lma_model_set_global.argtypes = [vp, vp, C.c_double, C.c_int64, C.c_int]
    lib.lma_model_set_global.restype = C.c_int
    lib.lma_fit_predict.argtypes = [P, H, O, C.c_int64, vp, vp, C.c_int, C.c_int, vp, vp, C.POINTER(vp)]
    lib.lma_fit_predict.restype = C.c_int
    lib.lma_predict_cov.argtypes = [vp, C.c_int64, vp, vp, C.c_int, C.c_int, vp, vp, vp]
    lib.lma_predict_cov.restype = C.c_int
    lib.lma_predict_cov_blocks.argtypes = [vp, C.c_int64, vp, vp, C.c_int, C.c_int, C.c_int64, vp, vp, vp, vp]
    lib.lma_predict_cov_blocks.restype = C.c_int
    lib.lma_profile_start.argtypes = [C.c_char_p]
    lib.lma_profile_start.restype = None
    lib.lma_profile_stop.argtypes = [C.c_char_p, C.c_int, vp, vp, C.c_int]
    lib.lma_profile_stop.restype = C.c_int
    lib.lma_profile_trace.argtypes = [C.c_char_p, C.c_int, vp, vp, C.c_int]
    lib.lma_profile_trace.restype = C.c_int
    lib.lma_model_precision.argtypes = [vp]
    lib.lma_model_precision.restype = C.c_int
    lib.lma_autotune.argtypes = [C.c_int]
    lib.lma_autotune.restype = None
    lib.lma_autotune_pin.argtypes = [C.c_char_p, C.c_int]
    lib.lma_autotune_pin.restype = None
    lib.lma_workspace_release.argtypes = []
    lib.lma_workspace_release.restype = C.c_int
    lib.lma_autotune_report.argtypes = [C.c_char_p, C.c_int]
    lib.lma_autotune_report.restype = C.c_int
    _lib = lib
    return lib


def check(status: int):
    if status == LMA_OK:
        return
    lib = load()
    blk = C.c_int64(0)
    msg = C.c_char_p()
    lib.lma_last_error_info(C.byref(blk), C.byref(msg))
    text = (msg.value or b"").decode(errors="replace") or lib.lma_status_string(status).decode()
    raise LMAError(status, text, blk.value)
