"""GB300-native LMA (low-rank-cum-Markov approximation) of GP regression.

The compute path is the CUDA library liblma_gb300.so (sources in csrc/,
C ABI in include/lma.h); this package is its thin Python binding.  Importing
the package does not load the library; the first call does, and fails loudly
if it has not been built.
"""
from .api import (  # noqa: F401
    FP64, MIXED, Model, lma_fit, lma_predict, lma_predict_async, lma_model_wait, lma_loglik, lma_loglik_grad, lma_model_loglik, lma_model_loglik_grad,
    lma_model_summary, lma_window_residual, lma_kernel_launch_count, problem_args, profile_start, profile_stop, profile_trace,
    lma_fit_local, lma_model_local_summary, lma_model_set_global, lma_fit_predict, lma_predict_cov, lma_predict_cov_blocks, lma_predict_cov_full, lma_model_precision,
    lma_autotune, lma_autotune_pin, lma_autotune_report, lma_workspace_release,
)
from ._abi import LMAError  # noqa: F401
