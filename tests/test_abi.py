"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/lma.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(lma_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1411_4510_gb300 import build
    build.build()
    from paper_1411_4510_gb300 import _abi
    return _abi.load()


def test_header_declares_the_paths_entry_points():
    names = _declared()
    for n in ("lma_fit", "lma_predict", "lma_loglik", "lma_loglik_grad", "lma_model_free"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_declares_every_exported_symbol(lib):
    from paper_1411_4510_gb300 import _abi
    assert sorted(_abi.EXPORTED) == _declared()


def test_status_strings(lib):
    assert lib.lma_status_string(0) == b"ok"
    assert b"positive definite" in lib.lma_status_string(2)


def test_invalid_arguments_rejected_on_host(lib):
    """Argument checks run before any device work, so they work without a GPU."""
    import numpy as np
    import paper_1411_4510_gb300 as L
    from workloads import make_random_problem
    p = make_random_problem(0, (5, 6, 7), d=2, s=4, B=1)
    args = L.problem_args(p)
    for bad in (dict(B=3), dict(B=-1), dict(block_ptr=np.array([0, 5, 5, 18])),
                dict(block_ptr=np.array([0, 5, 11, 17])), dict(log_ell=[np.nan, 0.0]), dict(jitter=-1.0)):
        kw = dict(args)
        kw.update(bad)
        with pytest.raises(L.LMAError) as ei:
            L.lma_fit(**kw)
        assert ei.value.status == 1, bad


def test_window_rows_follow_the_markov_blanket(lib):
    """lma_window_rows (host arithmetic only): |D_m u D^B_m| with the blanket
    D^B_m = D_{m+1} .. D_{min(m+B, M-1)} truncated at the last block (Sec. 3);
    0 for an invalid block index."""
    import ctypes as C
    import numpy as np
    from paper_1411_4510_gb300 import _abi
    rng = np.random.default_rng(5)
    for trial in range(20):
        M = int(rng.integers(1, 9))
        sizes = rng.integers(1, 20, size=M)
        ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        B = int(rng.integers(0, M))
        prob = _abi.lma_problem()
        prob.n, prob.d, prob.s, prob.m_blocks, prob.markov_order = int(ptr[-1]), 1, 1, M, B
        prob.block_ptr = ptr.ctypes.data
        for m in range(M):
            last = min(m + B, M - 1)
            assert lib.lma_window_rows(C.byref(prob), m) == int(ptr[last + 1] - ptr[m])
        assert lib.lma_window_rows(C.byref(prob), M) == 0
        assert lib.lma_window_rows(C.byref(prob), -1) == 0


def test_prediction_calls_reject_a_missing_model_on_host(lib):
    """The prediction entry points check their arguments before any device
    work: a null model is LMA_ERR_INVALID_ARG (1), also without a GPU."""
    import numpy as np
    tp = np.array([0, 0], dtype=np.int64)
    pairs = np.array([0, 0], dtype=np.int64)
    assert lib.lma_predict(None, 0, None, tp.ctypes.data, 1, 0, None, None) == 1
    assert lib.lma_predict_cov(None, 0, None, tp.ctypes.data, 1, 0, None, None, None) == 1
    assert lib.lma_predict_cov_blocks(None, 0, None, tp.ctypes.data, 1, 0, 1, pairs.ctypes.data, None, None, None) == 1
    assert lib.lma_predict_async(None, 0, None, tp.ctypes.data, 1, None, None) == 1
    assert lib.lma_model_wait(None) == 1
