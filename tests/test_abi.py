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
