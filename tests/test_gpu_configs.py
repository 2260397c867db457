"""GPU parity at configuration shapes beyond C1/C2: the C3 recipe (21-D
normal inputs, RFF draw, k-means blocks of uneven size, B = 2) at 24 blocks
and |S| = 256, with the oracle predicting a sample of test blocks (the first
two, a middle one and the last two, where blankets are truncated); and the C5
recipe (8-D Morton blocks) for the log-likelihood.  Tolerances as in
test_gpu_parity.py."""
import numpy as np
import pytest

from _parity import check, check_scalar

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9
MEAN_TOL_MIXED = 1e-4
MEAN_ELEM_MIXED = 3e-4
VAR_TOL_MIXED = 6e-4
VAR_ELEM_MIXED = 5e-2
LL_TOL_MIXED = 1.5e-4


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1411_4510_gb300 import build
    build.build()
    import paper_1411_4510_gb300 as L
    torch.cuda.set_device(0)
    return L


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def c3():
    from oracle import lma_oracle as O2
    from workloads import make_problem
    p = make_problem("C3", N=12288, M=24, s=256, U=512, B=2)
    sizes = p.block_sizes()
    assert sizes.min() < sizes.max()          # uneven windows
    f = O2.fit(p)
    blocks = [0, 1, 11, 22, 23]
    m, v = O2.predict(f, blocks=blocks)
    sel = np.concatenate([np.arange(p.test_block_ptr[b], p.test_block_ptr[b + 1]) for b in blocks])
    return p, f, m[sel], v[sel], sel


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_c3_shaped_uneven_blocks(L, c3, prec):
    import torch
    p, f, m_ref, v_ref, sel = c3
    args = L.problem_args(p)
    dev = torch.device("cuda:0")
    args.update(X=torch.as_tensor(p.X, device=dev), y=torch.as_tensor(p.y, device=dev),
                S=torch.as_tensor(p.S, device=dev))
    model = L.lma_fit(precision=getattr(L, prec), **args)
    assert L.lma_model_precision(model) == getattr(L, prec), "the mixed fit was redone in FP64"
    mean, var = L.lma_predict(model, torch.as_tensor(p.XU, device=dev), p.test_block_ptr)
    mean, var = mean.cpu().numpy()[sel], var.cpu().numpy()[sel]
    ll = L.lma_model_loglik(model)
    t = f"c3_reduced_{prec.lower()}"
    if prec == "FP64":
        check(t, "mean", mean, m_ref, TOL_FP64, TOL_FP64)
        check(t, "var", var, v_ref, TOL_FP64, TOL_FP64, positive=True)
        check_scalar(t, "loglik", ll, f.loglik, TOL_FP64)
    else:
        check(t, "mean", mean, m_ref, MEAN_TOL_MIXED, MEAN_ELEM_MIXED)
        check(t, "var", var, v_ref, VAR_TOL_MIXED, VAR_ELEM_MIXED, positive=True)
        check_scalar(t, "loglik", ll, f.loglik, LL_TOL_MIXED)


def test_c5_shaped_loglik(L):
    from oracle import lma_oracle as O2
    from workloads import make_problem
    p = make_problem("C5", N=8192, M=16, s=256, U=0, B=2)
    ref = O2.fit(p).loglik
    for prec, tol in (("FP64", TOL_FP64), ("MIXED", LL_TOL_MIXED)):
        ll = L.lma_loglik(precision=getattr(L, prec), **L.problem_args(p))
        check_scalar(f"c5_reduced_{prec.lower()}", "loglik", ll, ref, tol)
