"""lma_fit_predict (global step on a second stream, overlapping the
prediction) returns what lma_fit followed by lma_predict returns.  In the
mixed form it appends the test right-hand sides to the window buffers, where
the fit's sweep solves them, instead of running the separate prediction
sweep: the same quantities through other FP32 kernels, so there the two agree
to FP32 accuracy rather than bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1411_4510_gb300 import build
    build.build()
    import paper_1411_4510_gb300 as L
    torch.cuda.set_device(0)
    return L


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("B", [1, 2])
def test_fit_predict_equals_fit_then_predict(L, prec, B):
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=B)
    args = L.problem_args(p)
    pr = getattr(L, prec)
    m = L.lma_fit(precision=pr, **args)
    mean0, var0 = L.lma_predict(m, p.XU, p.test_block_ptr)
    mean1, var1, m1 = L.lma_fit_predict(XU=p.XU, test_block_ptr=p.test_block_ptr, precision=pr, keep_model=True,
                                        **args)
    if prec == "FP64":
        assert np.allclose(mean1, mean0, rtol=1e-12, atol=1e-14)
        assert np.allclose(var1, var0, rtol=1e-12, atol=1e-14)
    else:
        assert np.linalg.norm(mean1 - mean0) <= 2e-5 * np.linalg.norm(mean0)
        assert np.linalg.norm(var1 - var0) <= 1e-4 * np.linalg.norm(var0)
    # the fit itself is the same either way
    assert L.lma_model_loglik(m1) == pytest.approx(L.lma_model_loglik(m), rel=1e-13)
    # the returned model predicts like the separately fitted one
    mean2, _ = L.lma_predict(m1, p.XU, p.test_block_ptr)
    assert np.allclose(mean2, mean0, rtol=1e-12, atol=1e-14)


def test_fit_predict_device_io(L):
    import torch
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=1)
    args = L.problem_args(p)
    dev = torch.device("cuda:0")
    dargs = dict(args, X=torch.as_tensor(p.X, device=dev), y=torch.as_tensor(p.y, device=dev),
                 S=torch.as_tensor(p.S, device=dev))
    mean, var = L.lma_fit_predict(XU=torch.as_tensor(p.XU, device=dev), test_block_ptr=p.test_block_ptr, **dargs)
    mean_h, var_h = L.lma_fit_predict(XU=p.XU, test_block_ptr=p.test_block_ptr, **args)
    # device and host buffers take the same path
    assert np.array_equal(mean.cpu().numpy(), mean_h)
    assert np.array_equal(var.cpu().numpy(), var_h)
    m = L.lma_fit(**args)
    mean0, var0 = L.lma_predict(m, p.XU, p.test_block_ptr)
    assert np.linalg.norm(mean.cpu().numpy() - mean0) <= 2e-5 * np.linalg.norm(mean0)
    assert np.linalg.norm(var.cpu().numpy() - var0) <= 1e-4 * np.linalg.norm(var0)
