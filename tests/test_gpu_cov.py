"""Predictive covariance of each test block (Eq. vapvar on U_n x U_n)
through lma_predict_cov against the oracle's local route (itself pinned to
the dense definition); its diagonal is the variance of the same call (to
rounding in the mixed form, whose variance takes the tensor-core path)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-9
TOL_MIXED = 2e-3


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1411_4510_gb300 import build
    build.build()
    import paper_1411_4510_gb300 as L
    torch.cuda.set_device(0)
    return L


@pytest.fixture(scope="module", params=[1, 2])
def case(request):
    from oracle import lma_oracle as O2
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=request.param)
    f = O2.fit(p)
    return p, O2.predict_cov(f, noisy=True)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_block_covariance(L, case, prec):
    p, ref = case
    model = L.lma_fit(precision=getattr(L, prec), **L.problem_args(p))
    mean, var, covs = L.lma_predict_cov(model, p.XU, p.test_block_ptr)
    tol = TOL_FP64 if prec == "FP64" else TOL_MIXED
    num = den = 0.0
    for n, (C, R) in enumerate(zip(covs, ref)):
        if R is None:
            assert C is None
            continue
        num += np.sum((C - R) ** 2)
        den += np.sum(R ** 2)
        # the variance comes from the compensated tensor-core path in the mixed form
        dtol = 1e-10 if prec == "FP64" else 1e-3
        assert np.allclose(np.diag(C), var[p.test_block_ptr[n]:p.test_block_ptr[n + 1]], rtol=dtol, atol=dtol * 1e-2)
    assert np.sqrt(num / den) <= tol
    m0, v0 = L.lma_predict(model, p.XU, p.test_block_ptr)
    assert np.array_equal(m0, mean)


def test_block_covariance_device_io(L, case):
    import torch
    p, ref = case
    model = L.lma_fit(precision=L.FP64, **L.problem_args(p))
    _, _, covs = L.lma_predict_cov(model, torch.as_tensor(p.XU, device="cuda:0"), p.test_block_ptr)
    for C, R in zip(covs, ref):
        if R is not None:
            assert np.allclose(C.cpu().numpy(), R, rtol=1e-8, atol=1e-10)
