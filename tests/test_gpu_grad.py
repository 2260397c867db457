"""GPU parity of the log-likelihood gradient (hand adjoint) against the FP64
oracle's adjoint, central finite differences and the autograd wrapper.

Tolerance for the FP64 form: 1e-9 relative, norm-wise and element-wise (the
accuracy target; measured at most 2.4e-13 on these cases).  Mixed form:
the adjoint inherits the FP32 error of the residual precision R_W^-1 through
every term; it is held to about three times the largest error measured on
the GB300 at the default jitter (tests/_parity.py reports it).
"""
import numpy as np
import pytest

from _parity import check, check_scalar

pytestmark = pytest.mark.gpu

GRAD_TOL_FP64 = 1e-9
GRAD_TOL_MIXED = 5e-4
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


CASES = [
    (0, (70, 90, 65, 80, 75), 1, 3, 40),
    (2, (130, 5, 77, 140), 0, 4, 70),
    (3, (50, 61, 72, 83), 3, 2, 33),
    (4, (1, 129, 2, 66, 3, 100), 2, 5, 100),
]


def _p(case, jitter=None):
    from workloads import make_random_problem
    seed, sizes, B, d, s = case
    p = make_random_problem(seed, sizes, d=d, s=s, B=B, test_sizes=np.zeros(len(sizes), dtype=np.int64))
    if jitter is not None:
        p.jitter = jitter
    return p


@pytest.mark.parametrize("case", CASES)
def test_grad_fp64_matches_oracle(L, case):
    from oracle import lma_oracle as O2
    p = _p(case)
    ll_ref, g_ref = O2.loglik_grad(p)
    ll, g = L.lma_loglik_grad(precision=L.FP64, **L.problem_args(p))
    t = f"grad_tiny{case[0]}_fp64"
    check_scalar(t, "loglik", ll, ll_ref, 1e-9)
    check(t, "grad", g, g_ref, GRAD_TOL_FP64, GRAD_TOL_FP64)


@pytest.mark.parametrize("case", CASES)
def test_grad_mixed_matches_oracle(L, case):
    from oracle import lma_oracle as O2
    p = _p(case)
    ll_ref, g_ref = O2.loglik_grad(p)
    ll, g = L.lma_loglik_grad(precision=L.MIXED, **L.problem_args(p))
    t = f"grad_tiny{case[0]}_mixed"
    check_scalar(t, "loglik", ll, ll_ref, LL_TOL_MIXED)
    check(t, "grad", g, g_ref, GRAD_TOL_MIXED, GRAD_TOL_MIXED)


def test_grad_c5_shaped_central_fd(L):
    """C5 recipe (8-D uniform inputs, RFF draw, Morton blocks, B = 2) at 16
    blocks of 256 and |S| = 128: GPU FP64 adjoint vs the oracle and vs
    central differences (h = 1e-4 in log space) of the GPU FP64 likelihood."""
    from oracle import lma_oracle as O2
    from workloads import make_problem
    p = make_problem("C5", N=4096, M=16, s=128, U=0, B=2)
    ll_ref, g_ref = O2.loglik_grad(p)
    args = L.problem_args(p)
    ll, g = L.lma_loglik_grad(precision=L.FP64, **args)
    check("grad_c5_reduced_fp64", "grad", g, g_ref, GRAD_TOL_FP64, GRAD_TOL_FP64)
    th = np.concatenate([p.log_ell, [p.log_sigma_s, p.log_sigma_n]])
    h = 1e-4
    fd = np.empty_like(th)
    d = p.d
    for k in range(th.size):
        vals = []
        for sgn in (1, -1):
            t = th.copy()
            t[k] += sgn * h
            a = dict(args, log_ell=t[:d], log_sigma_s=t[d], log_sigma_n=t[d + 1])
            vals.append(L.lma_loglik(precision=L.FP64, **a))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    # truncation error of the central difference ~ h^2 |f'''|: relative 1e-6
    check("grad_c5_reduced_fp64", "grad vs central difference", g, fd, 1e-6, 1e-6)
    llm, gm = L.lma_loglik_grad(precision=L.MIXED, **args)
    check("grad_c5_reduced_mixed", "grad", gm, g_ref, GRAD_TOL_MIXED, GRAD_TOL_MIXED)
    check_scalar("grad_c5_reduced_mixed", "loglik", llm, ll_ref, LL_TOL_MIXED)


def test_autograd_wrapper(L):
    import torch
    p = _p(CASES[0])
    args = L.problem_args(p)
    ll_ref, g_ref = L.lma_loglik_grad(precision=L.FP64, **args)
    data = {k: v for k, v in args.items() if k not in ("log_ell", "log_sigma_s", "log_sigma_n")}
    data["precision"] = L.FP64
    le = torch.tensor(p.log_ell, dtype=torch.float64, requires_grad=True)
    ls = torch.tensor(p.log_sigma_s, dtype=torch.float64, requires_grad=True)
    ln = torch.tensor(p.log_sigma_n, dtype=torch.float64, requires_grad=True)
    from paper_1411_4510_gb300.api import lma_loglik_autograd
    out = lma_loglik_autograd(le, ls, ln, data)
    (2.0 * out).backward()
    g = np.concatenate([le.grad.numpy(), [ls.grad.item(), ln.grad.item()]])
    assert out.item() == pytest.approx(ll_ref, rel=1e-12)
    assert np.allclose(g, 2.0 * g_ref, rtol=1e-12, atol=0)
