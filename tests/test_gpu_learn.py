"""Hyperparameter learning on the GPU (L-BFGS on lma_loglik_grad) on a
C2-shaped synthetic problem: started away from the generating values, it
climbs above the starting log-likelihood, ends at least as high as the
generating point, and recovers the generating noise level and length-scale;
the mixed and FP64 forms agree.  On a smaller problem it also reaches the
optimum that the same optimiser finds on the FP64 oracle's log-likelihood
and adjoint from the same start (tests/golden/learn.json)."""
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


@pytest.fixture(scope="module")
def runs(L):
    from paper_1411_4510_gb300 import learn
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=0, B=1)
    args = L.problem_args(p)
    d = p.X.shape[1]
    gen = learn.pack(p.log_ell, p.log_sigma_s, p.log_sigma_n, d)
    th0 = gen + np.concatenate([np.full(d, 0.4), [-0.3, 0.5]])
    out = {}
    for prec in ("FP64", "MIXED"):
        pr = getattr(L, prec)
        ll_gen = L.lma_loglik(precision=pr, **args)
        a0 = dict(args, log_ell=th0[:d], log_sigma_s=th0[d], log_sigma_n=th0[d + 1])
        ll0 = L.lma_loglik(precision=pr, **a0)
        r = learn.learn_hyperparameters(args, theta0=th0, precision=pr, max_iter=60)
        out[prec] = (r, ll0, ll_gen)
    return p, gen, out


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_learning_climbs_and_recovers(runs, prec):
    p, gen, out = runs
    r, ll0, ll_gen = out[prec]
    d = p.X.shape[1]
    assert r.loglik > ll0 + 50.0
    assert r.loglik >= ll_gen - 1e-3 * abs(ll_gen)
    assert abs(r.log_sigma_n - gen[d + 1]) < 0.15          # noise level within 16%
    assert abs(np.mean(r.log_ell) - np.mean(gen[:d])) < 0.35


def test_mixed_and_fp64_agree(runs):
    _, _, out = runs
    a, b = out["FP64"][0], out["MIXED"][0]
    assert np.max(np.abs(a.theta - b.theta)) < 0.05
    assert abs(a.loglik - b.loglik) < 1e-3 * abs(a.loglik)


@pytest.mark.parametrize("prec,tol_theta,tol_ll", [("FP64", 1e-6, 1e-9), ("MIXED", 5e-4, 1.5e-4)])
def test_learning_reaches_oracle_optimum(L, prec, tol_theta, tol_ll):
    import json
    import os
    from paper_1411_4510_gb300 import learn
    from workloads import make_problem
    from _parity import report
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "learn.json")))
    p = make_problem("C2", N=1200, M=8, s=40, U=0, B=1)
    assert g["fingerprints"]["N"] == p.N and g["fingerprints"]["s"] == p.s
    args = L.problem_args(p)
    r = learn.learn_hyperparameters(args, theta0=np.asarray(g["theta0"]), precision=getattr(L, prec), max_iter=200,
                                    gtol=1e-7)
    dth = float(np.max(np.abs(r.theta - np.asarray(g["theta"]))))
    dll = abs(r.loglik - g["loglik"]) / abs(g["loglik"])
    report(f"learn_{prec.lower()}", "theta", "max_abs", dth, tol_theta)
    report(f"learn_{prec.lower()}", "loglik", "scalar", dll, tol_ll)
    assert dth <= tol_theta, (r.theta, g["theta"])
    assert dll <= tol_ll
