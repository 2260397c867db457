"""Hyperparameter learning (maximum likelihood, Sec. 5) driven by the
summary-form oracle's log-likelihood and hand adjoint on the CPU: the
optimiser must climb to a stationary point of the LMA log-likelihood."""
import dataclasses

import numpy as np
import pytest

from oracle import lma_oracle as O2
from paper_1411_4510_gb300 import learn
from workloads import make_random_problem


def _args(p):
    return dict(X=p.X, y=p.y, block_ptr=p.block_ptr, S=p.S, B=p.B, log_ell=p.log_ell, log_sigma_s=p.log_sigma_s,
                log_sigma_n=p.log_sigma_n, jitter=p.jitter, mean=p.mean)


def _oracle_loglik_grad(p):
    d = p.X.shape[1]

    def f(_, th):
        q = dataclasses.replace(p, log_ell=np.asarray(th[:d]), log_sigma_s=float(th[d]), log_sigma_n=float(th[d + 1]))
        return O2.loglik_grad(q)
    return f


def test_learn_reaches_a_stationary_point():
    p = make_random_problem(7, (9, 8, 10, 9, 8), d=2, s=8, B=1, ell=0.35, sigma_n=0.1)
    f = _oracle_loglik_grad(p)
    d = p.X.shape[1]
    th0 = learn.pack(p.log_ell + 0.5, p.log_sigma_s - 0.4, p.log_sigma_n + 0.6, d)
    ll0, _ = f(None, th0)
    r = learn.learn_hyperparameters(_args(p), theta0=th0, loglik_grad=f, max_iter=200, gtol=1e-8)
    assert r.loglik > ll0 + 1.0
    assert np.max(np.abs(r.grad)) / p.X.shape[0] < 1e-5
    # a local maximum: no coordinate step of 1e-3 improves it
    for i in range(th0.size):
        for h in (-1e-3, 1e-3):
            t = r.theta.copy()
            t[i] += h
            assert f(None, t)[0] <= r.loglik + 1e-7


def test_learn_respects_bounds():
    p = make_random_problem(8, (8, 9, 7), d=2, s=6, B=1)
    f = _oracle_loglik_grad(p)
    d = p.X.shape[1]
    th0 = learn.pack(p.log_ell, p.log_sigma_s, p.log_sigma_n, d)
    lo, hi = th0 - 0.05, th0 + 0.05
    r = learn.learn_hyperparameters(_args(p), theta0=th0, loglik_grad=f, bounds=(lo, hi), max_iter=50)
    assert np.all(r.theta >= lo - 1e-12) and np.all(r.theta <= hi + 1e-12)
    assert r.loglik >= f(None, th0)[0] - 1e-9
