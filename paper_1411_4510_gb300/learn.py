"""Hyperparameter learning for LMA by maximising its log-likelihood.

The paper learns the SE hyperparameters by maximum likelihood (Sec. 5); this
module maximises log N(y_D; mu, Sigma-bar_DD) of the LMA model itself over
theta = (log l_1..log l_d, log sigma_s, log sigma_n) with L-BFGS, using the
library's log-likelihood and hand-written adjoint (lma_loglik_grad, both on
the GPU).  The partition, the support set, the jitter and the Markov order
stay fixed.  The objective is scaled by 1/N so the optimiser's tolerances do
not depend on the problem size.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import api


@dataclass
class LearnResult:
    theta: np.ndarray                  # (log l_1..d, log sigma_s, log sigma_n)
    loglik: float                      # log-likelihood at theta
    grad: np.ndarray                   # its gradient at theta
    iterations: int
    evaluations: int
    converged: bool
    message: str
    history: list = field(default_factory=list)   # loglik after each evaluation

    @property
    def log_ell(self):
        return self.theta[:-2]

    @property
    def log_sigma_s(self):
        return float(self.theta[-2])

    @property
    def log_sigma_n(self):
        return float(self.theta[-1])


def pack(log_ell, log_sigma_s, log_sigma_n, d):
    return np.concatenate([np.broadcast_to(np.asarray(log_ell, dtype=np.float64), (d,)),
                           [float(log_sigma_s), float(log_sigma_n)]])


def learn_hyperparameters(args: dict, theta0=None, precision=api.MIXED, max_iter: int = 50, gtol: float = 1e-5,
                          bounds=None, loglik_grad=None) -> LearnResult:
    """Maximise the LMA log-likelihood over theta with L-BFGS-B.

    args: problem arguments as from api.problem_args (X, y, block_ptr, S, B,
    log_ell, log_sigma_s, log_sigma_n, jitter, mean); the hyperparameters in
    it are the starting point unless theta0 is given.  bounds: optional
    (lower, upper) arrays for theta.  loglik_grad(args, theta) -> (loglik,
    grad) defaults to the CUDA library's lma_loglik_grad."""
    from scipy.optimize import minimize

    X = np.asarray(args["X"])
    n, d = X.shape
    if theta0 is None:
        theta0 = pack(args["log_ell"], args["log_sigma_s"], args["log_sigma_n"], d)
    theta0 = np.asarray(theta0, dtype=np.float64)
    if loglik_grad is None:
        base = {k: v for k, v in args.items() if k not in ("log_ell", "log_sigma_s", "log_sigma_n")}

        def loglik_grad(_, th):
            return api.lma_loglik_grad(log_ell=th[:d], log_sigma_s=th[d], log_sigma_n=th[d + 1],
                                       precision=precision, **base)

    history = []

    def objective(th):
        ll, g = loglik_grad(args, th)
        history.append(float(ll))
        return -ll / n, -np.asarray(g, dtype=np.float64) / n

    bnds = None
    if bounds is not None:
        lo, hi = (np.broadcast_to(np.asarray(b, dtype=np.float64), theta0.shape) for b in bounds)
        bnds = list(zip(lo, hi))
    res = minimize(objective, theta0, jac=True, method="L-BFGS-B", bounds=bnds,
                   options=dict(maxiter=int(max_iter), gtol=float(gtol)))
    ll, g = loglik_grad(args, res.x)
    return LearnResult(theta=np.asarray(res.x), loglik=float(ll), grad=np.asarray(g), iterations=int(res.nit),
                       evaluations=int(res.nfev), converged=bool(res.success), message=str(res.message),
                       history=history)
