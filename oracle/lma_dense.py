"""Dense-definition LMA oracle (O1) — TEST INFRASTRUCTURE ONLY (tiny N).

Builds the |V| x |V| matrices of Section 3 explicitly and evaluates the
definitions directly, with no use of the summary machinery:

  * covariance: SE-ARD of Section 5,
      sigma_xx' = sigma_s^2 exp(-1/2 sum_i (x_i - x'_i)^2 / l_i^2) + sigma_n^2 delta_xx'.
    Reading of the noise term: delta applies to an observation paired with
    itself (the D-D diagonal, and the U-U diagonal when the noisy output
    variance is asked for); Sigma_SS and the cross-covariances with S are
    noise-free.  Sigma_SS carries an absolute jitter on its diagonal.
  * Q_BB' = Sigma_BS Sigma_SS^-1 Sigma_SB' and R = Sigma - Q (Section 3).
  * R-bar over V = D u U blocked as V_m = D_m u U_m by the recursion of
    Eq. (ares); Sigma-bar = Q + R-bar (Eq. acov).
  * predictive mean and covariance by Eqs. (vapmu) and (vapvar) with dense
    solves; log-likelihood log N(y_D; mu, Sigma-bar_DD).

Pins (tests/test_oracle_dense.py): B = M-1 reproduces the textbook full GP
(Section 2), B = 0 the PIC prior Q + blockdiag(R) (Section 3), the inverse
of R-bar_DD is B-block-banded (Proposition 1), tr(R_DD R-bar_DD^-1) = |D|
(proof of Theorem 1), and the KL-optimality of Theorem 1.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


def se_ard(X1: np.ndarray, X2: np.ndarray, log_ell, log_sigma_s: float) -> np.ndarray:
    """Noise-free SE-ARD covariance sigma_s^2 exp(-1/2 sum_i ((x_i - x'_i)/l_i)^2)."""
    ell = np.exp(np.asarray(log_ell, dtype=np.float64))
    A = X1 / ell
    Bm = X2 / ell
    D = A[:, None, :] - Bm[None, :, :]
    return math.exp(2.0 * log_sigma_s) * np.exp(-0.5 * np.sum(D * D, axis=-1))


def _blocks(ptr):
    return [np.arange(ptr[m], ptr[m + 1]) for m in range(len(ptr) - 1)]


def _prior(prob, noisy: bool):
    """Sigma over V = [D; U] (rows of D first, then U), Q and R."""
    N, U = prob.X.shape[0], prob.XU.shape[0]
    P = np.vstack([prob.X, prob.XU])
    K = se_ard(P, P, prob.log_ell, prob.log_sigma_s)
    sn2 = math.exp(2.0 * prob.log_sigma_n)
    Sigma = K.copy()
    Sigma[np.arange(N), np.arange(N)] += sn2
    if noisy and U > 0:
        Sigma[N + np.arange(U), N + np.arange(U)] += sn2
    Kss = se_ard(prob.S, prob.S, prob.log_ell, prob.log_sigma_s) + prob.jitter * np.eye(prob.S.shape[0])
    Kps = se_ard(P, prob.S, prob.log_ell, prob.log_sigma_s)
    Q = Kps @ np.linalg.solve(Kss, Kps.T)
    Q = 0.5 * (Q + Q.T)
    return Sigma, Q, Sigma - Q


def rbar(R: np.ndarray, Dm, Vm, B: int) -> np.ndarray:
    """R-bar_VV by the recursion of Eq. (ares) on the blocks V_m (index sets into R).

    |m-n| <= B : R_{V_m V_n}
    n-m > B > 0: R_{V_m D^B_m} R_{D^B_m D^B_m}^-1 Rbar_{D^B_m V_n}
    m-n > B > 0: Rbar_{V_m D^B_n} R_{D^B_n D^B_n}^-1 R_{D^B_n V_n}
    |m-n| > B = 0: 0
    with D^B_m the union of D_{m+1} .. D_{min(m+B, M)} (the next B blocks).
    Pairs are filled in order of increasing |m-n| so every recursive
    reference is already available.
    """
    M = len(Vm)
    Rb = np.zeros_like(R)

    def blanket(m):
        ks = range(m + 1, min(m + B, M - 1) + 1)
        return np.concatenate([Dm[k] for k in ks]) if len(ks) else np.zeros(0, dtype=np.int64)

    for dist in range(M):
        for m in range(M):
            for n in (m - dist, m + dist) if dist else (m,):
                if n < 0 or n >= M:
                    continue
                vm, vn = Vm[m], Vm[n]
                if abs(m - n) <= B:
                    Rb[np.ix_(vm, vn)] = R[np.ix_(vm, vn)]
                elif B == 0:
                    Rb[np.ix_(vm, vn)] = 0.0
                elif n - m > B:
                    Db = blanket(m)
                    Rb[np.ix_(vm, vn)] = R[np.ix_(vm, Db)] @ np.linalg.solve(R[np.ix_(Db, Db)], Rb[np.ix_(Db, vn)])
                else:
                    Db = blanket(n)
                    Rb[np.ix_(vm, vn)] = Rb[np.ix_(vm, Db)] @ np.linalg.solve(R[np.ix_(Db, Db)], R[np.ix_(Db, vn)])
    return Rb


def lma_dense(prob, B: int | None = None, noisy: bool = True) -> dict:
    """Dense LMA: returns Sigma, Q, R, Rbar, Sigmabar (V ordered [D; U]),
    the predictive mean / variance / covariance (vapmu / vapvar) and the
    log-likelihood log N(y_D; mu, Sigmabar_DD)."""
    B = prob.B if B is None else int(B)
    N, U = prob.X.shape[0], prob.XU.shape[0]
    Sigma, Q, R = _prior(prob, noisy)
    Dm = _blocks(prob.block_ptr)
    Um = [N + u for u in _blocks(prob.test_block_ptr)]
    Vm = [np.concatenate([Dm[m], Um[m]]) for m in range(len(Dm))]
    Rb = rbar(R, Dm, Vm, B)
    Sb = Q + Rb
    d_idx = np.arange(N)
    u_idx = N + np.arange(U)
    r = prob.y - prob.mean
    Sdd = Sb[np.ix_(d_idx, d_idx)]
    Sud = Sb[np.ix_(u_idx, d_idx)]
    cf = sla.cho_factor(Sdd, lower=True)
    mean = prob.mean + Sud @ sla.cho_solve(cf, r)
    cov = Sb[np.ix_(u_idx, u_idx)] - Sud @ sla.cho_solve(cf, Sud.T)
    Lc = np.linalg.cholesky(Sdd)
    w = sla.solve_triangular(Lc, r, lower=True)
    loglik = -0.5 * w @ w - np.sum(np.log(np.diag(Lc))) - 0.5 * N * math.log(2.0 * math.pi)
    return dict(Sigma=Sigma, Q=Q, R=R, Rbar=Rb, Sigmabar=Sb, mean=mean, cov=cov,
                var=np.diag(cov).copy(), loglik=loglik, d_idx=d_idx, u_idx=u_idx)


def full_gp(prob, noisy: bool = True) -> dict:
    """Textbook full-rank GP posterior and log marginal likelihood (Section 2)."""
    N = prob.X.shape[0]
    sn2 = math.exp(2.0 * prob.log_sigma_n)
    Kdd = se_ard(prob.X, prob.X, prob.log_ell, prob.log_sigma_s) + sn2 * np.eye(N)
    Kud = se_ard(prob.XU, prob.X, prob.log_ell, prob.log_sigma_s)
    Kuu = se_ard(prob.XU, prob.XU, prob.log_ell, prob.log_sigma_s)
    if noisy:
        Kuu = Kuu + sn2 * np.eye(prob.XU.shape[0])
    r = prob.y - prob.mean
    cf = sla.cho_factor(Kdd, lower=True)
    mean = prob.mean + Kud @ sla.cho_solve(cf, r)
    cov = Kuu - Kud @ sla.cho_solve(cf, Kud.T)
    return dict(mean=mean, var=np.diag(cov).copy(), cov=cov, K=Kdd)


def pic_prior(prob, noisy: bool = True) -> np.ndarray:
    """PIC prior over V: Q + blockdiag_m(R_{V_m V_m}) (Section 3, B = 0)."""
    N = prob.X.shape[0]
    Sigma, Q, R = _prior(prob, noisy)
    Dm = _blocks(prob.block_ptr)
    Um = [N + u for u in _blocks(prob.test_block_ptr)]
    mask = np.zeros_like(R, dtype=bool)
    for m in range(len(Dm)):
        v = np.concatenate([Dm[m], Um[m]])
        mask[np.ix_(v, v)] = True
    return Q + np.where(mask, R, 0.0)


def gaussian_posterior(Sb: np.ndarray, prob) -> dict:
    """mean / covariance of U given y_D under a joint prior Sb over [D; U]."""
    N, U = prob.X.shape[0], prob.XU.shape[0]
    d_idx, u_idx = np.arange(N), N + np.arange(U)
    Sdd = Sb[np.ix_(d_idx, d_idx)]
    Sud = Sb[np.ix_(u_idx, d_idx)]
    cf = sla.cho_factor(Sdd, lower=True)
    r = prob.y - prob.mean
    mean = prob.mean + Sud @ sla.cho_solve(cf, r)
    cov = Sb[np.ix_(u_idx, u_idx)] - Sud @ sla.cho_solve(cf, Sud.T)
    return dict(mean=mean, var=np.diag(cov).copy(), cov=cov)
