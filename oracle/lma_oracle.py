"""Summary-form LMA oracle (O2), FP64 — TEST INFRASTRUCTURE ONLY.

Follows the paper's steps in its own notation; numpy/scipy Cholesky,
triangular solves and matrix products serve as library steps.  No blocking,
fusion or reordering beyond what the definitions state.  Memory is
O(window^2 + |S|^2) so it runs at every configuration size (slowly).

fit()            Definition 1 (local summary of block m: R', y-dot_m,
                 R-dot_m, Sigma-dot^m_S) and Definition 2 (global summary
                 y-ddot_S, Sigma-ddot_SS), then alpha = Sigma-ddot_SS^-1 y-ddot_S.
loglik           log N(y_D; mu, Sigma-bar_DD) in summary form:
                 y^T Sigma-bar^-1 y uses Eq. (pitck) and log|Sigma-bar_DD| the
                 determinant lemma on the same identity; log|R-bar_DD| is the
                 sum of log|R-dot_m^-1| (Lemma 1: R-bar^-1 = U^T U with
                 U_mm^T U_mm = R-dot_m).
predict_cov()    The same local route for the full covariance of each test
                 block (Eq. vapvar on U_n x U_n).
predict_cov_blocks()  Eq. (vapvar) between any two test blocks U_n x U_n':
                 the local route on one side, R-bar_{D u'} by the recursion
                 of Eq. (ares) on the other.
predict_thm2()   Theorem 2 given Sigma-bar_DU (paper's route; tiny N only).
predict()        Local route: for u in U_n the row R-bar_{uD} R-bar_DD^-1 is
                 supported on the blocks J = n-B..n+B and equals
                 R_{u D_J} (R-bar_JJ)^-1, with (R-bar_JJ)^-1 assembled by
                 Lemma 1 on the sub-chain J (blankets truncated at the end of
                 J).  Then, with e = y - mu - Sigma_DS alpha and
                 z_u = R_{u D_J} (R-bar_JJ)^-1:
                   mean_u = mu + Sigma_uS alpha + z_u e_J
                   var_u  = sigma_uu - Sigma_uS Sigma_SS^-1 Sigma_Su
                            - z_u R_{D_J u} + g_u^T Sigma-ddot_SS^-1 g_u,
                   g_u    = Sigma_{S D_J} z_u^T - Sigma_Su.
                 This is an algebraic rearrangement of Eqs. (vapmu)/(vapvar)
                 (derived with Eq. (pitck)); tests pin it to the dense
                 definition and to Theorem 2.
loglik_grad()    Hand adjoint of the summary-form log-likelihood with respect
                 to (log l_1..d, log sigma_s, log sigma_n).  Not in the paper;
                 pinned by central finite differences of loglik and, at
                 B = M-1, by the closed-form full-GP gradient.

Readings of the paper used here:
  * noise sigma_n^2 on the D-D diagonal (and U-U when noisy) only;
  * Sigma_SS = K_SS + jitter I, the same matrix in Q and in Sigma-ddot_SS;
  * constant prior mean mu;
  * D^B_m = blocks m+1..min(m+B, M) (0-based: m+1..min(m+B, M-1)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .lma_dense import se_ard

LOG2PI = math.log(2.0 * math.pi)


def _rows(ptr, m):
    return np.arange(ptr[m], ptr[m + 1])


def _logdet_chol(c):
    return 2.0 * float(np.sum(np.log(np.diag(c))))


@dataclass
class LMAFit:
    prob: object
    B: int
    Sigma_SS: np.ndarray        # K_SS + jitter I
    L_SS: np.ndarray            # chol(Sigma_SS)
    ydd_S: np.ndarray           # global summary y-ddot_S
    Sdd_SS: np.ndarray          # global summary Sigma-ddot_SS
    alpha: np.ndarray           # Sigma-ddot_SS^-1 y-ddot_S
    quad: float                 # sum_m y-dot_m^T R-dot_m y-dot_m
    logdet_R: float             # sum_m log|R-dot_m^-1| = log|R-bar_DD|
    loglik: float
    blocks: list = field(default_factory=list)   # optional Definition-1 terms

    @property
    def sn2(self):
        return math.exp(2.0 * self.prob.log_sigma_n)


class _Cov:
    """Covariance pieces of one problem (no caching of N x N objects)."""

    def __init__(self, prob):
        self.p = prob
        self.sn2 = math.exp(2.0 * prob.log_sigma_n)
        self.ss2 = math.exp(2.0 * prob.log_sigma_s)
        self.Sigma_SS = se_ard(prob.S, prob.S, prob.log_ell, prob.log_sigma_s) + prob.jitter * np.eye(prob.S.shape[0])
        self.L_SS = np.linalg.cholesky(self.Sigma_SS)

    def K(self, A, Bx):
        return se_ard(A, Bx, self.p.log_ell, self.p.log_sigma_s)

    def KS(self, A):
        return self.K(A, self.p.S)

    def W(self, A):
        """L_SS^-1 Sigma_{S A} (so that Q_AB = W(A)^T W(B))."""
        return sla.solve_triangular(self.L_SS, self.KS(A).T, lower=True)

    def R_train(self, ia, ib):
        """Residual R over training rows ia x ib: Sigma - Q with noise where a row meets itself."""
        Xa, Xb = self.p.X[ia], self.p.X[ib]
        out = self.K(Xa, Xb) - self.W(Xa).T @ self.W(Xb)
        same = ia[:, None] == ib[None, :]
        return out + self.sn2 * same


def _local_terms(cv: _Cov, r, m: int, B: int):
    """Definition 1 for block m (whitened support coordinates): the rows I of
    D_m and Bk of D^B_m, R' = R_{D_m D^B_m} R_{D^B_m D^B_m}^-1, y-dot_m,
    R-dot_m^-1, Sigma-dot^m_S L^-T and the Cholesky factor of R-dot_m^-1."""
    prob = cv.p
    ptr = prob.block_ptr
    M = len(ptr) - 1
    I = _rows(ptr, m)
    last = min(m + B, M - 1)
    Bk = np.arange(ptr[m + 1], ptr[last + 1]) if last > m else np.zeros(0, dtype=np.int64)
    R_II = cv.R_train(I, I)
    W_I = cv.W(prob.X[I]).T                                             # Sigma_{D_m S} L^-T
    if Bk.size:
        R_IB = cv.R_train(I, Bk)
        R_BB = cv.R_train(Bk, Bk)
        Rp = sla.cho_solve(sla.cho_factor(R_BB, lower=True), R_IB.T).T      # R' = R_IB R_BB^-1
        ydot = r[I] - Rp @ r[Bk]
        Rdot_inv = R_II - Rp @ R_IB.T
        Sdot = W_I - Rp @ cv.W(prob.X[Bk]).T
    else:
        Rp = np.zeros((I.size, 0))
        ydot = r[I].copy()
        Rdot_inv = R_II
        Sdot = W_I
    cf = sla.cho_factor(Rdot_inv, lower=True)
    return I, Bk, Rp, ydot, Rdot_inv, Sdot, cf


def local_summaries(prob, blocks, B: int | None = None):
    """Sums of the local summaries (Definition 1) over the given blocks, in the
    whitened support coordinates: (A, y-ddot, quad, log|R-bar|) with
    A = sum Sigma-dot^T R-dot Sigma-dot, y-ddot = sum Sigma-dot^T R-dot y-dot,
    quad = sum y-dot^T R-dot y-dot and the sum of log|R-dot_m^-1|.  Over all
    blocks these are the global sums of Definition 2; over a machine's own
    blocks they are what that machine contributes (Remark 1)."""
    B = prob.B if B is None else int(B)
    cv = _Cov(prob)
    s = prob.S.shape[0]
    r = prob.y - prob.mean
    ydd = np.zeros(s)
    A = np.zeros((s, s))
    quad = 0.0
    logdet_R = 0.0
    for m in blocks:
        _, _, _, ydot, _, Sdot, cf = _local_terms(cv, r, m, B)
        t = sla.cho_solve(cf, np.column_stack([ydot, Sdot]))                 # R-dot [y-dot, Sigma-dot]
        ydd += Sdot.T @ t[:, 0]
        A += Sdot.T @ t[:, 1:]
        quad += float(ydot @ t[:, 0])
        logdet_R += _logdet_chol(np.tril(cf[0]))
    return A, ydd, quad, logdet_R


def fit(prob, B: int | None = None, keep_blocks: bool = False) -> LMAFit:
    """Definition 1 per block, Definition 2 sums, alpha, summary-form loglik.

    The support-set columns are taken in the whitened basis
    Sigma_DS L_SS^-T (L_SS = chol(Sigma_SS)): every quantity of Section 3 is
    invariant under an invertible change of basis of the support coordinates
    (Q_BB' = Sigma_BS Sigma_SS^-1 Sigma_SB' does not change), and in this basis
    Sigma_SS becomes I, so the global summary I + L^-1 (Sigma-ddot_SS -
    Sigma_SS) L^-T no longer inherits the jitter-level conditioning of
    Sigma_SS.  The paper-basis summaries are recovered as
    y-ddot_S = L y-ddot and Sigma-ddot_SS = L (I + A) L^T."""
    B = prob.B if B is None else int(B)
    cv = _Cov(prob)
    ptr = prob.block_ptr
    M = len(ptr) - 1
    s = prob.S.shape[0]
    r = prob.y - prob.mean
    ydd = np.zeros(s)          # whitened y-ddot
    A = np.zeros((s, s))       # whitened sum of Sigma-dot^T R-dot Sigma-dot
    quad = 0.0
    logdet_R = 0.0
    blocks = []
    for m in range(M):
        I, Bk, Rp, ydot, Rdot_inv, Sdot, cf = _local_terms(cv, r, m, B)
        t = sla.cho_solve(cf, np.column_stack([ydot, Sdot]))                 # R-dot [y-dot, Sigma-dot]
        ydd += Sdot.T @ t[:, 0]
        A += Sdot.T @ t[:, 1:]
        quad += float(ydot @ t[:, 0])
        logdet_R += _logdet_chol(np.tril(cf[0]))
        if keep_blocks:
            blocks.append(dict(I=I, Bk=Bk, Rp=Rp, ydot=ydot, Rdot_inv=Rdot_inv,
                               Sdot=Sdot @ cv.L_SS.T))                        # paper basis
    A = 0.5 * (A + A.T)
    C = np.eye(s) + A
    Lc = np.linalg.cholesky(C)
    w = sla.solve_triangular(Lc, ydd, lower=True)
    beta = sla.solve_triangular(Lc, w, lower=True, trans="T")              # C^-1 y-ddot
    L = cv.L_SS
    alpha = sla.solve_triangular(L, beta, lower=True, trans="T")           # Sigma-ddot_SS^-1 y-ddot_S
    N = prob.X.shape[0]
    loglik = (-0.5 * (quad - w @ w)
              - 0.5 * (logdet_R + _logdet_chol(Lc))
              - 0.5 * N * LOG2PI)
    f = LMAFit(prob=prob, B=B, Sigma_SS=cv.Sigma_SS, L_SS=L, ydd_S=L @ ydd,
               Sdd_SS=L @ C @ L.T, alpha=alpha, quad=quad, logdet_R=logdet_R,
               loglik=float(loglik), blocks=blocks)
    f.A_white, f.ydd_white, f.Lc, f.beta = A, ydd, Lc, beta
    return f


def _subchain_precision(cv: _Cov, ptr, Jb, B: int):
    """(R-bar_JJ)^-1 for the consecutive blocks Jb by Lemma 1 applied to the
    sub-chain: block row m is [U_mm, U^B_m] = U_mm [I, -R'] with the blanket
    truncated at the last block of Jb; returns the dense |D_J| x |D_J| sum of
    (block row)^T (block row) = [I; -R'^T] R-dot_m [I, -R']."""
    rows = np.concatenate([_rows(ptr, m) for m in Jb])
    pos0 = {m: int(ptr[m] - ptr[Jb[0]]) for m in Jb}
    nJ = rows.size
    P = np.zeros((nJ, nJ))
    lastJ = Jb[-1]
    for m in Jb:
        I = _rows(ptr, m)
        last = min(m + B, lastJ)
        Bk = np.arange(ptr[m + 1], ptr[last + 1]) if last > m else np.zeros(0, dtype=np.int64)
        R_II = cv.R_train(I, I)
        if Bk.size:
            R_IB = cv.R_train(I, Bk)
            R_BB = cv.R_train(Bk, Bk)
            Rp = sla.cho_solve(sla.cho_factor(R_BB, lower=True), R_IB.T).T
            Rdot_inv = R_II - Rp @ R_IB.T
        else:
            Rp = np.zeros((I.size, 0))
            Rdot_inv = R_II
        T = np.hstack([np.eye(I.size), -Rp])
        pos = np.arange(pos0[m], pos0[m] + I.size + Bk.size)
        P[np.ix_(pos, pos)] += T.T @ sla.cho_solve(sla.cho_factor(Rdot_inv, lower=True), T)
    return rows, P


def predict(f: LMAFit, XU=None, test_block_ptr=None, noisy: bool = True,
            blocks=None) -> tuple[np.ndarray, np.ndarray]:
    """Local-route predictive mean and variance (module docstring)."""
    p = f.prob
    XU = p.XU if XU is None else XU
    tptr = p.test_block_ptr if test_block_ptr is None else test_block_ptr
    cv = _Cov(p)
    ptr = p.block_ptr
    M = len(ptr) - 1
    B = f.B
    U = XU.shape[0]
    mean = np.full(U, np.nan)
    var = np.full(U, np.nan)
    it = range(M) if blocks is None else blocks
    for n in it:
        u = np.arange(tptr[n], tptr[n + 1])
        if u.size == 0:
            continue
        Jb = list(range(max(0, n - B), min(M - 1, n + B) + 1))
        rows, P = _subchain_precision(cv, ptr, Jb, B)
        Xu = XU[u]
        XJ = p.X[rows]
        Wu = cv.W(Xu)
        WJ = cv.W(XJ)
        Ru = cv.K(XJ, Xu) - WJ.T @ Wu                       # R_{D_J u} (u not in D: no noise)
        Z = P @ Ru                                          # columns z_u^T
        # whitened support basis: Sigma_uS alpha = W_u^T beta, and with
        # h = L_SS^-1 g:  g^T Sigma-ddot_SS^-1 g = h^T (I + A)^-1 h
        eJ = p.y[rows] - p.mean - WJ.T @ f.beta
        mean[u] = p.mean + Wu.T @ f.beta + Z.T @ eJ
        h = WJ @ Z - Wu                                     # L_SS^-1 (Sigma_{S D_J} z^T - Sigma_Su)
        hc = sla.solve_triangular(f.Lc, h, lower=True)
        prior = cv.ss2 + (cv.sn2 if noisy else 0.0)
        var[u] = (prior - np.sum(Wu * Wu, axis=0) - np.sum(Ru * Z, axis=0)
                  + np.sum(hc * hc, axis=0))
    return mean, var


def predict_cov(f: LMAFit, XU=None, test_block_ptr=None, noisy: bool = True, blocks=None) -> list:
    """Predictive covariance of each test block U_n (Eq. vapvar restricted to
    U_n x U_n, where Sigma-bar_UU = Sigma_UU since the pairs are in-band), by
    the local route of predict():
        Cov_n = Sigma_{U_n U_n} - W_u^T W_u - R_{D_J u}^T (R-bar_JJ)^-1 R_{D_J u}
                + hc^T hc.
    Returns one |U_n| x |U_n| matrix per test block (None for empty blocks
    and blocks not asked for)."""
    p = f.prob
    XU = p.XU if XU is None else XU
    tptr = p.test_block_ptr if test_block_ptr is None else test_block_ptr
    cv = _Cov(p)
    ptr = p.block_ptr
    M = len(ptr) - 1
    B = f.B
    out = [None] * M
    it = range(M) if blocks is None else blocks
    for n in it:
        u = np.arange(tptr[n], tptr[n + 1])
        if u.size == 0:
            continue
        Jb = list(range(max(0, n - B), min(M - 1, n + B) + 1))
        rows, P = _subchain_precision(cv, ptr, Jb, B)
        Xu = XU[u]
        XJ = p.X[rows]
        Wu = cv.W(Xu)
        WJ = cv.W(XJ)
        Ru = cv.K(XJ, Xu) - WJ.T @ Wu
        Z = P @ Ru
        h = WJ @ Z - Wu
        hc = sla.solve_triangular(f.Lc, h, lower=True)
        Kuu = cv.K(Xu, Xu) + (cv.sn2 * np.eye(u.size) if noisy else 0.0)
        out[n] = Kuu - Wu.T @ Wu - Ru.T @ Z + hc.T @ hc
    return out


def _blanket_solver(cv: _Cov, ptr, B: int, k: int, cache: dict):
    """Rows I of D_k, rows Bk of its blanket D^B_k, R_{D_k D^B_k} and the
    Cholesky factor of R_{D^B_k D^B_k} (computed once per block)."""
    if k not in cache:
        M = len(ptr) - 1
        I = _rows(ptr, k)
        last = min(k + B, M - 1)
        Bk = np.arange(ptr[k + 1], ptr[last + 1])
        cache[k] = (I, Bk, cv.R_train(I, Bk), sla.cho_factor(cv.R_train(Bk, Bk), lower=True))
    return cache[k]


def _rbar_to_test(cv: _Cov, ptr, B: int, k: int, Xq, nq: int, memo: dict, bl: dict):
    """R-bar_{D_k q} for the test points Xq of test block nq, by Eq. (ares):
    R_{D_k q} when |k - nq| <= B (in the band); for k < nq - B the recursion
    R_{D_k D^B_k} R_{D^B_k D^B_k}^-1 R-bar_{D^B_k q} over the blanket of
    block k; 0 off the band when B = 0.  Only k <= nq + B is asked for."""
    if k in memo:
        return memo[k]
    p = cv.p
    M = len(ptr) - 1
    I = _rows(ptr, k)
    if abs(k - nq) <= B:
        Wk = cv.W(p.X[I])
        out = cv.K(p.X[I], Xq) - Wk.T @ cv.W(Xq)           # test points are not in D: no noise
    elif B == 0:
        out = np.zeros((I.size, Xq.shape[0]))
    else:
        assert k < nq - B
        last = min(k + B, M - 1)
        _, _, R_IB, cf = _blanket_solver(cv, ptr, B, k, bl)
        rho_B = np.vstack([_rbar_to_test(cv, ptr, B, j, Xq, nq, memo, bl) for j in range(k + 1, last + 1)])
        out = R_IB @ sla.cho_solve(cf, rho_B)
    memo[k] = out
    return out


def predict_cov_blocks(f: LMAFit, pairs, XU=None, test_block_ptr=None, noisy: bool = True) -> list:
    """Predictive covariance between test blocks U_n and U_n' (Eq. vapvar on
    U_n x U_n') for each requested (n, n'); returns one |U_n| x |U_n'| matrix
    per pair.  In the whitened support coordinates (W = L_SS^-1 Sigma_S.),
    Eq. (vapvar) splits as
        Cov(u, u') = R-bar_{uu'} - R-bar_{uD} R-bar_DD^-1 R-bar_{Du'} + hc_u^T hc_u'
    (Woodbury on Sigma-bar_DD = Q_DD + R-bar_DD; hc = L_C^-1 h with h the
    vector of predict()).  For n <= n' the middle term is z_u rho_J with
    z_u = R_{u D_J} (R-bar_JJ)^-1 on the sub-chain J = n-B..n+B (the local
    route of predict()) and rho_J = R-bar_{D_J u'} by Eq. (ares)
    (_rbar_to_test); R-bar_{uu'} is R_{uu'} in the band (|n - n'| <= B; plus
    sigma_n^2 where a noisy point meets itself) and otherwise
    R_{u D^B_n} R_{D^B_n D^B_n}^-1 R-bar_{D^B_n u'} (Eq. ares; 0 when B = 0).
    n > n' is the transpose of (n', n)."""
    p = f.prob
    XU = p.XU if XU is None else XU
    tptr = p.test_block_ptr if test_block_ptr is None else test_block_ptr
    cv = _Cov(p)
    ptr = p.block_ptr
    M = len(ptr) - 1
    B = f.B

    sides: dict = {}
    memos: dict = {}
    bl: dict = {}

    def side(n):
        if n in sides:
            return sides[n]
        u = np.arange(tptr[n], tptr[n + 1])
        Jb = list(range(max(0, n - B), min(M - 1, n + B) + 1))
        rows, P = _subchain_precision(cv, ptr, Jb, B)
        Xu = XU[u]
        WJ = cv.W(p.X[rows])
        Wu = cv.W(Xu)
        Ru = cv.K(p.X[rows], Xu) - WJ.T @ Wu
        Z = P @ Ru
        hc = sla.solve_triangular(f.Lc, WJ @ Z - Wu, lower=True)
        sides[n] = (u, Jb, Z, hc)
        return sides[n]

    def block(n, n2):                                        # n <= n2
        u, Jb, Z, hc = side(n)
        u2, _, _, hc2 = side(n2)
        if u.size == 0 or u2.size == 0:
            return np.zeros((u.size, u2.size))
        X1, X2 = XU[u], XU[u2]
        memo = memos.setdefault(n2, {})                      # R-bar_{D_k u'} for the points of block n2
        if n2 - n <= B:
            Rb = cv.K(X1, X2) - cv.W(X1).T @ cv.W(X2)
            if noisy and n == n2:
                Rb = Rb + cv.sn2 * np.eye(u.size)
        elif B == 0:
            Rb = np.zeros((u.size, u2.size))
        else:
            last = min(n + B, M - 1)
            _, Bk, _, cf = _blanket_solver(cv, ptr, B, n, bl)
            rho_B = np.vstack([_rbar_to_test(cv, ptr, B, j, X2, n2, memo, bl) for j in range(n + 1, last + 1)])
            R_uB = cv.K(X1, p.X[Bk]) - cv.W(X1).T @ cv.W(p.X[Bk])
            Rb = R_uB @ sla.cho_solve(cf, rho_B)
        rho_J = np.vstack([_rbar_to_test(cv, ptr, B, k, X2, n2, memo, bl) for k in Jb])
        return Rb - Z.T @ rho_J + hc.T @ hc2

    out = []
    for n, n2 in pairs:
        n, n2 = int(n), int(n2)
        out.append(block(n, n2) if n <= n2 else block(n2, n).T)
    return out


def predict_thm2(f: LMAFit, Sigmabar_DU: np.ndarray, Sigma_UU_diag: np.ndarray):
    """Theorem 2 from the local summaries (Definition 1, needs keep_blocks=True)
    and the global summary (Definition 2), given Sigma-bar_DU:
      Sigma-dot^m_U = Sigma-bar_{D_m U} - R' Sigma-bar_{D^B_m U}
      y-ddot_U = sum (Sigma-dot^m_U)^T R-dot_m y-dot_m,
      Sigma-ddot_US = sum (Sigma-dot^m_U)^T R-dot_m Sigma-dot^m_S,
      diag Sigma-ddot_UU = diag sum (Sigma-dot^m_U)^T R-dot_m Sigma-dot^m_U,
      mean = mu + y-ddot_U - Sigma-ddot_US Sigma-ddot_SS^-1 y-ddot_S,
      var  = diag Sigma_UU - diag Sigma-ddot_UU + diag(Sigma-ddot_US Sigma-ddot_SS^-1 Sigma-ddot_US^T)."""
    assert f.blocks, "fit(..., keep_blocks=True) required"
    U = Sigmabar_DU.shape[1]
    s = f.Sdd_SS.shape[0]
    ydd_U = np.zeros(U)
    Sdd_US = np.zeros((U, s))
    Sdd_UU = np.zeros(U)
    for blk in f.blocks:
        SdotU = Sigmabar_DU[blk["I"]] - blk["Rp"] @ Sigmabar_DU[blk["Bk"]]
        cf = sla.cho_factor(blk["Rdot_inv"], lower=True)
        t = sla.cho_solve(cf, np.column_stack([blk["ydot"], blk["Sdot"], SdotU]))
        ydd_U += SdotU.T @ t[:, 0]
        Sdd_US += SdotU.T @ t[:, 1:1 + s]
        Sdd_UU += np.sum(SdotU * t[:, 1 + s:], axis=0)
    cfS = sla.cho_factor(f.Sdd_SS, lower=True)
    mean = f.prob.mean + ydd_U - Sdd_US @ sla.cho_solve(cfS, f.ydd_S)
    var = Sigma_UU_diag - Sdd_UU + np.sum(Sdd_US.T * sla.cho_solve(cfS, Sdd_US.T), axis=0)
    return mean, var


def loglik(prob, B: int | None = None) -> float:
    return fit(prob, B).loglik


def _tri_adj_chol(L, Lbar):
    """Adjoint of Sigma -> L = chol(Sigma): Sigma-bar = L^-T Phi(L^T L-bar) L^-1,
    Phi = lower triangle with halved diagonal (derived from
    L^-1 dSigma L^-T = L^-1 dL + (L^-1 dL)^T)."""
    X = L.T @ np.tril(Lbar)
    Phi = np.tril(X) - 0.5 * np.diag(np.diag(X))
    Y = sla.solve_triangular(L, Phi.T, lower=True, trans="T").T    # Phi L^-1 ... (right solve)
    Y = sla.solve_triangular(L, Y, lower=True, trans="T")           # L^-T (Phi L^-1)
    return 0.5 * (Y + Y.T)


def loglik_grad(prob, B: int | None = None, windows=None) -> tuple[float, np.ndarray]:
    """Hand adjoint of the summary-form log-likelihood.

    In the whitened support coordinates V = L_SS^-1 Sigma_SD (Vt = V^T,
    N x s) the forward pass is, per block m with window W_m = D_m u D^B_m
    and blanket B_m = D^B_m (Lemma 1 gives R-bar^-1 = sum_m pad(R_W^-1) -
    pad(R_B^-1)):
        C = I + sum_m [Vt_W^T R_W^-1 Vt_W - Vt_B^T R_B^-1 Vt_B],
        y = sum_m [Vt_W^T R_W^-1 r_W - Vt_B^T R_B^-1 r_B], quad likewise,
        log|R-bar| = sum_m log|R_W| - log|R_B|,
        loglik = -1/2 (quad - y^T C^-1 y) - 1/2 (log|R-bar| + log|C|) - N/2 log 2 pi.
    Reverse sweep with beta = C^-1 y, e = r - Vt beta, C = Lc Lc^T,
    Y-hat_X = [e_X | Vt_X Lc^-T] for X in {W_m, B_m}:
        G_X = 1/2 (R_X^-1 Y-hat_X Y-hat_X^T R_X^-1 - R_X^-1),  G_m = G_W - pad(G_B)
        Vt-bar_W += R_W^-1 (e_W beta^T - Vt_W C^-1) - pad(same for B) - 2 G_m Vt_W
        (R_W = K_W + sigma_n^2 I - Vt_W Vt_W^T)
        theta-bar += <G_m, dK_W/dtheta> + 2 sigma_n^2 tr(G_m) (log sigma_n)
    then Vt = K_DS L_SS^-T: K_DS-bar = Vt-bar L_SS^-1, L_SS-bar = -L_SS^-T Vt-bar^T Vt
    and the Cholesky adjoint back to Sigma_SS.
    Returns (loglik, grad) with grad ordered (log l_1..d, log sigma_s, log sigma_n).

    windows: the blocks m whose window terms enter (default: all).  Beta and
    Lc are the whole fit's; every step after the window loop is linear in
    Vbar and g, so the results for a partition of the blocks add up to the
    whole gradient (a sharded gradient is one sum of d+2 values)."""
    B = prob.B if B is None else int(B)
    f = fit(prob, B)
    cv = _Cov(prob)
    p = prob
    ptr = p.block_ptr
    M = len(ptr) - 1
    N, d = p.X.shape
    s = p.S.shape[0]
    ell = np.exp(p.log_ell)
    L = cv.L_SS
    Vt = np.empty((N, s))
    for i in range(0, N, 8192):
        Vt[i:i + 8192] = cv.W(p.X[i:i + 8192]).T
    beta = f.beta                                            # C^-1 y_V
    Lc = f.Lc                                                # chol(C), C = I + A
    Cinv = sla.cho_solve((Lc, True), np.eye(s))
    r = p.y - p.mean
    e = r - Vt @ beta
    Vtp = sla.solve_triangular(Lc, Vt.T, lower=True).T       # Vt Lc^-T
    Vbar = np.zeros((N, s))
    g = np.zeros(d + 2)

    def win_terms(idx):
        R = cv.R_train(idx, idx)
        cf = sla.cho_factor(R, lower=True)
        Rinv = sla.cho_solve(cf, np.eye(idx.size))
        Yh = np.column_stack([e[idx], Vtp[idx]])
        Phi = Rinv @ Yh
        G = 0.5 * (Phi @ Phi.T - Rinv)
        Vdir = Rinv @ (np.outer(e[idx], beta) - Vt[idx] @ Cinv)
        return G, Vdir

    for m in (range(M) if windows is None else windows):
        last = min(m + B, M - 1)
        W = np.arange(ptr[m], ptr[last + 1])
        G, Vdir = win_terms(W)
        if last > m:
            Bk = np.arange(ptr[m + 1], ptr[last + 1])
            GB, VdirB = win_terms(Bk)
            off = int(ptr[m + 1] - ptr[m])
            G[off:, off:] -= GB
            Vdir[off:] -= VdirB
        Vbar[W] += Vdir - 2.0 * G @ Vt[W]
        XW = p.X[W] / ell
        K = cv.K(p.X[W], p.X[W])
        GK = G * K
        for k in range(d):
            dx = XW[:, k][:, None] - XW[:, k][None, :]
            g[k] += np.sum(GK * dx * dx)
        g[d] += 2.0 * np.sum(GK)
        g[d + 1] += 2.0 * cv.sn2 * np.trace(G)
    # Vt = K_DS L^-T
    KbarDS = sla.solve_triangular(L, Vbar.T, lower=True, trans="T").T   # Vbar L^-1
    Lbar = -sla.solve_triangular(L, Vbar.T @ Vt, lower=True, trans="T")  # -L^-T Vbar^T Vt
    Sbar = _tri_adj_chol(L, Lbar)
    Ss = p.S / ell
    for i in range(0, N, 8192):
        Xi = p.X[i:i + 8192]
        KDS = cv.KS(Xi)
        GK = KbarDS[i:i + 8192] * KDS
        Xs = Xi / ell
        for k in range(d):
            dx = Xs[:, k][:, None] - Ss[:, k][None, :]
            g[k] += np.sum(GK * dx * dx)
        g[d] += 2.0 * np.sum(GK)
    KSS = cv.K(p.S, p.S)
    GK = Sbar * KSS
    for k in range(d):
        dx = Ss[:, k][:, None] - Ss[:, k][None, :]
        g[k] += np.sum(GK * dx * dx)
    g[d] += 2.0 * np.sum(GK)
    return f.loglik, g
