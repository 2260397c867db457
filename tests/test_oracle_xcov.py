"""Pins of the oracle's covariance between test blocks (Eq. vapvar on
U_n x U_n', predict_cov_blocks) against the dense definition, and of the two
facts the CUDA path builds on (no GPU):

* the residual part of the predictive covariance,
  R-bar_UU - R-bar_UD R-bar_DD^-1 R-bar_DU, vanishes between test blocks more
  than B apart (Eq. ares: off the band R-bar runs through D-blankets only), so
  there the covariance is the low-rank term alone;
* within the band (n <= n' <= n + B) that part equals
  R_{uu'} - sum_{m = n'-B}^{n} P_(n,m)[u] . P_(n',m)[u'] over the kept window
  columns, P_(n,m) = (L_m^-1 R_{W_m U_n})^T with L_m the blanket-first
  Cholesky factor of window m (Lemma 1), i.e. products of the prediction's
  own right-hand sides: windows m < n' - B drop out because their block rows
  of L_m^-1 R-bar_{W_m u'} are zero when R-bar_{D_m u'} is the recursion of
  Eq. (ares) over block m's blanket.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import lma_dense as O1
from oracle import lma_oracle as O2
from workloads import make_random_problem

CASES = [
    # (seed, block sizes, test sizes, B, d, s)
    (3, (30, 25, 28, 31, 27, 26), (4, 0, 5, 4, 3, 4), 0, 3, 12),
    (4, (30, 25, 28, 31, 27, 26), (4, 0, 5, 4, 3, 4), 1, 3, 12),
    (5, (30, 25, 28, 31, 27, 26), (4, 0, 5, 4, 3, 4), 2, 3, 12),
    (6, (30, 25, 28, 31, 27, 26), (4, 0, 5, 4, 3, 4), 3, 3, 12),
    (7, (12, 9, 14, 8, 11, 10, 13), (3, 2, 0, 4, 1, 3, 2), 1, 2, 7),
    (8, (12, 9, 14, 8, 11, 10, 13), (3, 2, 0, 4, 1, 3, 2), 6, 2, 7),   # B = M-1: the full GP
]


def _p(seed, sizes, tsizes, B, d, s):
    return make_random_problem(seed, sizes, d=d, s=s, B=B, test_sizes=tsizes)


def _all_pairs(p):
    M = len(p.block_ptr) - 1
    return [(a, b) for a in range(M) for b in range(M)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("noisy", [True, False])
def test_cov_blocks_equal_dense_definition(case, noisy):
    p = _p(*case)
    o = O1.lma_dense(p, noisy=noisy)
    f = O2.fit(p)
    tp = p.test_block_ptr
    pairs = _all_pairs(p)
    blocks = O2.predict_cov_blocks(f, pairs, noisy=noisy)
    scale = np.abs(o["cov"]).max()
    for (a, b), C in zip(pairs, blocks):
        ref = o["cov"][tp[a]:tp[a + 1], tp[b]:tp[b + 1]]
        assert C.shape == ref.shape
        if C.size:
            assert np.abs(C - ref).max() <= 1e-10 * scale, (a, b)


@pytest.mark.parametrize("case", CASES[:4])
def test_in_block_equals_predict_cov(case):
    p = _p(*case)
    f = O2.fit(p)
    M = len(p.block_ptr) - 1
    diag = O2.predict_cov_blocks(f, [(n, n) for n in range(M)])
    within = O2.predict_cov(f)
    for n in range(M):
        if within[n] is None:
            assert diag[n].size == 0
        else:
            assert np.allclose(diag[n], within[n], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("case", CASES[:5])
def test_residual_part_vanishes_off_band(case):
    """Dense definition: the posterior covariance of the R-bar part is
    B-block-banded over the test blocks (and nonzero inside the band)."""
    p = _p(*case)
    B = p.B
    o = O1.lma_dense(p)
    Rb, d, u = o["Rbar"], o["d_idx"], o["u_idx"]
    T = Rb[np.ix_(u, u)] - Rb[np.ix_(u, d)] @ np.linalg.solve(Rb[np.ix_(d, d)], Rb[np.ix_(d, u)])
    tp = p.test_block_ptr
    M = len(tp) - 1
    scale = np.abs(T).max()
    inside = 0.0
    for a in range(M):
        for b in range(M):
            blk = T[tp[a]:tp[a + 1], tp[b]:tp[b + 1]]
            if not blk.size:
                continue
            if abs(a - b) > B:
                assert np.abs(blk).max() <= 1e-12 * scale, (a, b)
            elif a != b:
                inside = max(inside, np.abs(blk).max())
    if B > 0:
        assert inside > 1e-6 * scale   # the band is not trivially empty


def _window_factors(cv, p, B):
    ptr = p.block_ptr
    M = len(ptr) - 1
    L, rows, nB = {}, {}, {}
    for m in range(M):
        last = min(m + B, M - 1)
        r = np.arange(ptr[m], ptr[last + 1])[::-1]          # blanket first (reversed rows)
        L[m] = np.linalg.cholesky(cv.R_train(r, r))
        rows[m] = r
        nB[m] = int(ptr[last + 1] - ptr[m + 1])
    return L, rows, nB


@pytest.mark.parametrize("case", CASES)
def test_in_band_residual_part_from_window_rhs(case):
    p = _p(*case)
    B = p.B
    o = O1.lma_dense(p)
    f = O2.fit(p)
    cv = O2._Cov(p)
    L, rows, nB = _window_factors(cv, p, B)
    tp = p.test_block_ptr
    M = len(tp) - 1

    def rhs(n, m):
        Xu = p.XU[tp[n]:tp[n + 1]]
        X = p.X[rows[m]]
        R = cv.K(X, Xu) - cv.W(X).T @ cv.W(Xu)
        return sla.solve_triangular(L[m], R, lower=True).T

    blocks = O2.predict_cov_blocks(f, _all_pairs(p))
    hc = _hc(f, cv, p, B)
    scale = np.abs(o["cov"]).max()
    for (a, b), C in zip(_all_pairs(p), blocks):
        if not C.size or abs(a - b) > B:
            continue
        lo, hi = min(a, b), max(a, b)
        X1, X2 = p.XU[tp[a]:tp[a + 1]], p.XU[tp[b]:tp[b + 1]]
        T = cv.K(X1, X2) - cv.W(X1).T @ cv.W(X2)
        if a == b:
            T = T + cv.sn2 * np.eye(X1.shape[0])
        for m in range(max(0, hi - B), lo + 1):
            c0 = nB[m] if m < lo else 0
            T = T - rhs(a, m)[:, c0:] @ rhs(b, m)[:, c0:].T
        ref = o["cov"][tp[a]:tp[a + 1], tp[b]:tp[b + 1]]
        assert np.abs(T + hc[a].T @ hc[b] - ref).max() <= 1e-10 * scale, (a, b)
        assert np.abs(T + hc[a].T @ hc[b] - C).max() <= 1e-10 * scale, (a, b)


def _hc(f, cv, p, B):
    """hc = L_C^-1 h per test block, h = W_J z^T - W_u (the vector of the local route)."""
    ptr, tp = p.block_ptr, p.test_block_ptr
    M = len(ptr) - 1
    out = {}
    for n in range(M):
        Xu = p.XU[tp[n]:tp[n + 1]]
        Jb = list(range(max(0, n - B), min(M - 1, n + B) + 1))
        rows, P = O2._subchain_precision(cv, ptr, Jb, B)
        WJ, Wu = cv.W(p.X[rows]), cv.W(Xu)
        Z = P @ (cv.K(p.X[rows], Xu) - WJ.T @ Wu)
        out[n] = sla.solve_triangular(f.Lc, WJ @ Z - Wu, lower=True)
    return out


@pytest.mark.parametrize("noisy", [True, False])
def test_full_markov_order_is_the_full_gp_covariance(noisy):
    """B = M-1: the approximation is exact (R-bar = R), so the covariance
    between any two test blocks is the textbook GP posterior covariance."""
    p = make_random_problem(11, (9, 12, 7, 10, 8), d=2, s=6, B=4, test_sizes=(3, 0, 4, 2, 3))
    f = O2.fit(p)
    full = O1.full_gp(p, noisy=noisy)["cov"]
    tp = p.test_block_ptr
    pairs = _all_pairs(p)
    scale = np.abs(full).max()
    for (a, b), C in zip(pairs, O2.predict_cov_blocks(f, pairs, noisy=noisy)):
        ref = full[tp[a]:tp[a + 1], tp[b]:tp[b + 1]]
        if ref.size:
            assert np.abs(C - ref).max() <= 1e-9 * scale, (a, b)
