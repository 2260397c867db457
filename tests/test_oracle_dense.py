"""Pins of the dense-definition oracle against what the paper and the
mathematics fix (no GPU)."""
import math

import numpy as np
import pytest
import scipy.stats

from oracle import lma_dense as O1
from workloads import make_random_problem


def _prob(seed=0, sizes=(5, 7, 6, 8, 5), B=1, d=2, s=6, test_sizes=None):
    return make_random_problem(seed, sizes, d=d, s=s, B=B, test_sizes=test_sizes)


# ---- SE-ARD covariance (Section 5): closed-form values -----------------------

def test_se_ard_hand_values():
    log_ell = np.log([0.5, 2.0])
    ls = math.log(1.3)
    x0 = np.array([[0.1, -0.4]])
    # identical points: sigma_s^2
    assert O1.se_ard(x0, x0, log_ell, ls)[0, 0] == pytest.approx(1.3 ** 2, rel=1e-15)
    # one length-scale apart along axis 0: sigma_s^2 exp(-1/2)
    x1 = x0 + np.array([[0.5, 0.0]])
    assert O1.se_ard(x0, x1, log_ell, ls)[0, 0] == pytest.approx(1.69 * math.exp(-0.5), rel=1e-14)
    # (0.5, 2.0) apart = one length-scale on each axis: exp(-1)
    x2 = x0 + np.array([[0.5, 2.0]])
    assert O1.se_ard(x0, x2, log_ell, ls)[0, 0] == pytest.approx(1.69 * math.exp(-1.0), rel=1e-14)
    # symmetric in its arguments
    X = np.random.default_rng(0).normal(size=(7, 2))
    K = O1.se_ard(X, X, log_ell, ls)
    assert np.allclose(K, K.T, rtol=0, atol=0)


# ---- special cases (Section 3) ------------------------------------------------

@pytest.mark.parametrize("noisy", [True, False])
def test_B_full_is_full_gp(noisy):
    p = _prob(1, sizes=(4, 6, 5, 7))
    M = len(p.block_ptr) - 1
    dn = O1.lma_dense(p, B=M - 1, noisy=noisy)
    fg = O1.full_gp(p, noisy=noisy)
    assert np.allclose(dn["mean"], fg["mean"], rtol=1e-10, atol=1e-11)
    assert np.allclose(dn["var"], fg["var"], rtol=1e-9, atol=1e-11)
    # Sigma-bar equals Sigma at B = M-1 (Section 3)
    assert np.allclose(dn["Sigmabar"], dn["Sigma"], atol=1e-11)
    # log-likelihood: scipy's multivariate normal at the exact GP covariance
    ref = scipy.stats.multivariate_normal(mean=np.full(p.N, p.mean), cov=fg["K"]).logpdf(p.y)
    assert dn["loglik"] == pytest.approx(ref, rel=1e-11)


def test_B0_is_pic():
    p = _prob(2, sizes=(5, 4, 6, 5))
    dn = O1.lma_dense(p, B=0)
    pic = O1.gaussian_posterior(O1.pic_prior(p), p)
    assert np.allclose(dn["mean"], pic["mean"], rtol=1e-11, atol=1e-12)
    assert np.allclose(dn["var"], pic["var"], rtol=1e-10, atol=1e-12)


def test_inband_blocks_equal_sigma():
    p = _prob(3, sizes=(4, 5, 6, 4, 5, 6), B=2)
    dn = O1.lma_dense(p)
    N = p.N
    ptr = p.block_ptr
    M = len(ptr) - 1
    for m in range(M):
        for n in range(M):
            if abs(m - n) <= 2:
                a = slice(ptr[m], ptr[m + 1])
                b = slice(ptr[n], ptr[n + 1])
                assert np.allclose(dn["Sigmabar"][a, b], dn["Sigma"][a, b], atol=1e-12)
    assert dn["Sigmabar"].shape == (N + p.U, N + p.U)


# ---- Proposition 1: R-bar_DD^-1 is B-block-banded -----------------------------

@pytest.mark.parametrize("B", [1, 2, 3])
def test_prop1_banded_inverse(B):
    p = _prob(4, sizes=(5, 6, 4, 7, 5, 6, 5), B=B)
    dn = O1.lma_dense(p)
    N = p.N
    Rb = dn["Rbar"][:N, :N]
    P = np.linalg.inv(Rb)
    ptr = p.block_ptr
    M = len(ptr) - 1
    scale = np.max(np.abs(P))
    for m in range(M):
        for n in range(M):
            blk = P[ptr[m]:ptr[m + 1], ptr[n]:ptr[n + 1]]
            if abs(m - n) > B:
                assert np.max(np.abs(blk)) < 1e-9 * scale, (m, n)
    # and it is not trivially banded: R-bar itself is dense off the band
    off = Rb[ptr[0]:ptr[1], ptr[B + 1]:ptr[B + 2]]
    assert np.max(np.abs(off)) > 1e-8


# ---- Theorem 1 and its proof ---------------------------------------------------

@pytest.mark.parametrize("B", [0, 1, 2])
def test_trace_identity(B):
    p = _prob(5, sizes=(5, 4, 6, 5, 6), B=B)
    dn = O1.lma_dense(p)
    N = p.N
    R, Rb = dn["R"][:N, :N], dn["Rbar"][:N, :N]
    assert np.trace(R @ np.linalg.inv(Rb)) == pytest.approx(N, rel=1e-10)


def _kl(R, Rh):
    A = R @ np.linalg.inv(Rh)
    sign, ld = np.linalg.slogdet(A)
    return 0.5 * (np.trace(A) - ld - R.shape[0])


def test_thm1_kl_optimal():
    B = 1
    p = _prob(6, sizes=(4, 5, 4, 5, 4), B=B)
    dn = O1.lma_dense(p)
    N = p.N
    R, Rb = dn["R"][:N, :N], dn["Rbar"][:N, :N]
    kl_bar = _kl(R, Rb)
    ptr = p.block_ptr
    M = len(ptr) - 1
    mask = np.zeros((N, N), dtype=bool)
    for m in range(M):
        for n in range(M):
            if abs(m - n) <= B:
                mask[ptr[m]:ptr[m + 1], ptr[n]:ptr[n + 1]] = True
    rng = np.random.default_rng(0)
    Pbar = np.linalg.inv(Rb)
    for t in range(20):
        E = rng.normal(size=(N, N))
        E = 0.5 * (E + E.T) * mask
        P = Pbar + 0.05 * E * np.max(np.abs(Pbar)) / max(1e-12, np.max(np.abs(E)))
        if np.min(np.linalg.eigvalsh(P)) <= 0:
            continue
        assert _kl(R, np.linalg.inv(P)) >= kl_bar - 1e-9
    # block-diagonal R (the PIC residual) has a 0-banded, hence B-banded,
    # inverse and must not beat R-bar
    bd = np.zeros((N, N), dtype=bool)
    for m in range(M):
        bd[ptr[m]:ptr[m + 1], ptr[m]:ptr[m + 1]] = True
    assert _kl(R, np.where(bd, R, 0.0)) > kl_bar + 1e-6


def test_lemma1_factor_structure():
    """Lemma 1: the upper Cholesky factor U of R-bar_DD^-1 (U^T U) has
    U_mn = 0 for m > n and n - m > B."""
    B = 1
    p = _prob(7, sizes=(4, 5, 3, 6, 4), B=B)
    dn = O1.lma_dense(p)
    N = p.N
    P = np.linalg.inv(dn["Rbar"][:N, :N])
    # U^T U = P with U upper triangular: U is the transpose of the lower
    # Cholesky factor of P
    Uu = np.linalg.cholesky(P).T
    assert np.allclose(Uu.T @ Uu, P, rtol=1e-9, atol=1e-9 * np.max(np.abs(P)))
    ptr = p.block_ptr
    M = len(ptr) - 1
    sc = np.max(np.abs(Uu))
    for m in range(M):
        for n in range(M):
            blk = Uu[ptr[m]:ptr[m + 1], ptr[n]:ptr[n + 1]]
            if m > n or n - m > B:
                assert np.max(np.abs(blk)) < 1e-8 * sc


def test_dense_loglik_is_gaussian_density():
    p = _prob(8, sizes=(5, 5, 6), B=1)
    dn = O1.lma_dense(p)
    N = p.N
    ref = scipy.stats.multivariate_normal(mean=np.full(N, p.mean), cov=dn["Sigmabar"][:N, :N]).logpdf(p.y)
    assert dn["loglik"] == pytest.approx(ref, rel=1e-11)
