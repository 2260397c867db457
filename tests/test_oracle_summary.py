"""Pins of the summary-form oracle (Definitions 1-2, Theorem 2, local-route
prediction, summary log-likelihood, hand adjoint) against the dense
definition, special cases, finite differences and invariances (no GPU)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import lma_dense as O1
from oracle import lma_oracle as O2
from workloads import make_random_problem, make_toy

CASES = [
    # (seed, sizes, B, d, s)
    (0, (5, 7, 6, 8, 5), 1, 2, 6),
    (1, (6, 4, 9, 5, 7, 6), 2, 3, 8),
    (2, (5, 5, 5, 5), 0, 2, 5),
    (3, (4, 6, 5, 7), 3, 2, 6),      # B = M-1
    (4, (9, 3, 6, 4, 8, 5, 6), 1, 4, 10),
    (5, (3, 8, 5, 6, 4, 7, 5, 6), 3, 2, 7),
]


def _p(seed, sizes, B, d, s):
    rng = np.random.default_rng(seed)
    ts = rng.integers(0, 4, size=len(sizes))
    return make_random_problem(seed, sizes, d=d, s=s, B=B, test_sizes=ts)


@pytest.mark.parametrize("case", CASES)
def test_summary_loglik_equals_dense(case):
    p = _p(*case)
    assert O2.fit(p).loglik == pytest.approx(O1.lma_dense(p)["loglik"], rel=1e-11, abs=1e-10)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("noisy", [True, False])
def test_local_route_equals_dense(case, noisy):
    p = _p(*case)
    dn = O1.lma_dense(p, noisy=noisy)
    mean, var = O2.predict(O2.fit(p), noisy=noisy)
    assert np.allclose(mean, dn["mean"], rtol=1e-10, atol=1e-11)
    assert np.allclose(var, dn["var"], rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("case", CASES[:4])
def test_theorem2_equals_dense(case):
    """Theorem 2 assembled from Definitions 1-2 reproduces Eqs. (vapmu)/(vapvar)."""
    p = _p(*case)
    dn = O1.lma_dense(p)
    f = O2.fit(p, keep_blocks=True)
    N = p.N
    SbDU = dn["Sigmabar"][:N, N:]
    Suu = np.diag(dn["Sigma"][N:, N:])
    mean, var = O2.predict_thm2(f, SbDU, Suu)
    assert np.allclose(mean, dn["mean"], rtol=1e-10, atol=1e-11)
    assert np.allclose(var, dn["var"], rtol=1e-9, atol=1e-11)


def test_global_summary_matches_dense_identity():
    """Sigma-ddot_SS - Sigma_SS = Sigma_SD R-bar_DD^-1 Sigma_DS and
    y-ddot_S = Sigma_SD R-bar_DD^-1 (y - mu) (proof of Theorem 2)."""
    p = _p(*CASES[1])
    dn = O1.lma_dense(p)
    f = O2.fit(p)
    N = p.N
    Rb = dn["Rbar"][:N, :N]
    KDS = O1.se_ard(p.X, p.S, p.log_ell, p.log_sigma_s)
    Pinv = np.linalg.inv(Rb)
    assert np.allclose(f.Sdd_SS - f.Sigma_SS, KDS.T @ Pinv @ KDS, rtol=1e-9, atol=1e-9)
    assert np.allclose(f.ydd_S, KDS.T @ Pinv @ (p.y - p.mean), rtol=1e-9, atol=1e-9)
    # log|R-bar_DD| = sum of log|R-dot_m^-1|
    assert f.logdet_R == pytest.approx(np.linalg.slogdet(Rb)[1], rel=1e-10)


def test_B_full_summary_is_full_gp():
    p = _p(3, (4, 6, 5, 7), 3, 2, 6)
    fg = O1.full_gp(p)
    mean, var = O2.predict(O2.fit(p))
    assert np.allclose(mean, fg["mean"], rtol=1e-10, atol=1e-11)
    assert np.allclose(var, fg["var"], rtol=1e-9, atol=1e-11)


def test_uneven_and_empty_test_blocks():
    p = make_random_problem(11, (3, 9, 2, 6, 5), d=2, s=5, B=2, test_sizes=(0, 3, 0, 0, 4))
    dn = O1.lma_dense(p)
    mean, var = O2.predict(O2.fit(p))
    assert mean.shape == (7,)
    assert np.allclose(mean, dn["mean"], rtol=1e-10, atol=1e-11)
    assert np.allclose(var, dn["var"], rtol=1e-9, atol=1e-11)


# ---- invariances -------------------------------------------------------------

def test_support_permutation_invariance():
    p = _p(*CASES[0])
    perm = np.random.default_rng(1).permutation(p.s)
    q = p.__class__(**{**p.__dict__, "S": p.S[perm]})
    a, b = O2.predict(O2.fit(p)), O2.predict(O2.fit(q))
    assert np.allclose(a[0], b[0], rtol=1e-10) and np.allclose(a[1], b[1], rtol=1e-9)
    assert O2.fit(p).loglik == pytest.approx(O2.fit(q).loglik, rel=1e-9)


def test_translation_invariance_and_target_scaling():
    p = _p(*CASES[4])
    sh = np.linspace(-3, 5, p.d)
    q = p.__class__(**{**p.__dict__, "X": p.X + sh, "S": p.S + sh, "XU": p.XU + sh})
    a, b = O2.predict(O2.fit(p)), O2.predict(O2.fit(q))
    assert np.allclose(a[0], b[0], rtol=1e-9) and np.allclose(a[1], b[1], rtol=1e-8)
    c = 2.5
    q2 = p.__class__(**{**p.__dict__, "y": p.mean + c * (p.y - p.mean)})
    m2, v2 = O2.predict(O2.fit(q2))
    assert np.allclose(m2 - p.mean, c * (a[0] - p.mean), rtol=1e-10, atol=1e-12)
    assert np.allclose(v2, a[1], rtol=1e-12)


# ---- gradient -----------------------------------------------------------------

def _with_theta(p, th):
    d = p.d
    return p.__class__(**{**p.__dict__, "log_ell": np.array(th[:d]), "log_sigma_s": float(th[d]),
                          "log_sigma_n": float(th[d + 1])})


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[2], CASES[4]])
def test_grad_central_fd(case):
    p = _p(*case)
    ll, g = O2.loglik_grad(p)
    assert ll == pytest.approx(O2.fit(p).loglik, rel=1e-13)
    th = np.concatenate([p.log_ell, [p.log_sigma_s, p.log_sigma_n]])
    h = 1e-5
    fd = np.empty_like(th)
    for k in range(th.size):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (O2.fit(_with_theta(p, tp)).loglik - O2.fit(_with_theta(p, tm)).loglik) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-6 * max(1.0, np.max(np.abs(fd))))


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[2], CASES[4]])
def test_grad_partition_of_windows_adds_up(case):
    """The adjoint is linear in the window terms after the window loop, so
    the gradients restricted to the windows of a partition of the blocks add
    up to the whole gradient (the sharded gradient's single reduction)."""
    p = _p(*case)
    _, g = O2.loglik_grad(p)
    M = len(p.block_ptr) - 1
    cuts = sorted({0, M // 3, (2 * M) // 3, M})
    parts = [O2.loglik_grad(p, windows=range(a, b))[1] for a, b in zip(cuts, cuts[1:])]
    assert np.allclose(sum(parts), g, rtol=1e-10, atol=1e-10 * np.max(np.abs(g)))
    _, g_all = O2.loglik_grad(p, windows=range(M))
    assert np.array_equal(g_all, g)


def test_grad_full_gp_closed_form():
    """At B = M-1 the LMA likelihood is the exact GP one, whose gradient is
    1/2 tr((a a^T - K^-1) dK/dtheta), a = K^-1 (y - mu)."""
    p = _p(3, (4, 6, 5, 7), 3, 2, 6)
    _, g = O2.loglik_grad(p)
    d = p.d
    ell = np.exp(p.log_ell)
    Kf = O1.se_ard(p.X, p.X, p.log_ell, p.log_sigma_s)
    sn2 = math.exp(2 * p.log_sigma_n)
    K = Kf + sn2 * np.eye(p.N)
    Ki = np.linalg.inv(K)
    a = Ki @ (p.y - p.mean)
    Wm = np.outer(a, a) - Ki
    ref = np.empty(d + 2)
    for k in range(d):
        dx = (p.X[:, k][:, None] - p.X[:, k][None, :]) / ell[k]
        ref[k] = 0.5 * np.sum(Wm * Kf * dx * dx)
    ref[d] = 0.5 * np.sum(Wm * 2 * Kf)
    ref[d + 1] = 0.5 * np.trace(Wm) * 2 * sn2
    assert np.allclose(g, ref, rtol=1e-7, atol=1e-8)


# ---- Appendix D toy (soft, Remark 4) -------------------------------------------

def test_toy_appendix_d():
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "toy_appendix_d.json")))
    p = make_toy(n_test=401)
    assert p.M == gold["M"] and p.B == gold["B"] and p.s == gold["S"] and p.N == gold["D"]
    assert math.exp(p.log_ell[0]) == pytest.approx(gold["ell"])
    assert math.exp(p.log_sigma_n) == pytest.approx(gold["sigma_n"])
    assert math.exp(p.log_sigma_s) == pytest.approx(gold["sigma_s"])
    assert p.mean == pytest.approx(gold["mu"])
    f = O2.fit(p)
    mean, var = O2.predict(f)
    x = p.XU[:, 0]
    order = np.argsort(x)
    x, mean, var = x[order], mean[order], var[order]
    truth = 1.0 + np.cos(x)
    inside = np.abs(mean - truth) <= 1.96 * np.sqrt(var) + 0.05
    assert np.mean(inside) > 0.95
    # no visible jump at the block boundaries: the step across each split is
    # a small fraction of the noise level (exact continuity is not claimed)
    sn = gold["sigma_n"]
    for b in gold["split_points"]:
        i = np.searchsorted(x, b)
        slope = (mean[i + 1] - mean[i - 2]) / (x[i + 1] - x[i - 2])
        jump = abs((mean[i] - mean[i - 1]) - slope * (x[i] - x[i - 1]))
        assert jump < 0.1 * sn, (b, jump)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("noisy", [True, False])
def test_block_covariance_equals_dense(case, noisy):
    """Eq. (vapvar) on each test block U_n x U_n: the local route's block
    covariance equals the dense definition's diagonal blocks, and its
    diagonal equals the local-route variance."""
    p = _p(*case)
    f = O2.fit(p)
    d = O1.lma_dense(p, noisy=noisy)
    covs = O2.predict_cov(f, noisy=noisy)
    _, var = O2.predict(f, noisy=noisy)
    tp = p.test_block_ptr
    for n, C in enumerate(covs):
        u = np.arange(tp[n], tp[n + 1])
        if u.size == 0:
            assert C is None
            continue
        ref = d["cov"][np.ix_(u, u)]
        assert np.allclose(C, ref, rtol=1e-9, atol=1e-11)
        assert np.allclose(np.diag(C), var[u], rtol=1e-12, atol=1e-13)
        assert np.allclose(C, C.T, rtol=0, atol=1e-12)
