"""Predictive covariance (Eq. vapvar).  Each test block with itself through
lma_predict_cov against the oracle's local route (itself pinned to the
dense definition); its diagonal is the variance of the same call (to
rounding in the mixed form, whose variance takes the tensor-core path).
Between test blocks through lma_predict_cov_blocks: every block pair of
small problems (B = 0..3, ragged 64-row tiles, an empty test block) against
the dense definition over V = D u U, and all 256 pairs of a 16-block C2
case against the oracle's predict_cov_blocks, off-band pairs (the low-rank
term alone) reported separately."""
import numpy as np
import pytest

from _parity import Collector

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


# ---- covariance between test blocks (lma_predict_cov_blocks) ----------------

TINY = [
    # (seed, block sizes, test sizes, B, d, s), as in tests/test_oracle_xcov.py
    (3, (30, 25, 28, 31, 27, 26), (4, 0, 5, 4, 3, 4), 0, 3, 12),
    (4, (30, 25, 28, 31, 27, 26), (4, 0, 5, 4, 3, 4), 1, 3, 12),
    (5, (30, 25, 28, 31, 27, 26), (4, 0, 5, 4, 3, 4), 2, 3, 12),
    (6, (30, 25, 28, 31, 27, 26), (4, 0, 5, 4, 3, 4), 3, 3, 12),
    (7, (70, 65, 90, 80, 75, 85, 60), (70, 9, 0, 66, 1, 130, 12), 1, 2, 40),   # several 64-row tiles, ragged
]
XCOV_MIXED = 1.5e-3        # measured at most 4.8e-4 (norm-wise, the |S| = 40, B = 1 ragged case); 1.5e-4 off the band


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("case", TINY, ids=[f"B{c[3]}_s{c[5]}" for c in TINY])
def test_full_covariance_equals_dense_definition(L, case, prec):
    """Every block pair against the dense Eq. (vapvar) over V = D u U with
    R-bar by the recursion of Eq. (ares): off-band pairs included."""
    from oracle import lma_dense as O1
    from workloads import make_random_problem
    seed, sizes, tsizes, B, d, s = case
    p = make_random_problem(seed, sizes, d=d, s=s, B=B, test_sizes=tsizes)
    ref = O1.lma_dense(p)["cov"]
    model = L.lma_fit(precision=getattr(L, prec), **L.problem_args(p))
    mean, var, C = L.lma_predict_cov_full(model, p.XU, p.test_block_ptr)
    assert C.shape == ref.shape
    tol = TOL_FP64 if prec == "FP64" else XCOV_MIXED
    c = Collector()
    c.check(f"xcov_dense_B{B}_s{s}_{prec.lower()}", "cov", C, ref, tol, tol)
    c.done()
    # the diagonal is the variance of the same call
    dtol = 1e-10 if prec == "FP64" else 1e-3
    assert np.allclose(np.diag(C), var, rtol=dtol, atol=dtol * 1e-2)


@pytest.fixture(scope="module", params=[1, 2])
def xcase(request):
    from oracle import lma_oracle as O2
    from workloads import make_problem
    p = make_problem("C2", N=1600, M=16, s=64, U=320, B=request.param)
    f = O2.fit(p)
    M = len(p.block_ptr) - 1
    pairs = [(a, b) for a in range(M) for b in range(M)]
    return p, pairs, O2.predict_cov_blocks(f, pairs)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_cross_block_covariance_matches_oracle(L, xcase, prec):
    """C2 recipe at N = 1,600 (16 k-means blocks, |S| = 64, 320 test points):
    all 256 block pairs against the oracle's predict_cov_blocks, the whole
    matrix symmetric, its in-block part equal to lma_predict_cov's."""
    p, pairs, ref = xcase
    model = L.lma_fit(precision=getattr(L, prec), **L.problem_args(p))
    mean, var, blocks = L.lma_predict_cov_blocks(model, p.XU, p.test_block_ptr, pairs)
    tp = p.test_block_ptr
    U = tp[-1]
    full, want = np.zeros((U, U)), np.zeros((U, U))
    band = np.zeros((U, U), dtype=bool)
    for (a, b), C, R in zip(pairs, blocks, ref):
        assert C.shape == R.shape
        full[tp[a]:tp[a + 1], tp[b]:tp[b + 1]] = C
        want[tp[a]:tp[a + 1], tp[b]:tp[b + 1]] = R
        band[tp[a]:tp[a + 1], tp[b]:tp[b + 1]] = abs(a - b) <= p.B
    tol = TOL_FP64 if prec == "FP64" else XCOV_MIXED
    test = f"xcov_c2_n1600_B{p.B}_{prec.lower()}"
    c = Collector()
    c.check(test, "cov", full, want, tol, tol)
    c.check(test, "cov off the band", full[~band], want[~band], tol, tol)
    c.done()
    stol = 1e-12 if prec == "FP64" else 1e-5
    assert np.abs(full - full.T).max() <= stol * np.abs(full).max()
    _, _, within = L.lma_predict_cov(model, p.XU, tp)
    for n, W in enumerate(within):
        if W is not None:
            assert np.array_equal(W, full[tp[n]:tp[n + 1], tp[n]:tp[n + 1]])


def test_cross_block_request_order_and_device_io(L, xcase):
    """Requests in any order, repeated, transposed and with an empty test
    block; device input gives device blocks equal to the host call's."""
    import torch
    p, pairs, ref = xcase
    tp = p.test_block_ptr
    M = len(tp) - 1
    empty = [n for n in range(M) if tp[n + 1] == tp[n]]
    req = [(5, 2), (2, 5), (0, 0), (15, 3), (5, 2), (7, 8)] + ([(empty[0], 3)] if empty else [])
    model = L.lma_fit(precision=L.FP64, **L.problem_args(p))
    _, _, host = L.lma_predict_cov_blocks(model, p.XU, tp, req)
    _, _, dev = L.lma_predict_cov_blocks(model, torch.as_tensor(p.XU, device="cuda:0"), tp, req)
    scale = max(np.abs(R).max() for R in ref if R.size)
    for (a, b), H, Dv in zip(req, host, dev):
        R = ref[pairs.index((a, b))]
        assert H.shape == R.shape == tuple(Dv.shape)
        if R.size:
            assert np.abs(H - R).max() <= TOL_FP64 * scale
            assert np.array_equal(H, Dv.cpu().numpy())
    assert np.array_equal(host[0], host[4])
    assert np.array_equal(host[0], host[1].T) or np.allclose(host[0], host[1].T, rtol=1e-13, atol=1e-15)


def test_cross_block_argument_errors(L, xcase):
    from paper_1411_4510_gb300 import _abi
    p, _, _ = xcase
    model = L.lma_fit(precision=L.FP64, **L.problem_args(p))
    M = len(p.block_ptr) - 1
    for bad in ([(0, M)], [(-1, 0)]):
        with pytest.raises(_abi.LMAError):
            L.lma_predict_cov_blocks(model, p.XU, p.test_block_ptr, bad)
