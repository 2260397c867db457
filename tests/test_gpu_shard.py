"""GPU side of the partitioned fit: two or three shards run one after the
other on one GPU (lma_fit_local on each sub-problem, the Grams summed on the
device, lma_model_set_global on each) must reproduce the whole fit's
log-likelihood and, shard by shard, its predictions of the test blocks each
shard owns; both are also checked directly against the FP64 oracle (Remark
1: the machines' local summaries add up to Definition 2's global summary),
with the FP64 bound 1e-9 and the mixed bounds of test_gpu_parity.py."""
import numpy as np
import pytest

from _parity import check, check_scalar

pytestmark = pytest.mark.gpu

_ORACLE = {}


def _oracle(B):
    """FP64 oracle fit and prediction of the shard tests' problem (cached per B)."""
    if B not in _ORACLE:
        from oracle import lma_oracle as O2
        from workloads import make_problem
        p = make_problem("C2", N=3200, M=16, s=100, U=400, B=B)
        f = O2.fit(p)
        m, v = O2.predict(f)
        _ORACLE[B] = (f.loglik, m, v)
    return _ORACLE[B]


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1411_4510_gb300 import build
    build.build()
    import paper_1411_4510_gb300 as L
    torch.cuda.set_device(0)
    return L


@pytest.mark.parametrize("prec,tol_ll,tol_mean", [("FP64", 1e-11, 1e-11), ("MIXED", 1e-6, 2e-5)])
@pytest.mark.parametrize("B,world", [(1, 2), (2, 2), (2, 3)])
def test_sharded_equals_whole(L, prec, tol_ll, tol_mean, B, world):
    import torch
    from paper_1411_4510_gb300 import api, shard
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=B)
    args = L.problem_args(p)
    precision = getattr(L, prec)
    whole = L.lma_fit(precision=precision, **args)
    assert L.lma_model_precision(whole) == precision, "the mixed fit was redone in FP64"
    ll_whole = L.lma_model_loglik(whole)
    mean_w, var_w = L.lma_predict(whole, p.XU, p.test_block_ptr)
    shards = [shard.plan(p.block_ptr, B, world, r) for r in range(world)]
    models, G, ld = [], None, 0.0
    for sh in shards:
        sub = shard.sub_problem(args, sh)
        m = api.lma_fit_local(**sub, win_begin=0, own_begin=sh.own_begin, own_end=sh.own_end, precision=precision)
        assert L.lma_model_precision(m) == precision, "the mixed local fit was redone in FP64"
        g, l = api.lma_model_local_summary(m, device=torch.device("cuda:0"))
        G = g if G is None else G + g
        ld += l
        models.append(m)
    for sh, m in zip(shards, models):
        api.lma_model_set_global(m, G, ld, p.block_ptr[-1])
        ll = L.lma_model_loglik(m)
        assert abs(ll - ll_whole) <= tol_ll * abs(ll_whole), (ll, ll_whole)
        u0, u1, tp = shard.test_rows(p.test_block_ptr, sh)
        mean, var = L.lma_predict(m, p.XU[u0:u1], tp)
        assert np.linalg.norm(mean - mean_w[u0:u1]) <= tol_mean * np.linalg.norm(mean_w[u0:u1])
        assert np.linalg.norm(var - var_w[u0:u1]) <= 10 * tol_mean * np.linalg.norm(var_w[u0:u1])
        ll_o, m_o, v_o = _oracle(B)
        t = f"shard_b{B}_w{world}_r{sh.rank}_{prec.lower()}"
        if prec == "FP64":
            check_scalar(t, "loglik", ll, ll_o, 1e-9)
            check(t, "mean", mean, m_o[u0:u1], 1e-9, 1e-9)
            check(t, "var", var, v_o[u0:u1], 1e-9, 1e-9, positive=True)
        else:
            check_scalar(t, "loglik", ll, ll_o, 1.5e-4)
            check(t, "mean", mean, m_o[u0:u1], 1e-4, 3e-4)
            check(t, "var", var, v_o[u0:u1], 6e-4, 5e-2, positive=True)


def test_fit_local_rejects_bad_ranges(L):
    from paper_1411_4510_gb300 import api
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=1)
    args = L.problem_args(p)
    for wb, ob, oe in ((0, 3, 3), (4, 3, 6), (0, 0, 17), (-1, 0, 4)):
        with pytest.raises(L.LMAError):
            api.lma_fit_local(**args, win_begin=wb, own_begin=ob, own_end=oe)


def test_predict_needs_global_and_windows(L):
    from paper_1411_4510_gb300 import api
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=1)
    args = L.problem_args(p)
    m = api.lma_fit_local(**args, win_begin=4, own_begin=4, own_end=8)
    with pytest.raises(L.LMAError):
        L.lma_model_loglik(m)
    G, ld = api.lma_model_local_summary(m)
    api.lma_model_set_global(m, G, ld, p.block_ptr[-1])
    # test block 2 needs window 1, which this model does not hold
    tp = np.zeros(17, dtype=np.int64)
    tp[3:] = 1
    with pytest.raises(L.LMAError):
        L.lma_predict(m, p.XU[:1], tp)


@pytest.mark.parametrize("prec,tol_whole,tol_oracle", [("FP64", 1e-11, 1e-9), ("MIXED", 5e-5, 1.5e-3)])
@pytest.mark.parametrize("B,world", [(1, 2), (2, 3)])
def test_sharded_gradient_adds_up(L, prec, tol_whole, tol_oracle, B, world):
    """lma_model_loglik_grad of each shard's model (its own windows' part of
    the adjoint) summed over the shards: the whole problem's gradient.

    Mixed bounds about three times the measurement: the shards' sum differs
    from the whole mixed gradient by 1.1e-5 element-wise (their global
    summaries are summed in another order and their edge windows compute the
    residual tiles the whole fit copies, so beta and L_C move in the last FP32
    bits, which the gradient's cancellation amplifies), and both are 4.6e-4
    from the oracle on this C2-recipe case (|S| = 100, sigma_s^2 / sigma_n^2
    = 400)."""
    import torch
    from oracle import lma_oracle as O2
    from paper_1411_4510_gb300 import api, shard
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=B)
    args = L.problem_args(p)
    precision = getattr(L, prec)
    ll_whole, g_whole = L.lma_loglik_grad(precision=precision, **args)
    shards = [shard.plan(p.block_ptr, B, world, r) for r in range(world)]
    models, G, ld = [], None, 0.0
    for sh in shards:
        sub = shard.sub_problem(args, sh)
        m = api.lma_fit_local(**sub, win_begin=0, own_begin=sh.own_begin, own_end=sh.own_end, precision=precision)
        assert L.lma_model_precision(m) == precision
        g, l = api.lma_model_local_summary(m, device=torch.device("cuda:0"))
        G = g if G is None else G + g
        ld += l
        models.append(m)
    total = 0.0
    for m in models:
        api.lma_model_set_global(m, G, ld, p.block_ptr[-1])
        total = total + L.lma_model_loglik_grad(m)
    t = f"shard_grad_b{B}_w{world}_{prec.lower()}"
    check(t, "grad vs whole", total, g_whole, tol_whole, tol_whole)
    _, g_o = O2.loglik_grad(p)
    check(t, "grad vs oracle", total, g_o, tol_oracle, tol_oracle)


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-12), ("MIXED", 1e-6)])
def test_model_gradient_equals_loglik_grad(L, prec, tol):
    """lma_model_loglik_grad on a model of lma_fit repeats lma_loglik_grad
    without refitting."""
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=1)
    args = L.problem_args(p)
    precision = getattr(L, prec)
    ll, g = L.lma_loglik_grad(precision=precision, **args)
    m = L.lma_fit(precision=precision, **args)
    check(f"model_grad_{prec.lower()}", "grad", L.lma_model_loglik_grad(m), g, tol, tol)

