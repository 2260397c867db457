"""Partitioned fit (Remark 1 as one all-reduce): the block plan, the halo of
the sub-problems and the reduction, exercised on CPU ranks (gloo, world size
2) with the summary-form oracle standing in for the GPU local step.  The GPU
side of the same path is tested in test_gpu_shard.py."""
import math
import os
import socket
import types

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import lma_oracle as O2
from paper_1411_4510_gb300 import shard
from workloads import make_random_problem


def _problem(seed=3, sizes=(6, 5, 7, 4, 6, 5, 8, 5), B=2, d=2, s=6):
    return make_random_problem(seed, sizes, d=d, s=s, B=B, test_sizes=[2] * len(sizes))


def _ns(args: dict, src):
    """A problem object for the oracle from shard.sub_problem's arguments."""
    return types.SimpleNamespace(X=args["X"], y=args["y"], block_ptr=np.asarray(args["block_ptr"]), S=args["S"],
                                 B=args["B"], log_ell=args["log_ell"], log_sigma_s=args["log_sigma_s"],
                                 log_sigma_n=args["log_sigma_n"], jitter=args["jitter"], mean=args["mean"])


def _args(p):
    return dict(X=p.X, y=p.y, block_ptr=p.block_ptr, S=p.S, B=p.B, log_ell=p.log_ell, log_sigma_s=p.log_sigma_s,
                log_sigma_n=p.log_sigma_n, jitter=p.jitter, mean=p.mean)


@pytest.mark.parametrize("M,world", [(1, 1), (8, 1), (8, 2), (8, 3), (9, 4), (5, 5)])
@pytest.mark.parametrize("B", [0, 1, 3])
def test_plan_partitions_blocks(M, world, B):
    rng = np.random.default_rng(M * 10 + world)
    ptr = np.concatenate([[0], np.cumsum(rng.integers(1, 9, size=M))])
    shards = [shard.plan(ptr, B, world, r) for r in range(world)]
    assert shards[0].m0 == 0 and shards[-1].m1 == M
    for a, b in zip(shards, shards[1:]):
        assert a.m1 == b.m0
    for sh in shards:
        assert sh.m0 < sh.m1
        assert sh.lo == max(0, sh.m0 - B) and sh.hi == min(M, sh.m1 + B)
        assert (sh.row0, sh.row1) == (ptr[sh.lo], ptr[sh.hi])


def test_plan_rejects_more_ranks_than_blocks():
    with pytest.raises(ValueError):
        shard.plan([0, 3, 6], 1, 3, 0)


def test_local_summaries_add_up():
    """Definition 2: the global sums are sums of per-block terms, so any
    partition of the blocks adds up to the whole fit's summaries."""
    p = _problem()
    f = O2.fit(p)
    parts = [O2.local_summaries(p, b) for b in ([0, 1, 2], [3, 4], [5, 6, 7])]
    A = sum(q[0] for q in parts)
    assert np.allclose(0.5 * (A + A.T), f.A_white, rtol=1e-11, atol=1e-12)
    assert np.allclose(sum(q[1] for q in parts), f.ydd_white, rtol=1e-11, atol=1e-12)
    assert sum(q[2] for q in parts) == pytest.approx(f.quad, rel=1e-12)
    assert sum(q[3] for q in parts) == pytest.approx(f.logdet_R, rel=1e-12)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("B", [0, 1, 2])
def test_sub_problem_halo_is_enough(world, B):
    """Each shard's owned blocks have the same local summaries on its
    sub-problem (its blocks plus the B-block halos) as on the whole problem."""
    p = _problem(B=B)
    args = _args(p)
    M = len(p.block_ptr) - 1
    for r in range(world):
        sh = shard.plan(p.block_ptr, B, world, r)
        sub = _ns(shard.sub_problem(args, sh), p)
        a = O2.local_summaries(sub, range(sh.own_begin, sh.own_end))
        b = O2.local_summaries(p, range(sh.m0, sh.m1))
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=1e-10, atol=1e-12)
    assert M == 8


def test_test_rows_select_owned_blocks():
    tp = np.array([0, 2, 2, 5, 6, 9])
    sh = shard.Shard(rank=1, world=2, m0=2, m1=4, lo=1, hi=5, row0=0, row1=0)
    u0, u1, sub = shard.test_rows(tp, sh)
    assert (u0, u1) == (2, 6)
    assert sub.tolist() == [0, 0, 3, 4, 4]


# --- oracle stand-ins for the GPU steps (test infrastructure) ---------------

def _oracle_fit_local(X, y, block_ptr, S, B, log_ell, log_sigma_s, log_sigma_n, win_begin, own_begin, own_end,
                      jitter, mean, precision=None, stream=None):
    sub = types.SimpleNamespace(X=X, y=y, block_ptr=np.asarray(block_ptr), S=S, B=B, log_ell=log_ell,
                                log_sigma_s=log_sigma_s, log_sigma_n=log_sigma_n, jitter=jitter, mean=mean)
    return dict(sub=sub, own=(own_begin, own_end))


def _oracle_local_summary(model, device=None):
    A, ydd, quad, ld = O2.local_summaries(model["sub"], range(*model["own"]))
    s = ydd.size
    G = np.zeros((s + 1, s + 1))
    G[0, 0] = quad
    G[0, 1:] = G[1:, 0] = ydd
    G[1:, 1:] = A
    return G, ld


def _oracle_set_global(model, G, logdet_R, n_total):
    G = np.asarray(G)
    A = 0.5 * (G[1:, 1:] + G[1:, 1:].T)
    Lc = np.linalg.cholesky(np.eye(A.shape[0]) + A)
    w = sla.solve_triangular(Lc, G[1:, 0], lower=True)
    model["loglik"] = (-0.5 * (G[0, 0] - w @ w) - 0.5 * (logdet_R + 2.0 * np.sum(np.log(np.diag(Lc))))
                       - 0.5 * n_total * math.log(2.0 * math.pi))
    model["G"] = G


def _rank_main(rank, world, port, B, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem(B=B)
        sh = shard.plan(p.block_ptr, B, world, rank)
        model = shard.sharded_fit(_args(p), sh, fit_local=_oracle_fit_local, local_summary=_oracle_local_summary,
                                  set_global=_oracle_set_global)
        np.save(f"{out_path}.{rank}.npy", np.concatenate([[model["loglik"]], np.asarray(model["G"]).ravel()]))
        # the shard's part of the gradient (the oracle's adjoint restricted to
        # the windows of its blocks) and the all-reduce of the d+2 values
        grad = shard.sharded_loglik_grad(model, model_grad=lambda m: O2.loglik_grad(p, windows=range(sh.m0, sh.m1))[1])
        np.save(f"{out_path}.grad.{rank}.npy", grad)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("B", [1, 2])
def test_sharded_fit_two_gloo_ranks(tmp_path, B):
    import torch.multiprocessing as mp
    world = 2
    out = str(tmp_path / "res")
    mp.start_processes(_rank_main, args=(world, _free_port(), B, out), nprocs=world, start_method="spawn")
    p = _problem(B=B)
    f = O2.fit(p)
    for r in range(world):
        v = np.load(f"{out}.{r}.npy")
        assert v[0] == pytest.approx(f.loglik, rel=1e-11)
        G = v[1:].reshape(p.S.shape[0] + 1, -1)
        assert np.allclose(0.5 * (G[1:, 1:] + G[1:, 1:].T), f.A_white, rtol=1e-10, atol=1e-12)
        assert G[0, 0] == pytest.approx(f.quad, rel=1e-11)
    _, g = O2.loglik_grad(p)
    for r in range(world):
        gr = np.load(f"{out}.grad.{r}.npy")
        assert np.allclose(gr, g, rtol=1e-10, atol=1e-10 * np.max(np.abs(g)))
