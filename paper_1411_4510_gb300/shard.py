"""Partitioned LMA fit and prediction across ranks.

Remark 1 of the paper runs LMA on a cluster: each machine computes the local
summaries (Definition 1) of its own blocks, a master sums them into the
global summary (Definition 2) and every machine then predicts its own test
blocks.  Here the gather-and-broadcast is one all-reduce (sum) of the
(s+1) x (s+1) FP64 Gram of local summaries and of the log-determinant sum;
every rank then does the small global step itself.

Rank r of W owns the contiguous block range [m0, m1).  Its sub-problem holds
the training rows of blocks [lo, hi) with lo = max(0, m0 - B) (the windows
m in [n - B, n] that its test blocks n need) and hi = min(M, m1 + B) (the
blankets D^B_m of its last blocks).  The windows of blocks [lo, m1) are
factorised; only those of [m0, m1) enter the local summary, so the B windows
before m0 are the halo that prediction repeats from the neighbouring rank.

The functions that touch the GPU default to the CUDA library's entry points
(lma_fit_local, lma_model_local_summary, lma_model_set_global); they are
parameters so that the host logic can be exercised with other
implementations.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import api


@dataclass(frozen=True)
class Shard:
    rank: int
    world: int
    m0: int        # first owned block (global index)
    m1: int        # one past the last owned block
    lo: int        # first block of the sub-problem
    hi: int        # one past the last block of the sub-problem
    row0: int      # first training row of the sub-problem
    row1: int      # one past its last training row

    @property
    def own_begin(self) -> int:
        """First owned block in sub-problem indices."""
        return self.m0 - self.lo

    @property
    def own_end(self) -> int:
        return self.m1 - self.lo


def plan(block_ptr, B: int, world: int, rank: int) -> Shard:
    """Contiguous block ranges with about equal training rows per rank."""
    ptr = np.asarray(block_ptr, dtype=np.int64)
    M = len(ptr) - 1
    if not (1 <= world <= M) or not (0 <= rank < world):
        raise ValueError(f"need 1 <= world ({world}) <= number of blocks ({M}) and 0 <= rank < world")
    n = int(ptr[-1])
    cuts = [0]
    for r in range(1, world):
        target = n * r / world
        m = int(np.searchsorted(ptr, target))          # first block boundary at or after the target
        m = min(max(m, cuts[-1] + 1), M - (world - r))  # every rank keeps at least one block
        cuts.append(m)
    cuts.append(M)
    m0, m1 = cuts[rank], cuts[rank + 1]
    lo, hi = max(0, m0 - int(B)), min(M, m1 + int(B))
    return Shard(rank, world, m0, m1, lo, hi, int(ptr[lo]), int(ptr[hi]))


def plan_range(block_ptr, B: int, m0: int, m1: int, rank: int = 0, world: int = 1) -> Shard:
    """The shard that owns the given block range [m0, m1), with the same halos
    as plan()."""
    ptr = np.asarray(block_ptr, dtype=np.int64)
    M = len(ptr) - 1
    if not (0 <= m0 < m1 <= M):
        raise ValueError(f"bad block range [{m0}, {m1}) of {M} blocks")
    lo, hi = max(0, m0 - int(B)), min(M, m1 + int(B))
    return Shard(rank, world, m0, m1, lo, hi, int(ptr[lo]), int(ptr[hi]))


def sub_problem(args: dict, sh: Shard) -> dict:
    """The problem arguments (as from api.problem_args) restricted to the shard."""
    ptr = np.asarray(args["block_ptr"], dtype=np.int64)
    out = dict(args)
    out["X"] = args["X"][sh.row0:sh.row1]
    out["y"] = args["y"][sh.row0:sh.row1]
    out["block_ptr"] = ptr[sh.lo:sh.hi + 1] - ptr[sh.lo]
    return out


def test_rows(test_block_ptr, sh: Shard):
    """(first, last+1) test rows of the shard's blocks and the test_block_ptr
    of its sub-problem (empty blocks outside [m0, m1))."""
    tp = np.asarray(test_block_ptr, dtype=np.int64)
    u0, u1 = int(tp[sh.m0]), int(tp[sh.m1])
    sub = np.zeros(sh.hi - sh.lo + 1, dtype=np.int64)
    for m in range(sh.lo, sh.hi):
        sub[m - sh.lo + 1] = sub[m - sh.lo] + (int(tp[m + 1] - tp[m]) if sh.m0 <= m < sh.m1 else 0)
    return u0, u1, sub


def allreduce_sum(G, logdet: float, group=None):
    """Sum (G, logdet) over the ranks of `group` with torch.distributed (one
    collective on G with logdet appended); the identity without a group."""
    import torch
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return G, logdet
    dev = G.device if isinstance(G, torch.Tensor) else torch.device("cpu")
    g = G if isinstance(G, torch.Tensor) else torch.as_tensor(np.asarray(G))
    buf = torch.cat([g.reshape(-1).to(torch.float64), torch.tensor([float(logdet)], dtype=torch.float64, device=dev)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf[:-1].reshape(g.shape), float(buf[-1].item())


def sharded_fit(args: dict, sh: Shard, group=None, device=None, precision=api.MIXED, stream=None,
                fit_local=None, local_summary=None, set_global=None, reduce=allreduce_sum):
    """Fit the shard's blocks, all-reduce the summaries, finish the global step.

    Returns the shard's model, which predicts the test blocks [m0, m1) of the
    whole problem (pass their rows with test_rows) and reports the whole
    problem's log-likelihood."""
    fit_local = fit_local or api.lma_fit_local
    local_summary = local_summary or api.lma_model_local_summary
    set_global = set_global or api.lma_model_set_global
    sub = sub_problem(args, sh)
    model = fit_local(**sub, win_begin=0, own_begin=sh.own_begin, own_end=sh.own_end, precision=precision,
                      stream=stream)
    G, logdet = local_summary(model, device)
    G, logdet = reduce(G, logdet, group)
    set_global(model, G, logdet, int(np.asarray(args["block_ptr"])[-1]))
    return model


def allreduce_vec(v, group=None):
    """Sum a host vector over the ranks of `group` (identity without one)."""
    import torch
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return np.asarray(v)
    t = torch.as_tensor(np.asarray(v, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def sharded_loglik_grad(model, group=None, model_grad=None, reduce=allreduce_vec):
    """Gradient of the whole problem's log-likelihood from a shard's model
    (sharded_fit): the adjoint of the shard's own windows, then one
    all-reduce of the d+2 values (the adjoint is linear in the window terms
    after them).  Returns the whole gradient on every rank."""
    model_grad = model_grad or api.lma_model_loglik_grad
    return reduce(model_grad(model), group)

