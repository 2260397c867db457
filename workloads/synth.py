"""Synthetic stand-ins for the paper's workloads (SARCOS, AIMPEAK, EMSLP are not
available; every input here is generated from a seed).

Five configurations follow the experiment shapes of Section 5 of the paper
(Tables 1-3, Fig. 2) at one-GPU scale, plus the 1-D toy of Appendix D:

  C1  N=2,000,   d=2,  U[0,1]^2, y = sin(6 x1) + cos(4 x2) + N(0, 0.1^2),
      16 blocks of 125 sorted by x1, |S|=64, B=1, 500 test points.
  C2  N=40,960,  d=5,  N(0, I_5), random-Fourier-feature SE draw (2,048
      features, l=1, sigma_s=1) + N(0, 0.05^2), 64 equal blocks of 640 in
      k-means-centroid order, |S|=512, B in {1,2,3}, 4,096 test points.
  C3  N=49,152,  d=21, N(0, I_21), RFF SE draw (4,096 features, l=3) +
      N(0, 0.1^2), 96 k-means blocks with sizes clamped to [256, 1024],
      |S|=1,024, B=2, 8,192 test points.
  C4  N=2,000,000, d=8, U[0,1]^8, RFF SE draw (4,096 features, l=0.3) +
      N(0, 0.1^2), 2,000 blocks of 1,000 in Morton order, |S|=2,048, B=1,
      100,000 test points.
  C5  N=65,536,  d=8, as C4 with 128 blocks of 512, |S|=1,024, B=2, no test
      points (log-likelihood and gradient workload).

The generator draws points, targets, the block partition (which the paper
delegates to a clustering scheme it does not specify), the support set (a
random subset of the training inputs, Section 5) and the test-point block
assignment (test points are partitioned like the training points, Section 3).
Numbers are drawn with numpy's PCG64 from SeedSequence(1411 + config index),
split into independent substreams for inputs, noise, RFF weights, the support
set, test points and the k-means initialisation.
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import Optional

import numpy as np

CONFIG_NAMES = ("C1", "C2", "C3", "C4", "C5")


@dataclasses.dataclass
class Problem:
    """One LMA regression problem (Section 3 notation).

    X        (N, d) training inputs D, rows grouped by block (block m owns
             rows block_ptr[m]:block_ptr[m+1]).
    y        (N,)   observed outputs y_D.
    block_ptr (M+1,) int64 partition of D into D_1..D_M.
    S        (s, d) support set inputs (a subset of the training inputs).
    XU, yU   (U, d), (U,) test inputs and their noisy held-out outputs.
    test_block_ptr (M+1,) int64 partition of U into U_1..U_M (same key as D).
    log_ell  (d,)  log length-scales; log_sigma_s, log_sigma_n log signal and
             noise standard deviations; jitter is the absolute value added to
             the diagonal of Sigma_SS; mean is the constant prior mean mu.
    B        Markov order.
    """

    name: str
    X: np.ndarray
    y: np.ndarray
    block_ptr: np.ndarray
    S: np.ndarray
    XU: np.ndarray
    yU: np.ndarray
    test_block_ptr: np.ndarray
    log_ell: np.ndarray
    log_sigma_s: float
    log_sigma_n: float
    jitter: float
    mean: float
    B: int
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def M(self) -> int:
        return int(self.block_ptr.shape[0] - 1)

    @property
    def s(self) -> int:
        return int(self.S.shape[0])

    @property
    def U(self) -> int:
        return int(self.XU.shape[0])

    def with_B(self, B: int) -> "Problem":
        return dataclasses.replace(self, B=int(B))

    def block_sizes(self) -> np.ndarray:
        return np.diff(self.block_ptr)


# ----------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------

def _streams(seed: int, n: int = 6):
    ss = np.random.SeedSequence(seed)
    return [np.random.Generator(np.random.PCG64(c)) for c in ss.spawn(n)]


def rff_draw(rng: np.random.Generator, d: int, n_features: int, ell: float,
             sigma_s: float):
    """Random-Fourier-feature approximation of an SE-kernel GP sample path
    (Rahimi & Recht 2007): f(x) = sigma_s sqrt(2/F) sum_f a_f cos(w_f.x + c_f),
    w_f ~ N(0, ell^-2 I), c_f ~ U[0, 2 pi), a_f ~ N(0, 1).

    The weights are drawn with numpy (bit-identical on every platform); f is
    evaluated in FP64 with torch's multithreaded CPU kernels (a 2-million-point
    draw with 4,096 features is ~8e9 cosines), which may differ from numpy's
    cosine in the last bit: the outputs y agree across machines to ~1e-15
    relative, the partition (built from the inputs only) exactly."""
    W = rng.standard_normal((n_features, d)) / ell
    c = rng.uniform(0.0, 2.0 * math.pi, n_features)
    a = rng.standard_normal(n_features)
    scale = sigma_s * math.sqrt(2.0 / n_features)

    def f(x: np.ndarray) -> np.ndarray:
        import torch
        out = torch.empty(x.shape[0], dtype=torch.float64)
        xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
        Wt, ct, at = torch.from_numpy(W), torch.from_numpy(c), torch.from_numpy(a)
        chunk = 32768
        with torch.no_grad():
            for i in range(0, x.shape[0], chunk):
                ph = torch.addmm(ct, xt[i:i + chunk], Wt.T)
                out[i:i + chunk] = torch.cos_(ph) @ at
        return scale * out.numpy()

    return f


def _sqdist(X: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Squared distances of the rows of X to the point c (or, for c of shape
    (k, d), to each row of c), accumulated axis by axis with elementwise
    operations only: IEEE-exact, so the same bits on every platform (a BLAS
    product or a vectorised reduction could differ in the last bit and flip a
    nearest-centre decision)."""
    if c.ndim == 1:
        out = np.zeros(X.shape[0])
        for q in range(X.shape[1]):
            t = X[:, q] - c[q]
            out += t * t
        return out
    out = np.zeros((X.shape[0], c.shape[0]))
    for q in range(X.shape[1]):
        t = X[:, q][:, None] - c[:, q][None, :]
        out += t * t
    return out


def _dot_axes(X: np.ndarray, v) -> np.ndarray:
    """X @ v accumulated axis by axis (platform-exact, see _sqdist)."""
    out = np.zeros(X.shape[0])
    for q in range(X.shape[1]):
        out += X[:, q] * float(v[q])
    return out


def _kmeans(rng: np.random.Generator, X: np.ndarray, k: int, iters: int = 15):
    """Seeded Lloyd iterations from a k-means++ initialisation (platform-exact:
    distances by _sqdist, sums by np.bincount's in-order accumulation and
    math.fsum)."""
    n = X.shape[0]
    sub = X if n <= 20000 else X[rng.choice(n, 20000, replace=False)]
    centers = np.empty((k, X.shape[1]))
    centers[0] = sub[rng.integers(sub.shape[0])]
    d2 = _sqdist(sub, centers[0])
    for j in range(1, k):
        p = d2 / math.fsum(d2)
        centers[j] = sub[rng.choice(sub.shape[0], p=p)]
        d2 = np.minimum(d2, _sqdist(sub, centers[j]))
    for _ in range(iters):
        lab = _nearest(X, centers)
        cnt = np.bincount(lab, minlength=k)
        for q in range(X.shape[1]):
            sums = np.bincount(lab, weights=X[:, q], minlength=k)
            centers[:, q] = np.where(cnt > 0, sums / np.maximum(cnt, 1), centers[:, q])
    return centers, _nearest(X, centers)


def _nearest(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    out = np.empty(X.shape[0], dtype=np.int64)
    for i in range(0, X.shape[0], 16384):
        out[i:i + 16384] = np.argmin(_sqdist(X[i:i + 16384], C), axis=1)
    return out


def _top_axis(P: np.ndarray, iters: int = 300) -> np.ndarray:
    """Leading principal axis of the rows of P (centred), by a fixed number of
    power iterations on P^T P with exactly rounded sums (math.fsum), so that
    it is bit-identical on every platform; sign: largest component positive."""
    k, d = P.shape
    cov = [[math.fsum(float(P[j, a]) * float(P[j, b]) for j in range(k)) for b in range(d)] for a in range(d)]
    v = [1.0 / math.sqrt(d)] * d
    for _ in range(iters):
        w = [math.fsum(cov[a][b] * v[b] for b in range(d)) for a in range(d)]
        nrm = math.sqrt(math.fsum(x * x for x in w))
        if nrm == 0.0:
            break
        v = [x / nrm for x in w]
    big = max(range(d), key=lambda a: abs(v[a]))
    if v[big] < 0:
        v = [-x for x in v]
    return np.array(v)


def _cluster_order_keys(X: np.ndarray, centers: np.ndarray, labels: np.ndarray):
    """Order clusters by their centroid's projection on the top principal axis
    of the centroids; points are keyed by (cluster rank, own projection)."""
    k, d = centers.shape
    mean = np.array([math.fsum(centers[:, q]) / k for q in range(d)])
    axis = _top_axis(centers - mean)
    rank_of_cluster = np.empty(len(centers), dtype=np.int64)
    rank_of_cluster[np.argsort(_dot_axes(centers, axis), kind="stable")] = np.arange(len(centers))
    return rank_of_cluster[labels], _dot_axes(X, axis), axis, rank_of_cluster


def _morton_keys(X01: np.ndarray, bits: int = 8) -> np.ndarray:
    """Interleaved-bit (Morton) key of points in [0,1]^d, `bits` bits per axis."""
    n, d = X01.shape
    assert d * bits <= 64
    q = np.clip((X01 * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1).astype(np.uint64)
    key = np.zeros(n, dtype=np.uint64)
    for b in range(bits - 1, -1, -1):
        for j in range(d):
            key = (key << np.uint64(1)) | ((q[:, j] >> np.uint64(b)) & np.uint64(1))
    return key


def _clamp_sizes(sizes: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Move boundary points between order-adjacent clusters until every size
    lies in [lo, hi] (total preserved)."""
    sizes = sizes.astype(np.int64).copy()
    for _ in range(4):
        for k in range(len(sizes) - 1):
            if sizes[k] < lo:
                dlt = lo - sizes[k]
                sizes[k] += dlt
                sizes[k + 1] -= dlt
            elif sizes[k] > hi:
                dlt = sizes[k] - hi
                sizes[k] -= dlt
                sizes[k + 1] += dlt
        for k in range(len(sizes) - 1, 0, -1):
            if sizes[k] < lo:
                dlt = lo - sizes[k]
                sizes[k] += dlt
                sizes[k - 1] -= dlt
            elif sizes[k] > hi:
                dlt = sizes[k] - hi
                sizes[k] -= dlt
                sizes[k - 1] += dlt
    assert sizes.sum() > 0 and np.all(sizes >= lo) and np.all(sizes <= hi), sizes
    return sizes


def _ptr_from_sizes(sizes) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(np.asarray(sizes, dtype=np.int64))]).astype(np.int64)


def _test_ptr(block_of_test: np.ndarray, M: int) -> tuple[np.ndarray, np.ndarray]:
    order = np.argsort(block_of_test, kind="stable")
    counts = np.bincount(block_of_test, minlength=M)
    return order, _ptr_from_sizes(counts)


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------

_DEFAULTS = {
    "C1": dict(N=2000, M=16, s=64, B=1, U=500),
    "C2": dict(N=40960, M=64, s=512, B=1, U=4096),
    "C3": dict(N=49152, M=96, s=1024, B=2, U=8192),
    "C4": dict(N=2_000_000, M=2000, s=2048, B=1, U=100_000),
    "C5": dict(N=65536, M=128, s=1024, B=2, U=0),
}

_cache: dict = {}


def make_problem(name: str, N: Optional[int] = None, M: Optional[int] = None,
                 s: Optional[int] = None, B: Optional[int] = None,
                 U: Optional[int] = None, jitter: float = 1e-6, draw: int = 0) -> Problem:
    """Build configuration `name` (C1..C5); keyword overrides shrink it for
    parity tests while keeping its distribution and partition recipe.
    draw > 0 gives another sample of inputs, noise, test points and partition
    of the same configuration (the same target function f)."""
    if name not in _DEFAULTS:
        raise ValueError(f"unknown configuration {name!r}")
    p = dict(_DEFAULTS[name])
    for k, v in dict(N=N, M=M, s=s, B=B, U=U).items():
        if v is not None:
            p[k] = int(v)
    key = (name, p["N"], p["M"], p["s"], p["U"], jitter, int(draw))
    if key in _cache:
        return _cache[key].with_B(p["B"])
    idx = CONFIG_NAMES.index(name)
    rx, rnoise, rrff, rS, rtest, rpart = _streams(1411 + idx)
    if draw:
        rx, rnoise, _, rS, rtest, rpart = _streams(1411 + idx + 100_000 * int(draw))
    Nn, M_, s_, U_ = p["N"], p["M"], p["s"], p["U"]
    if name == "C1":
        d = 2
        X = rx.uniform(0.0, 1.0, (Nn, d))
        XU = rtest.uniform(0.0, 1.0, (U_, d))
        f = lambda x: np.sin(6.0 * x[:, 0]) + np.cos(4.0 * x[:, 1])  # noqa: E731
        sig_noise, ell, sigma_s = 0.1, np.full(d, 0.2), 1.0
        order = np.argsort(X[:, 0], kind="stable")
        X = X[order]
        sizes = np.full(M_, Nn // M_, dtype=np.int64)
        sizes[: Nn % M_] += 1
        block_ptr = _ptr_from_sizes(sizes)
        # test block: the x1 interval between block boundaries
        bounds = [0.5 * (X[block_ptr[k] - 1, 0] + X[block_ptr[k], 0]) for k in range(1, M_)]
        blk = np.searchsorted(np.asarray(bounds), XU[:, 0], side="right").astype(np.int64)
        meta = dict(partition="sorted by x1")
    elif name in ("C2", "C3"):
        d = 5 if name == "C2" else 21
        X = rx.standard_normal((Nn, d))
        XU = rtest.standard_normal((U_, d))
        nf, ellv, sig_noise = (2048, 1.0, 0.05) if name == "C2" else (4096, 3.0, 0.1)
        sigma_s = 1.0
        ell = np.full(d, ellv)
        f = rff_draw(rrff, d, nf, ellv, sigma_s)
        centers, lab = _kmeans(rpart, X, M_)
        crank, proj, axis, rank_of_cluster = _cluster_order_keys(X, centers, lab)
        order = np.lexsort((proj, crank))
        X = X[order]
        crank_s, proj_s = crank[order], proj[order]
        if name == "C2":
            sizes = np.full(M_, Nn // M_, dtype=np.int64)
            sizes[: Nn % M_] += 1
        else:
            lo = max(1, min(256, Nn // M_))
            hi = max(lo, 1024 if Nn // M_ <= 1024 else 2 * (Nn // M_))
            sizes = _clamp_sizes(np.bincount(crank_s, minlength=M_), lo, hi)
        block_ptr = _ptr_from_sizes(sizes)
        # test points: same key (cluster rank, projection) -> position -> block
        tl = _nearest(XU, centers)
        tr, tp = rank_of_cluster[tl], _dot_axes(XU, axis)
        pos = np.empty(U_, dtype=np.int64)
        starts = np.searchsorted(crank_s, np.arange(M_), side="left")
        ends = np.searchsorted(crank_s, np.arange(M_), side="right")
        for i in range(U_):
            a, b = starts[tr[i]], ends[tr[i]]
            pos[i] = a + np.searchsorted(proj_s[a:b], tp[i])
        pos = np.clip(pos, 0, Nn - 1)
        blk = (np.searchsorted(block_ptr, pos, side="right") - 1).astype(np.int64)
        meta = dict(partition="k-means centroid order", rff_features=nf)
    else:  # C4, C5
        d = 8
        X = rx.uniform(0.0, 1.0, (Nn, d))
        XU = rtest.uniform(0.0, 1.0, (U_, d))
        nf, ellv, sig_noise, sigma_s = 4096, 0.3, 0.1, 1.0
        ell = np.full(d, ellv)
        f = rff_draw(rrff, d, nf, ellv, sigma_s)
        mkey = _morton_keys(X)
        order = np.argsort(mkey, kind="stable")
        X, mkey = X[order], mkey[order]
        sizes = np.full(M_, Nn // M_, dtype=np.int64)
        sizes[: Nn % M_] += 1
        block_ptr = _ptr_from_sizes(sizes)
        if U_ > 0:
            pos = np.clip(np.searchsorted(mkey, _morton_keys(XU)), 0, Nn - 1)
            blk = (np.searchsorted(block_ptr, pos, side="right") - 1).astype(np.int64)
        else:
            blk = np.zeros(0, dtype=np.int64)
        meta = dict(partition="Morton order", rff_features=nf)
    y = f(X) + sig_noise * rnoise.standard_normal(Nn)
    yU = f(XU) + sig_noise * rnoise.standard_normal(U_) if U_ > 0 else np.zeros(0)
    torder, test_block_ptr = _test_ptr(blk, M_)
    XU, yU = XU[torder], yU[torder]
    Sidx = np.sort(rS.choice(Nn, size=s_, replace=False))
    prob = Problem(
        name=name, X=np.ascontiguousarray(X), y=y, block_ptr=block_ptr,
        S=np.ascontiguousarray(X[Sidx]), XU=np.ascontiguousarray(XU), yU=yU,
        test_block_ptr=test_block_ptr, log_ell=np.log(ell),
        log_sigma_s=math.log(sigma_s), log_sigma_n=math.log(sig_noise),
        jitter=jitter, mean=0.0, B=p["B"], meta=meta)
    if Nn <= 200_000 or os.environ.get("LMA_SYNTH_CACHE_ALL"):
        _cache[key] = prob
    return prob


def make_replicated(name: str, copies: int, B: Optional[int] = None, first_draw: int = 0, **kw) -> Problem:
    """`copies` draws of configuration `name` (draws first_draw,
    first_draw + 1, ...) joined into one problem: their blocks and test
    blocks are concatenated in draw order and the support set is the first
    draw's.  Every draw has the configuration's size, so a problem split by
    draws into shards keeps the work per shard fixed (weak scaling)."""
    parts = [make_problem(name, B=B, draw=first_draw + k, **kw) for k in range(int(copies))]
    p0 = parts[0]
    if len(parts) == 1:
        return dataclasses.replace(p0, meta=dict(p0.meta, copies=1, first_draw=int(first_draw)))
    off, toff = 0, 0
    ptrs, tptrs = [np.zeros(1, dtype=np.int64)], [np.zeros(1, dtype=np.int64)]
    for q in parts:
        ptrs.append(q.block_ptr[1:] + off)
        tptrs.append(q.test_block_ptr[1:] + toff)
        off += q.N
        toff += q.U
    return dataclasses.replace(
        p0, name=f"{name}x{copies}", X=np.concatenate([q.X for q in parts]), y=np.concatenate([q.y for q in parts]),
        block_ptr=np.concatenate(ptrs), XU=np.concatenate([q.XU for q in parts]),
        yU=np.concatenate([q.yU for q in parts]), test_block_ptr=np.concatenate(tptrs),
        meta=dict(p0.meta, copies=int(copies), first_draw=int(first_draw)))


def make_random_problem(seed: int, sizes, d: int = 2, s: int = 6, B: int = 1,
                        test_sizes=None, ell: float = 0.4, sigma_s: float = 1.0,
                        sigma_n: float = 0.1, jitter: float = 1e-6,
                        mean: float = 0.3, aniso: bool = True) -> Problem:
    """Tiny problem with uneven blocks for exact (dense) checks.  Inputs are
    uniform on [0,1]^d sorted by their first coordinate, outputs a smooth
    function plus noise, length-scales jittered per axis when `aniso`."""
    rx, rn, rs, rt, rh, _ = _streams(10_000 + seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    M = len(sizes)
    N = int(sizes.sum())
    X = rx.uniform(0.0, 1.0, (N, d))
    X = X[np.argsort(X[:, 0], kind="stable")]
    block_ptr = _ptr_from_sizes(sizes)
    if test_sizes is None:
        test_sizes = np.full(M, 2, dtype=np.int64)
    test_sizes = np.asarray(test_sizes, dtype=np.int64)
    # test points lie inside their block's x1 range
    XU = []
    for m in range(M):
        lo = X[block_ptr[m], 0]
        hi = X[block_ptr[m + 1] - 1, 0]
        pts = rt.uniform(0.0, 1.0, (int(test_sizes[m]), d))
        pts[:, 0] = lo + (hi - lo) * pts[:, 0]
        XU.append(pts)
    XU = np.concatenate(XU, axis=0) if len(XU) else np.zeros((0, d))
    g = lambda x: np.sin(5.0 * x[:, 0]) + 0.5 * np.cos(3.0 * x.sum(axis=1))  # noqa: E731
    y = g(X) + sigma_n * rn.standard_normal(N)
    yU = g(XU) + sigma_n * rn.standard_normal(XU.shape[0])
    Sidx = np.sort(rs.choice(N, size=s, replace=False))
    log_ell = np.log(np.full(d, ell))
    if aniso:
        log_ell = log_ell + rh.uniform(-0.3, 0.3, d)
    return Problem(
        name=f"random{seed}", X=X, y=y, block_ptr=block_ptr, S=X[Sidx].copy(),
        XU=XU, yU=yU, test_block_ptr=_ptr_from_sizes(test_sizes), log_ell=log_ell,
        log_sigma_s=math.log(sigma_s), log_sigma_n=math.log(sigma_n),
        jitter=jitter, mean=mean, B=int(B), meta=dict(partition="sorted by x1"))


def make_toy(n_test: int = 201, seed: int = 0) -> Problem:
    """The 1-D toy of Appendix D: 400 inputs on [-5, 5], four blocks of 100
    split at -2.5, 0, 2.5, y = 1 + cos(x) + 0.1 eps, |S| = 16, B = 1, and the
    hyperparameters the appendix prints (l = 1.2270, sigma_n = 0.0939,
    sigma_s = 0.6836, mu = 1.1072).  The test grid is assigned to blocks by
    the same split points."""
    rx, rn, rs, _, _, _ = _streams(20_000 + seed)
    edges = [-5.0, -2.5, 0.0, 2.5, 5.0]
    X = np.concatenate([np.sort(rx.uniform(edges[k], edges[k + 1], 100)) for k in range(4)])[:, None]
    y = 1.0 + np.cos(X[:, 0]) + 0.1 * rn.standard_normal(400)
    block_ptr = np.array([0, 100, 200, 300, 400], dtype=np.int64)
    Sidx = np.sort(rs.choice(400, size=16, replace=False))
    XU = np.linspace(-5.0, 5.0, n_test)[:, None]
    blk = np.searchsorted(np.array(edges[1:4]), XU[:, 0], side="right").astype(np.int64)
    order, tptr = _test_ptr(blk, 4)
    XU = XU[order]
    yU = 1.0 + np.cos(XU[:, 0])
    return Problem(
        name="toy", X=X, y=y, block_ptr=block_ptr, S=X[Sidx].copy(), XU=XU, yU=yU,
        test_block_ptr=tptr, log_ell=np.log(np.array([1.2270])),
        log_sigma_s=math.log(0.6836), log_sigma_n=math.log(0.0939), jitter=1e-6,
        mean=1.1072, B=1, meta=dict(partition="split at -2.5, 0, 2.5"))
