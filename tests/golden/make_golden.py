"""Writes the full-size expected values of the GPU parity tests
(tests/golden/<case>.json) from the FP64 oracle — test infrastructure only.

Every value here comes from `oracle/` (the summary-form FP64 LMA, O2) on the
seeded synthetic workloads of `workloads/`; nothing comes from the CUDA path.
The workloads are rebuilt bit-identically on any machine (numpy PCG64 draws,
platform-exact partitions); only the outputs y may differ in the last bit
between machines (the random-Fourier-feature cosines), which moves every
value below by ~1e-15 relative.  Each file therefore records fingerprints
of the inputs, which the tests check before comparing.

Cases (full configuration sizes):
  c2_b1, c2_b2  C2 (N=40,960, |S|=512, 64 k-means blocks of 640) at B=1, 2:
                fit (Definitions 1-2), log-likelihood, the local-route
                predictions of every test point, and the RMSE.
  c3            C3 (N=49,152, |S|=1,024, 96 uneven k-means blocks, B=2): fit,
                log-likelihood, predictions of the sampled test blocks.
  c4            C4 (N=2,000,000, |S|=2,048, 2,000 Morton blocks, B=1): fit,
                log-likelihood, global-summary probes, predictions of the
                sampled test blocks (first two, middle, last two).
  c5            C5 (N=65,536, |S|=1,024, 128 Morton blocks, B=2): log-likelihood,
                the oracle's hand-adjoint gradient and central differences
                (h = 1e-4 in log space) of the oracle log-likelihood for
                three components.
  learn         maximum-likelihood hyperparameters (Sec. 5) of a small
                C2-shaped problem (N=1,200, |S|=40, 8 blocks, B=1): L-BFGS-B
                (scipy) on the oracle's log-likelihood and hand adjoint, from
                a start away from the generating values.

Usage: python tests/golden/make_golden.py c2_b1 c2_b2 c3 c4 c5
(about 2.5 hours on 8 cores, C4 taking most of it).
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lma_oracle as O2  # noqa: E402
from workloads import make_problem  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def fingerprints(p) -> dict:
    """Exact fingerprints of the inputs (X, S, XU, both partitions) and the
    exactly rounded sum of y (compared with a relative tolerance)."""
    h = lambda a: hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:32]  # noqa: E731
    return {"X_sha": h(p.X), "S_sha": h(p.S), "XU_sha": h(p.XU),
            "block_ptr_sha": h(p.block_ptr.astype(np.int64)),
            "test_block_ptr_sha": h(p.test_block_ptr.astype(np.int64)),
            "y_fsum": math.fsum(p.y), "yU_fsum": math.fsum(p.yU),
            "N": p.N, "d": p.d, "M": p.M, "s": p.s, "U": p.U, "B": p.B, "jitter": p.jitter}


def sampled_blocks(p) -> list[int]:
    """First two, a middle one and the last two non-empty test blocks."""
    nz = [n for n in range(p.M) if p.test_block_ptr[n + 1] > p.test_block_ptr[n]]
    pick = [nz[0], nz[1], nz[len(nz) // 2], nz[-2], nz[-1]]
    return sorted(set(pick))


def fit_record(f) -> dict:
    """Log-likelihood pieces and a few global-summary entries (whitened support
    coordinates: A = L_SS^-1 (Sigma-ddot_SS - Sigma_SS) L_SS^-T, y-ddot = L_SS^-1 y-ddot_S)."""
    w = np.linalg.solve(f.Lc, f.ydd_white)
    return {"loglik": f.loglik, "quad": f.quad, "logdet_R": f.logdet_R,
            "logdet_C": 2.0 * float(np.sum(np.log(np.diag(f.Lc)))), "wCw": float(w @ w),
            "ydd_head": f.ydd_white[:16].tolist(), "A_diag_head": np.diag(f.A_white)[:16].tolist(),
            "A_trace": float(np.trace(f.A_white)), "ydd_norm": float(np.linalg.norm(f.ydd_white))}


def pred_case(name: str, B: int, full_predict: bool) -> dict:
    p = make_problem(name, B=B)
    t0 = time.time()
    f = O2.fit(p)
    t_fit = time.time() - t0
    rec = {"case": f"{name} B={B}", "fingerprints": fingerprints(p), "fit": fit_record(f), "noisy": True}
    blocks = sampled_blocks(p)
    rec["sampled_blocks"] = blocks
    t0 = time.time()
    if full_predict:
        mean, var = O2.predict(f)
        rec["rmse_all"] = float(np.sqrt(np.mean((mean - p.yU) ** 2)))
    else:
        mean, var = O2.predict(f, blocks=blocks)
    t_pred = time.time() - t0
    idx = np.concatenate([np.arange(p.test_block_ptr[n], p.test_block_ptr[n + 1]) for n in blocks])
    rec["sample_rows"] = idx.tolist()
    rec["mean"] = mean[idx].tolist()
    rec["var"] = var[idx].tolist()
    rec["rmse_sample"] = float(np.sqrt(np.mean((mean[idx] - p.yU[idx]) ** 2)))
    rec["oracle_seconds"] = {"fit": t_fit, "predict": t_pred}
    return rec


def grad_case() -> dict:
    p = make_problem("C5")
    t0 = time.time()
    ll, g = O2.loglik_grad(p)
    t_grad = time.time() - t0
    h = 1e-4
    fd = {}
    d = p.d
    comps = [0, d, d + 1]  # log l_1, log sigma_s, log sigma_n
    for k in comps:
        vals = []
        for sgn in (+1.0, -1.0):
            q = dataclasses.replace(p, log_ell=p.log_ell.copy())
            if k < d:
                q.log_ell[k] += sgn * h
            elif k == d:
                q.log_sigma_s += sgn * h
            else:
                q.log_sigma_n += sgn * h
            vals.append(O2.loglik(q))
        fd[str(k)] = (vals[0] - vals[1]) / (2.0 * h)
    return {"case": "C5 B=2", "fingerprints": fingerprints(p), "loglik": ll, "grad": g.tolist(),
            "fd_h": h, "fd": fd, "oracle_seconds": {"loglik_grad": t_grad}}


def learn_case() -> dict:
    from scipy.optimize import minimize
    p = make_problem("C2", N=1200, M=8, s=40, U=0, B=1)
    d = p.d
    gen = np.concatenate([p.log_ell, [p.log_sigma_s, p.log_sigma_n]])
    th0 = gen + np.concatenate([np.full(d, 0.4), [-0.3, 0.5]])
    evals = []

    def at(th):
        return dataclasses.replace(p, log_ell=np.array(th[:d]), log_sigma_s=float(th[d]),
                                   log_sigma_n=float(th[d + 1]))

    def objective(th):
        ll, g = O2.loglik_grad(at(th))
        evals.append(ll)
        return -ll / p.N, -np.asarray(g) / p.N

    t0 = time.time()
    res = minimize(objective, th0, jac=True, method="L-BFGS-B", options=dict(maxiter=200, gtol=1e-7))
    ll, g = O2.loglik_grad(at(res.x))
    return {"case": "learning, C2 recipe N=1200 M=8 s=40 B=1", "fingerprints": fingerprints(p),
            "theta0": th0.tolist(), "theta_generating": gen.tolist(), "theta": np.asarray(res.x).tolist(),
            "loglik": ll, "grad": np.asarray(g).tolist(), "loglik0": evals[0], "iterations": int(res.nit),
            "evaluations": int(res.nfev), "converged": bool(res.success), "optimizer": "scipy L-BFGS-B, "
            "objective -loglik/N, gtol 1e-7", "oracle_seconds": time.time() - t0}


CASES = {
    "c2_b1": lambda: pred_case("C2", 1, True),
    "c2_b2": lambda: pred_case("C2", 2, True),
    "c3": lambda: pred_case("C3", 2, False),
    "c4": lambda: pred_case("C4", 1, False),
    "c5": grad_case,
    "learn": learn_case,
}


def main(argv):
    for name in argv or list(CASES):
        t0 = time.time()
        rec = CASES[name]()
        rec["written_by"] = "tests/golden/make_golden.py (oracle/ only)"
        with open(os.path.join(HERE, f"{name}.json"), "w") as fh:
            json.dump(rec, fh, indent=1)
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
