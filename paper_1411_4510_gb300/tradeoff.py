"""Accuracy-versus-time trade-off of the support-set size |S| and the Markov
order B (Remark 3, Fig. 2 of the paper): LMA spends its budget either on the
low-rank part (|S|) or on the Markov part (B).  For each (|S|, B) this fits
and predicts a synthetic configuration with the CUDA library and reports the
test RMSE against the held-out noisy outputs, the log-likelihood and the
CUDA-event time of lma_fit_predict (median of `repeats`, after one warm-up).

    python -m paper_1411_4510_gb300.tradeoff --config C2 --s 128 256 512 1024 --B 0 1 2 3

prints one JSON object per line.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np

from . import api


def run_point(p, precision=api.MIXED, repeats: int = 3) -> dict:
    """Fit+predict one problem on the current CUDA device; returns the row."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    args = api.problem_args(p)
    d = {k: (torch.as_tensor(v, device=dev) if k in ("X", "y", "S") else v) for k, v in args.items()}
    XU = torch.as_tensor(p.XU, device=dev)
    st = torch.cuda.current_stream()
    out = None
    times = []
    for it in range(repeats + 1):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        out = api.lma_fit_predict(XU=XU, test_block_ptr=p.test_block_ptr, precision=precision, keep_model=True, **d)
        b.record(st)
        torch.cuda.synchronize()
        if it:
            times.append(a.elapsed_time(b))
    mean, _, model = out
    m = mean.cpu().numpy()
    return dict(s=p.s, B=p.B, N=p.N, M=p.M, U=p.U, rmse=float(np.sqrt(np.mean((m - p.yU) ** 2))),
                loglik=api.lma_model_loglik(model), ms=statistics.median(times))


def sweep(config: str = "C2", s_values=(128, 256, 512), B_values=(0, 1, 2), precision=api.MIXED, repeats: int = 3,
          **sizes) -> list:
    from workloads import make_problem
    rows = []
    for s in s_values:
        for B in B_values:
            p = make_problem(config, s=int(s), B=int(B), **sizes)
            rows.append(run_point(p, precision, repeats))
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--config", default="C2")
    ap.add_argument("--s", type=int, nargs="+", default=[128, 256, 512, 1024])
    ap.add_argument("--B", type=int, nargs="+", default=[0, 1, 2, 3])
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--M", type=int, default=None)
    ap.add_argument("--U", type=int, default=None)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--repeats", type=int, default=3)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    sizes = {k: v for k, v in dict(N=a.N, M=a.M, U=a.U).items() if v is not None}
    for row in sweep(a.config, a.s, a.B, api.FP64 if a.fp64 else api.MIXED, a.repeats, **sizes):
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
