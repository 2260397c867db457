"""The |S| x B trade-off sweep (Remark 3, Fig. 2) on a small C2-shaped
problem: more support points or a higher Markov order do not make the test
RMSE worse (within 3%), every row carries a positive time, and two cells'
RMSE and log-likelihood match the FP64 oracle's for the same (|S|, B)
(RMSE within 0.1 %, the accuracy target; log-likelihood within the mixed
bound of test_gpu_parity.py)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rows():
    import torch
    from paper_1411_4510_gb300 import build, tradeoff
    build.build()
    torch.cuda.set_device(0)
    return tradeoff.sweep("C2", s_values=(32, 128), B_values=(0, 2), repeats=1, N=3200, M=16, U=400)


def test_rows_complete(rows):
    assert {(r["s"], r["B"]) for r in rows} == {(32, 0), (32, 2), (128, 0), (128, 2)}
    assert all(r["ms"] > 0 and r["rmse"] > 0 for r in rows)


@pytest.mark.parametrize("cell", [(32, 0), (128, 2)])
def test_cells_match_oracle(rows, cell):
    import numpy as np
    from oracle import lma_oracle as O2
    from workloads import make_problem
    from _parity import check_scalar
    s, B = cell
    p = make_problem("C2", s=s, B=B, N=3200, M=16, U=400)
    f = O2.fit(p)
    m, _ = O2.predict(f)
    rm_ref = float(np.sqrt(np.mean((m - p.yU) ** 2)))
    row = {(x["s"], x["B"]): x for x in rows}[cell]
    check_scalar(f"tradeoff_s{s}_b{B}", "rmse", row["rmse"], rm_ref, 1e-3)
    check_scalar(f"tradeoff_s{s}_b{B}", "loglik", row["loglik"], f.loglik, 1.5e-4)


def test_more_support_points_or_markov_order_help(rows):
    r = {(x["s"], x["B"]): x["rmse"] for x in rows}
    assert r[(128, 0)] <= 1.03 * r[(32, 0)]
    assert r[(32, 2)] <= 1.03 * r[(32, 0)]
    assert r[(128, 2)] <= 1.03 * r[(128, 0)]
