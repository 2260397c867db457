"""GPU parity of every launch shape the autotuner can choose for the FP64
factorisations of Sigma_SS and I + A (Definition 2, Theorem 2's global
summary): one launch per column panel, two launches per panel, one
cooperative launch with 1, 2 or 4 CTAs per SM (grid barriers), and the
dataflow form (one cooperative launch, per-tile flags).  Each shape is pinned with
lma_autotune_pin and the FP64 fit + prediction compared with the oracle at
1e-9 relative, norm-wise and element-wise.

Support sets of 40 (3 column panels of 16, ragged), 100 and 512 (32 panels,
with 512 identity rows appended) cover one-panel tails, ragged pads and the
longest barrier chain of the configurations.
"""
import pytest

from _parity import Collector

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9
VARIANTS = [0, 1, 2, 3, 4, 5]


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1411_4510_gb300 import build
    build.build()
    import paper_1411_4510_gb300 as L
    torch.cuda.set_device(0)
    yield L
    L.lma_autotune_pin(None)


def _problems():
    from workloads import make_problem, make_random_problem
    return {
        "s40": make_random_problem(0, (70, 90, 65, 80, 75), d=3, s=40, B=1, test_sizes=(9, 0, 12, 7, 10)),
        "s100": make_problem("C2", N=3200, M=16, s=100, U=400, B=2),
        "s512": make_problem("C2", N=6400, M=10, s=512, U=300, B=1),
    }


@pytest.fixture(scope="module")
def cases():
    from oracle import lma_oracle as O2
    out = {}
    for name, p in _problems().items():
        f = O2.fit(p)
        m, v = O2.predict(f)
        out[name] = (p, f.loglik, m, v)
    return out


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("name", ["s40", "s100", "s512"])
def test_fp64_factorisation_shapes_match_oracle(L, cases, name, variant):
    import torch
    p, ll, m, v = cases[name]
    L.lma_autotune_pin(None)
    L.lma_autotune_pin("fp64 factor", variant)
    dev = torch.device("cuda:0")
    args = L.problem_args(p)
    args.update(X=torch.as_tensor(p.X, device=dev), y=torch.as_tensor(p.y, device=dev),
                S=torch.as_tensor(p.S, device=dev))
    model = L.lma_fit(precision=L.FP64, **args)
    mean, var = L.lma_predict(model, torch.as_tensor(p.XU, device=dev), p.test_block_ptr)
    summ = L.lma_model_summary(model)
    L.lma_autotune_pin(None)
    test = f"fp64_shape_{name}_v{variant}"
    c = Collector()
    c.check_scalar(test, "loglik", summ["loglik"], ll, TOL_FP64)
    c.check(test, "mean", mean.cpu().numpy(), m, TOL_FP64, TOL_FP64)
    c.check(test, "var", var.cpu().numpy(), v, TOL_FP64, TOL_FP64, positive=True)
    c.done()

