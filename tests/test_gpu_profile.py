"""Launch profiler: the per-launch trace agrees with the per-kernel totals,
and the traced launches are the ones the launch counter saw."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1411_4510_gb300 import build
    build.build()
    import paper_1411_4510_gb300 as L
    torch.cuda.set_device(0)
    return L


def test_trace_matches_totals(L):
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=1)
    args = L.problem_args(p)
    L.lma_fit_predict(XU=p.XU, test_block_ptr=p.test_block_ptr, precision=L.MIXED, **args)  # warm-up
    n0 = L.lma_kernel_launch_count()
    L.profile_start("")
    L.lma_fit_predict(XU=p.XU, test_block_ptr=p.test_block_ptr, precision=L.MIXED, **args)
    trace = L.profile_trace()
    tot = L.profile_stop()
    assert len(trace) == L.lma_kernel_launch_count() - n0
    assert trace[0][1] == 0.0
    for name, t0, t1 in trace:
        assert 0.0 <= t0 <= t1
    assert {nm for nm, _, _ in trace} == set(tot)
    for nm, (ms, cnt) in tot.items():
        mine = [(t0, t1) for n, t0, t1 in trace if n == nm]
        assert len(mine) == cnt
        assert sum(b - a for a, b in mine) == pytest.approx(ms, rel=1e-3, abs=1e-3)
    # the launch order is the library's: the support-set factor comes first
    assert trace[0][0] in ("k_scale", "k_build_kss")
