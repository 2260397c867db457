"""The fit workspace kept between calls (lma_workspace_release): consecutive
fits that reuse it give identical results, releasing it returns its device
memory, and a fit after the release allocates it again and still agrees."""
import numpy as np
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


def test_workspace_reuse_and_release(L):
    import torch
    from workloads import make_problem
    p = make_problem("C2", B=1)   # N = 40,960, |S| = 512: K_SD planes 3 x 40,960 x 512 bfloat16 = 126 MB
    dev = torch.device("cuda:0")
    args = L.problem_args(p)
    args.update(X=torch.as_tensor(p.X, device=dev), y=torch.as_tensor(p.y, device=dev),
                S=torch.as_tensor(p.S, device=dev))
    XU = torch.as_tensor(p.XU, device=dev)

    def run():
        m, v = L.lma_fit_predict(XU=XU, test_block_ptr=p.test_block_ptr, precision=L.MIXED, **args)
        torch.cuda.synchronize()
        return m.cpu().numpy(), v.cpu().numpy()

    m1, v1 = run()
    m2, v2 = run()                      # the same workspace again
    assert np.array_equal(m1, m2) and np.array_equal(v1, v2)
    free0, _ = torch.cuda.mem_get_info()
    L.lma_workspace_release()
    free1, _ = torch.cuda.mem_get_info()
    expect = 3 * p.X.shape[0] * 512 * 2
    assert free1 - free0 >= 0.9 * expect, (free0, free1, expect)
    L.lma_workspace_release()           # nothing held: a no-op
    m3, v3 = run()                      # allocated again
    assert np.array_equal(m1, m3) and np.array_equal(v1, v3)
