"""GPU tests of the enqueued prediction (lma_predict_async / lma_model_wait):
it gives the same numbers as lma_predict, several calls can be queued before
one wait, and a host buffer is refused at once."""
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


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_async_equals_sync(L, prec):
    import torch
    from workloads import make_problem
    p = make_problem("C2", N=3200, M=16, s=100, U=400, B=2)
    dev = torch.device("cuda:0")
    args = L.problem_args(p)
    args.update(X=torch.as_tensor(p.X, device=dev), y=torch.as_tensor(p.y, device=dev),
                S=torch.as_tensor(p.S, device=dev))
    model = L.lma_fit(precision=getattr(L, prec), **args)
    XU = torch.as_tensor(p.XU, device=dev).contiguous()
    m_sync, v_sync = L.lma_predict(model, XU, p.test_block_ptr)
    torch.cuda.synchronize()
    outs = [L.lma_predict_async(model, XU, p.test_block_ptr) for _ in range(3)]
    L.lma_model_wait(model)
    rtol = 1e-12 if prec == "FP64" else 1e-6   # the same kernels on the same inputs
    for m, v in outs:
        assert np.allclose(m.cpu().numpy(), m_sync.cpu().numpy(), rtol=rtol, atol=0)
        assert np.allclose(v.cpu().numpy(), v_sync.cpu().numpy(), rtol=rtol, atol=0)


def test_async_refuses_host_buffers(L):
    import torch
    from workloads import make_problem
    p = make_problem("C2", N=1280, M=4, s=40, U=100, B=1)
    model = L.lma_fit(precision=L.FP64, **L.problem_args(p))
    with pytest.raises(ValueError):
        L.lma_predict_async(model, torch.as_tensor(p.XU), p.test_block_ptr)
    # through the C ABI directly: host XU is an argument error, returned at once
    from paper_1411_4510_gb300 import _abi
    lib = _abi.load()
    mean = torch.empty(p.U, dtype=torch.float64, device="cuda:0")
    var = torch.empty(p.U, dtype=torch.float64, device="cuda:0")
    XU = np.ascontiguousarray(p.XU)
    tp = np.ascontiguousarray(p.test_block_ptr.astype(np.int64))
    st = lib.lma_predict_async(model.handle, p.U, XU.ctypes.data, tp.ctypes.data, 1, mean.data_ptr(),
                               var.data_ptr())
    assert st == 1
    L.lma_model_wait(model)
