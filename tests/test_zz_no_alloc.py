"""lma_global_step_noalloc, the allocation-free global step.

It is meant for callers that cannot allocate device memory on their call
path (a runtime that pre-provisions all device memory and forbids allocation
while serving a request, or a caller whose device memory belongs to another
allocator).  Its results must match those of the global step that lma_fit
runs (reported by lma_model_summary) within the FP64 tolerance the other
tests use, on three calls in a row: the library-held scratch array keeps the
previous call's contents, so the second call checks that nothing stale
leaks into it.  Around each call the test also checks the property the entry
point exists for: the device's stream-ordered memory pool (which the other
entry points allocate from) sees no new use, and the free device memory does
not change.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-9


class _Pool:
    """High-water mark of the used memory of device 0's default stream-ordered
    memory pool, through the CUDA driver API (CU_MEMPOOL_ATTR_USED_MEM_CURRENT
    = 7, CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8; setting the high mark resets it
    to the current use)."""

    def __init__(self):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int(0)
        assert self.cu.cuDeviceGet(C.byref(dev), 0) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = C.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, 8, C.byref(z)) == 0
        return self._get(7)

    def high(self):
        return self._get(8)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1411_4510_gb300 import build
    build.build()
    import paper_1411_4510_gb300 as L
    from paper_1411_4510_gb300 import _abi
    torch.cuda.set_device(0)
    return L, _abi, _abi.load()


@pytest.mark.parametrize("prec,shape", [("FP64", (3200, 16, 100)), ("MIXED", (10240, 16, 512))])
def test_noalloc_global_step_matches_fit(env, prec, shape):
    import torch
    from workloads import make_problem
    L, abi, lib = env
    N, M, s = shape
    p = make_problem("C2", N=N, M=M, s=s, U=64, B=1)
    model = L.lma_fit(precision=getattr(L, prec), **L.problem_args(p))
    summ = L.lma_model_summary(model)
    A = torch.as_tensor(summ["A"], device="cuda").contiguous()
    yv = torch.as_tensor(summ["y"], device="cuda").contiguous()
    beta_ref = np.linalg.solve(np.eye(s) + summ["A"], summ["y"])
    st = torch.cuda.current_stream().cuda_stream
    pool = _Pool()
    beta = torch.empty((s,), dtype=torch.float64, device="cuda")
    sc = torch.empty((3,), dtype=torch.float64, device="cuda")
    for call in range(3):
        beta.fill_(float("nan"))
        sc.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        used0 = pool.reset_high()
        abi.check(lib.lma_global_step_noalloc(s, p.N, A.data_ptr(), yv.data_ptr(), summ["quad"], summ["logdet_R"],
                                              beta.data_ptr(), sc.data_ptr(), st))
        torch.cuda.synchronize()
        assert pool.high() == used0, "the allocation-free global step used the stream-ordered pool"
        if call > 0:  # the first call may still load the entry point's kernels (lazy module loading)
            assert torch.cuda.mem_get_info()[0] == free0, "device memory changed across the allocation-free call"
        out = sc.cpu().numpy()
        b = beta.cpu().numpy()
        assert abs(out[1] - summ["logdet_C"]) <= TOL * abs(summ["logdet_C"])
        assert abs(out[2] - summ["loglik"]) <= TOL * abs(summ["loglik"])
        assert np.linalg.norm(b - beta_ref) <= TOL * np.linalg.norm(beta_ref)


def test_noalloc_rejects_oversize(env):
    L, abi, lib = env
    null = C.c_void_p(16)
    st = lib.lma_global_step_noalloc(1025, 10, null, null, 1.0, 0.0, null, null, None)
    assert st == abi.LMA_ERR_INVALID_ARG
    blk = C.c_int64(0)
    msg = C.c_char_p()
    lib.lma_last_error_info(C.byref(blk), C.byref(msg))
    assert b"1024" in msg.value
