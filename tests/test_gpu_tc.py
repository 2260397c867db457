"""Tensor-core (tcgen05, 3xTF32) tile product against an FP64 product of the
same FP32 operands.  Bound, relative to sum_k |a_ik||b_jk|: each 3xTF32
product keeps ~22 bits (2^-22 = 2.4e-7; the dropped lo*lo term is 2^-22 too)
and the FP32 accumulation in tensor memory over K terms adds ~K^(1/2) 2^-24
in expectation; the test allows 2^-21 + 4 K^(1/2) 2^-24 (8e-7 + 2.4e-7
K^(1/2)), i.e. 6.2e-6 at K = 512."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1411_4510_gb300 import build
    build.build()
    from paper_1411_4510_gb300 import _abi
    torch.cuda.set_device(0)
    return _abi.load()


@pytest.mark.parametrize("tile_n", [64, 128])
@pytest.mark.parametrize("shape", [(128, 64, 32), (300, 200, 96), (256, 128, 512), (1000, 130, 1024)])
def test_tc_gemm_3xtf32(lib, shape, tile_n):
    import torch
    from paper_1411_4510_gb300 import _abi
    M, N, K = shape
    g = torch.Generator(device="cpu").manual_seed(M * 131 + N * 7 + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float32).cuda()
    B = torch.randn(N, K, generator=g, dtype=torch.float32).cuda()
    Cm = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    _abi.check(lib.lma_tc_gemm_check(M, N, K, A.data_ptr(), K, B.data_ptr(), K, Cm.data_ptr(), N, tile_n, st))
    torch.cuda.synchronize()
    ref = (A.double() @ B.double().T).cpu().numpy()
    scale = (A.abs().double() @ B.abs().double().T).cpu().numpy()
    out = Cm.double().cpu().numpy()
    assert np.all(np.isfinite(out))
    err = np.max(np.abs(out - ref) / scale)
    bound = 2.0 ** -21 + 4.0 * np.sqrt(K) * 2.0 ** -24
    assert err <= bound, (err, bound)
