"""tcgen05 building blocks (shared-memory descriptors, instruction descriptor, TMEM
accumulator, MMA completion): a BF16 GEMM through the library's tensor-core probe against
an FP32 matmul of the same BF16 values."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02322_gb300 import api, build

    build.build()
    L = api.lib()
    L.mqct_probe_tc_gemm.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.mqct_probe_tc_gemm.restype = C.c_int
    return api


@pytest.mark.parametrize("n,k", [(16, 16), (32, 64), (48, 32), (128, 128), (256, 256)])
def test_tc_gemm_probe(mq, n, k):
    import torch

    g = torch.Generator().manual_seed(n * 1000 + k)
    a = torch.randn(128, k, generator=g).to(torch.bfloat16).cuda()
    b = torch.randn(n, k, generator=g).to(torch.bfloat16).cuda()
    d = torch.full((128, n), float("nan"), dtype=torch.float32, device="cuda")
    st = mq.lib().mqct_probe_tc_gemm(n, k, a.data_ptr(), b.data_ptr(), d.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert st == mq.OK, mq.lib().mqct_last_error()
    ref = (a.double() @ b.double().T).float()
    err = (d - ref).abs().max().item()
    assert err < 1e-4 * max(1.0, ref.abs().max().item()), err
