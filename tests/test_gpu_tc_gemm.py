"""The tcgen05 GEMM behind the mixed-precision GAP products, through its diagnostic C-ABI
entry point: C = A B^T with FP16 operands against an FP32 product of the same operands.
Shapes span several 128-row tiles, ragged row counts and K from one to many 64-blocks."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def model():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_02142_gb300 import build
    build.build()
    from paper_1905_02142_gb300.api import SoapGap
    return SoapGap(r_cut=4.0, n_max=4, l_max=2, precision="mixed")


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (300, 200, 128), (129, 257, 192), (300, 256, 128),
                                   (1000, 640, 1920), (64, 130, 4096), (20000, 1024, 192)])
def test_tc_gemm_matches_fp32_product(model, m, n, k):
    g = torch.Generator(device="cuda").manual_seed(m * 7 + n * 3 + k)
    a = torch.randn(m, k, device="cuda", generator=g).half()
    b = torch.randn(n, k, device="cuda", generator=g).half()
    c = torch.full((m, n), float("nan"), device="cuda")
    rc = model.lib.soapgap_tc_gemm_f16(model.h, a.data_ptr(), m, b.data_ptr(), n, k, c.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert rc == 0, model.lib.soapgap_last_error(model.h)
    ref = a.double() @ b.double().T
    err = (c.double() - ref).abs().max().item() / ref.abs().max().item()
    # FP16 x FP16 products are exact in FP32; the bound is that of FP32 summation over K
    assert err < k * 2.0 ** -24, err
