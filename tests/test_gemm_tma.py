"""The tensor-copy-fed tcgen05 GEMM (bf16 operands in memory, float32
accumulation): C = A B^T against float64 products of the same bf16 values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 512, 192), (384, 768, 640), (1024, 1024, 1024),
                                   (2048, 256, 4096)])
def test_gemm_tma_matches_float64_products(lib, M, N, K):
    import torch
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    A = torch.randn((M, K), generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), generator=g).to(torch.bfloat16)
    ref = A.double().numpy() @ B.double().numpy().T
    Cd = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    lib.gemm_bf16_tma(A.cuda(), B.cuda(), Cd)
    lib.gemm_synchronize()
    got = Cd.cpu().numpy().astype(np.float64)
    # float32 accumulation of K exact bf16 products: error ~ sqrt(K) u |A||B|
    err = np.max(np.abs(got - ref)) / np.sqrt(K)
    assert np.all(np.isfinite(got))
    assert err <= 5e-5, err


def test_gemm_tma_rejects_unsupported_shapes(lib):
    import torch
    A = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((256, 64), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((128, 256), dtype=torch.float32, device="cuda")
    L = lib.lib()
    import ctypes as Ct
    assert L.psatd_gemm_bf16_tma(100, 256, 64, Ct.c_void_p(A.data_ptr()), Ct.c_void_p(B.data_ptr()),
                                 Ct.c_void_p(C.data_ptr()), None) == lib.ERR_ARG
    assert L.psatd_gemm_bf16_tma(128, 256, 60, Ct.c_void_p(A.data_ptr()), Ct.c_void_p(B.data_ptr()),
                                 Ct.c_void_p(C.data_ptr()), None) == lib.ERR_ARG
    assert L.psatd_gemm_bf16_tma(128, 256, 64, None, Ct.c_void_p(B.data_ptr()),
                                 Ct.c_void_p(C.data_ptr()), None) == lib.ERR_ARG
