"""The tcgen05 tensor-core update kernel (C <- C - A B, FP32 data, 3xTF32) against an
FP64 product of the same FP32 inputs.

Bar: 3xTF32 drops only the lo*lo term and keeps FP32 accumulation, so each product term
carries ~2^-21 relative error and the K-term sum ~K*2^-24; we require
max|C_gpu - C_ref| <= 8 * K * 2^-21 * max(|A| |B|)_row-col sums, stated in the test.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_5522_gb300 import build
    build.build()


def colmajor(x):
    return x.t().contiguous().t()


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (256, 384, 256), (300, 200, 96), (77, 45, 64),
                                   (1000, 520, 128)])
def test_gemm_sub_matches_fp64(M, N, K):
    from paper_1401_5522_gb300 import luqr
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = colmajor(torch.randn(M, K, device="cuda", generator=g))
    B = colmajor(torch.randn(K, N, device="cuda", generator=g))
    C = colmajor(torch.randn(M, N, device="cuda", generator=g))
    ref = C.double() - A.double() @ B.double()
    st = torch.zeros(8, dtype=torch.int32, device="cuda")
    luqr.gemm_sub_f32(C, A, B, status=st)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    scale = (A.double().abs() @ B.double().abs()).max().item()
    err = (C.double() - ref).abs().max().item()
    assert err <= 8 * K * 2.0 ** -21 * scale / K + 4 * 2.0 ** -24 * scale, (err, scale)


def test_gemm_sub_leading_dimensions():
    from paper_1401_5522_gb300 import luqr
    big = colmajor(torch.randn(512, 512, device="cuda"))
    A = big[10:300, 0:64]
    B = big[100:164, 200:450]
    C0 = colmajor(torch.randn(400, 400, device="cuda"))
    C = C0[50:340, 20:270]
    ref = C.double() - A.double() @ B.double()
    outside = C0.clone()
    luqr.gemm_sub_f32(C, A, B)
    torch.cuda.synchronize()
    assert (C.double() - ref).abs().max().item() < 1e-4
    mask = torch.ones_like(C0, dtype=torch.bool)
    mask[50:340, 20:270] = False
    assert torch.equal(C0[mask], outside[mask])      # nothing written outside C
