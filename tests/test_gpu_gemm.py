"""The tcgen05 BF16 GEMM of the learned prolongation against an FP64 matmul of
the same BF16-rounded inputs.  FP32 accumulation of K <= 128 products of
BF16 values: relative error of each output ~ K * 2^-24 of the sum of |terms|.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 16), (1000, 64, 128), (257, 128, 64),
                                   (5, 64, 32), (4096, 128, 128)])
def test_gemm_matches_fp64(mm, M, N, K):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = mm.gemm_bf16(A.cuda(), B.cuda()).cpu().numpy()
    a = A.double().numpy()
    b = B.double().numpy()
    ref = a @ b.T
    bound = 1e-5 * (np.abs(a) @ np.abs(b).T) + 1e-6
    assert np.all(np.abs(C - ref) <= bound)


def test_gemm_bias_relu_bf16(mm):
    g = torch.Generator(device="cpu").manual_seed(5)
    A = torch.randn(300, 128, generator=g).to(torch.bfloat16)
    B = torch.randn(64, 128, generator=g).to(torch.bfloat16)
    bias = torch.randn(64, generator=g)
    C, Cb = mm.gemm_bf16(A.cuda(), B.cuda(), bias=bias.cuda(), relu=True, out_bf16=True)
    ref = np.maximum(A.double().numpy() @ B.double().numpy().T + bias.double().numpy(), 0)
    np.testing.assert_allclose(C.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(Cb.float().cpu().numpy(), ref, rtol=1e-2, atol=1e-2)


@pytest.mark.parametrize("n,R", [(64, 128), (1000, 128), (4099, 16), (30001, 128), (7, 16),
                                 (200000, 128)])
def test_weight_gradient_gemm_matches_fp64(mm, n, R):
    # out = A^T B, contracted over the n rows (the vertices): K = n is split
    # into per-CTA vertex ranges (ragged last chunk, zero rows padding A^T to
    # 128 when R = 16) whose FP32 partials are added in a fixed order.  FP32
    # accumulation of n products: |error| <= n * 2^-23 of the sum of |terms|
    # (bounded here by 2e-7 n relative plus an absolute floor)
    g = torch.Generator(device="cpu").manual_seed(n + R)
    A = torch.randn(n, R, generator=g).to(torch.bfloat16)
    B = torch.randn(n, 64, generator=g).to(torch.bfloat16)
    C = mm.gemm_bf16_tn(A.cuda(), B.cuda()).cpu().numpy()
    a, b = A.double().numpy(), B.double().numpy()
    ref = a.T @ b
    bound = (2e-7 * n + 1e-6) * (np.abs(a).T @ np.abs(b)) + 1e-6
    assert np.all(np.abs(C - ref) <= bound)
    # the result does not depend on the call (fixed-order reduction)
    C2 = mm.gemm_bf16_tn(A.cuda(), B.cuda()).cpu().numpy()
    assert np.array_equal(C, C2)


def test_net_gemm_profile_reports_positive_times(mm):
    f, b = mm.net_gemm_profile(1 << 16, reps=3)
    assert f > 0 and b > 0


def test_gemm_rejects_unsupported_k(mm):
    # K is one of 16, 32, 64, 128 (the layer widths); anything else is an
    # argument error, not a launch
    A = torch.zeros(256, 48, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(64, 48, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(mm.MMError):
        mm.gemm_bf16(A, B)
