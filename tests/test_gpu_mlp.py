"""Tensor-core MLP kernels against the float64 reference (oracle/mlp.py).

The GEMM is checked against a float64 product of the same bfloat16 values
(FP32 accumulation: relative error well below 1e-4); the forward pass of the
model against the float64 forward to 1e-2 relative (BF16 operands); the
backward pass against the float64 gradients, which are themselves pinned to
finite differences in tests/test_mlp_oracle.py.
"""
import numpy as np
import pytest

from paper_2507_17087_gb300 import native as N

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N_,K", [(128, 64, 64), (128, 256, 64), (256, 256, 256), (384, 128, 192),
                                    (1024, 256, 4096), (128, 64, 1024)])
def test_gemm_bf16_against_float64(M, N_, K):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N_ * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N_, K, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N_), float("nan"), dtype=torch.float32, device="cuda")
    N.gemm_bf16(A, B, C)
    ref = A.double() @ B.double().T
    err = (C.double() - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= 1e-5 * scale * max(1.0, K / 256), (err, scale)
