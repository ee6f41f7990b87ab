"""The tcgen05 tensor-core GEMM against the exact product of the same bf16
inputs.  bf16 x bf16 products are exact in fp32, so the only error is the fp32
accumulation of K terms: |C - C_exact| <= K * 2^-23 * (|A| |B|^T) elementwise,
checked for tile-aligned and ragged shapes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02930_gb300 import api as a
    return a


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 64, 16), (256, 256, 512), (300, 200, 136),
                                   (1, 1, 8), (77, 130, 1000), (2560, 1024, 512), (1024, 256, 2560)])
@pytest.mark.parametrize("k_tile", [64, 32])
def test_tc_gemm_bf16(api, M, N, K, k_tile):
    import torch
    ctx = api.ctx_create(0)
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    Cm = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    api.k_gemm_bf16(ctx, A, B, Cm, k_tile)
    a = A.double().cpu()
    b = B.double().cpu()
    exact = (a @ b.T).numpy()
    bound = K * 2.0 ** -23 * (a.abs() @ b.abs().T).numpy() + 1e-30
    got = Cm.cpu().double().numpy()
    assert np.isfinite(got).all()
    assert (np.abs(got - exact) <= bound).all()
