"""FP64-class complex GEMM on the bf16 tensor cores (exact slicing into 7-bit digits)
against the FP64 product computed on the host.

Error model: each operand entry is truncated to 56 bits below its row (A) or
column (B) maximum and digit products of weight above 9 are dropped (each
below 2^-53 of the largest product), so
|C - C_exact|_ij <= c K 2^-52 max_k|A_ik| max_k|B_kj| with c small; the test
allows c = 8 and reports the worst ratio (native FP64 meets the same bar)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02930_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def ctx(api):
    return api.ctx_create(0)


def crand(rng, *shape, spread=0.0):
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if spread:
        a *= np.exp(spread * rng.standard_normal(shape[0]))[:, None]
    return a


@pytest.mark.parametrize("M,N,K,tA,tB,cA,cB", [
    (8, 8, 8, False, False, False, False),
    (128, 32, 64, False, False, False, False),
    (100, 70, 300, True, False, True, False),
    (33, 129, 77, False, True, False, True),
    (1280, 1024, 256, False, False, False, False),
    (1024, 256, 1280, False, False, False, False),
    (256, 256, 512, True, True, True, True),
])
def test_emulated_zgemm_matches_fp64(api, ctx, M, N, K, tA, tB, cA, cB):
    import torch
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = crand(rng, *((K, M) if tA else (M, K)), spread=2.0)
    B = crand(rng, *((N, K) if tB else (K, N)))
    opA = A.T if tA else A
    opB = B.T if tB else B
    if cA:
        opA = opA.conj()
    if cB:
        opB = opB.conj()
    exact = opA @ opB
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    for mode in (0, 1):
        Cd = torch.full((M, N), complex("nan"), dtype=torch.complex128, device="cuda")
        api.k_zgemm(ctx, Ad, Bd, Cd, mode=mode, conjA=cA, conjB=cB, transA=tA, transB=tB)
        got = Cd.cpu().numpy()
        rowmax = np.maximum(np.abs(opA.real), np.abs(opA.imag)).max(axis=1)
        colmax = np.maximum(np.abs(opB.real), np.abs(opB.imag)).max(axis=0)
        bound = 2 * K * 2.0 ** -52 * rowmax[:, None] * colmax[None, :]
        ratio = (np.abs(got - exact) / bound).max()
        print(f"mode {mode} M={M} N={N} K={K}: worst error / (2K 2^-52 rowmax colmax) = {ratio:.3g}")
        assert np.isfinite(got).all()
        assert ratio <= 8.0


def test_emulated_zgemm_alpha_beta(api, ctx):
    import torch
    rng = np.random.default_rng(5)
    A, B, C0 = crand(rng, 40, 50), crand(rng, 50, 60), crand(rng, 40, 60)
    want = (0.3 - 0.7j) * (A @ B) + (1.5 + 0.25j) * C0
    Cd = torch.from_numpy(C0.copy()).cuda()
    api.k_zgemm(ctx, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, mode=1,
                alpha=0.3 - 0.7j, beta=1.5 + 0.25j)
    assert np.abs(Cd.cpu().numpy() - want).max() < 1e-12 * np.abs(want).max()
