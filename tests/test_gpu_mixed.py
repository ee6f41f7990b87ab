"""The mixed-precision mode (reading c13 of the local solve): the persistent
low-precision tensor-core GEMM, the bf16/tf32 two-site H_eff built on it, the
refined local solve, and whole steps against the oracle with converged local
solves.

Bars.  The GEMM's products of bf16 (or tf32) values are exact in fp32 and
only the fp32 accumulation rounds: error <= K 2^-24 sum|a||b| per entry.  The
low-precision H_eff rounds L, X, the mixed intermediate and R to the operand
precision u (2^-8 bf16, 2^-11 tf32), so its error against the FP64 product is
a few u relative to the norms; the test allows 8u.  Refinement uses an
FP64-class residual, so converged local solves and whole steps meet FP64-class
bars: solutions to 1e-9 relative, step energies to 1e-8 relative (the mixed
mode's target) against the oracle run with local GMRES converged to 1e-12."""
import numpy as np
import pytest

from oracle import linsolve as ls, mpo as ompo, mps as omps, step as ostep
from paper_2606_02930_gb300 import inputs

pytestmark = pytest.mark.gpu

U = {"mixed_bf16": 2.0 ** -8, "mixed_tf32": 2.0 ** -11}


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02930_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def ctx(api):
    return api.ctx_create(0)


@pytest.mark.parametrize("pair", [False, True])
@pytest.mark.parametrize("tf32", [False, True])
@pytest.mark.parametrize("M,N,K,batch,bn,splits", [(128, 256, 64, 1, 256, 1),
                                                    (300, 520, 200, 3, 256, 1),
                                                    (257, 130, 1000, 2, 128, 3),
                                                    (200, 400, 296, 2, 192, 2),
                                                    (1024, 2048, 1024, 1, 256, 2)])
def test_lp_gemm_matches_exact_products(api, ctx, tf32, M, N, K, batch, bn, splits, pair):
    # pair: 256-row tiles computed by a pair of CTAs sharing each MMA
    import torch
    g = torch.Generator().manual_seed(M * 7 + N + K)
    dt = torch.float32 if tf32 else torch.bfloat16
    A = torch.randn(batch, M, K, generator=g).to(dt)
    B = torch.randn(N, K, generator=g).to(dt)
    if tf32:
        # values representable in tf32 (10 explicit mantissa bits), so that
        # the products the tensor core forms are exact
        A = (A.view(torch.int32) & ~0x1FFF).view(torch.float32)
        B = (B.view(torch.int32) & ~0x1FFF).view(torch.float32)
    Cd = torch.full((splits, batch, M, N), float("nan"), dtype=torch.float32, device="cuda")
    api.k_gemm_lp(ctx, A.cuda(), B.cuda(), Cd, bn=bn, splits=splits, pair=pair)
    got = Cd.double().sum(0).cpu()
    want = torch.einsum("bmk,nk->bmn", A.double(), B.double())
    bound = K * 2.0 ** -24 * torch.einsum("bmk,nk->bmn", A.double().abs(), B.double().abs())
    assert torch.all((got - want).abs() <= bound + 1e-30)


def _heff_case(rng, Ws, i, chlB, chlK, chrK, chrB):
    from tests.gpu_util import crandn
    D0, D2, d = Ws[i].shape[0], Ws[i + 1].shape[3], Ws[i].shape[1]
    L = crandn(rng, chlB, D0, chlK) / np.sqrt(chlK)
    R = crandn(rng, chrB, D2, chrK) / np.sqrt(chrK)
    X = crandn(rng, chlK, d, d, chrK)
    Z = crandn(rng, chlB, d, d, chrB)
    return L, R, X, Z


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_tf32"])
def test_lp_heff_matches_oracle(api, ctx, precision):
    import torch
    from tests.gpu_util import L_to_lib, R_to_lib, to_dev, to_host
    eps, V = inputs.flat_band_bath(5)
    cases = [(ompo.heisenberg_mpo(12), 4, (64, 64, 64, 64)),
             (ompo.heisenberg_mpo(12), 5, (60, 72, 56, 40)),
             (ompo.heisenberg_mpo(40), 20, (256, 256, 256, 256)),
             (ompo.anderson_mpo(-0.15, 0.3, eps, V), 2, (48, 40, 36, 44))]
    rng = np.random.default_rng(11)
    for Ws, i, dims in cases:
        H = api.mpo_create(ctx, Ws)
        L, R, X, Z = _heff_case(rng, Ws, i, *dims)
        alpha, gamma = 0.7 - 0.1j, 0.25
        want = alpha * ls.heff_apply(L, Ws[i], Ws[i + 1], R, X) + gamma * Z
        api.k_heff_lp_prepare(ctx, H, i, to_dev(L_to_lib(L)), to_dev(R_to_lib(R)), precision)
        Y = torch.full(Z.shape, float("nan"), dtype=torch.complex128, device="cuda")
        for _ in range(2):          # the prepared operands serve repeated matvecs
            api.k_heff_lp_apply(ctx, H, i, to_dev(X), Y, alpha, to_dev(Z), gamma)
            got = to_host(Y)
            err = np.linalg.norm(got - want) / np.linalg.norm(want - gamma * Z)
            assert err <= 8 * U[precision], (dims, err)
        # back-to-back matvecs leave Y as one matvec does
        Y2 = torch.full(Z.shape, float("nan"), dtype=torch.complex128, device="cuda")
        api.k_heff_lp_apply_n(ctx, H, i, to_dev(X), Y2, alpha, to_dev(Z), gamma, reps=3)
        assert np.array_equal(to_host(Y2), got)
    # an apply for another shape than the prepared one is refused
    H = api.mpo_create(ctx, ompo.heisenberg_mpo(12))
    Y = torch.zeros((8, 2, 2, 8), dtype=torch.complex128, device="cuda")
    X = torch.zeros((8, 2, 2, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(RuntimeError):
        api.k_heff_lp_apply(ctx, H, 4, X, Y)


@pytest.mark.parametrize("model,chi", [("heisenberg", 512), ("heisenberg", 1024),
                                       ("anderson", 512)])
def test_heff_lp_at_the_quoted_shapes(api, ctx, model, chi):
    # the bulk shapes whose H_eff rates the benchmark quotes: the low-precision
    # matvec against the FP64-class matvec (held to the oracle elsewhere) on
    # the same random environments, within 8u relative
    import torch
    from tests.gpu_util import crandn
    rng = np.random.default_rng(21)
    if model == "heisenberg":
        H, d, D = api.mpo_create_heisenberg(ctx, 40), 2, 5
    else:
        eps, V = inputs.flat_band_bath(39)
        H, d, D = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15), 4, 6

    def dev(*shape):
        return torch.from_numpy(crandn(rng, *shape) / np.sqrt(shape[-1])).to("cuda")
    L, R, X, Z = dev(D, chi, chi), dev(D, chi, chi), dev(chi, d, d, chi), dev(chi, d, d, chi)
    alpha, gamma = 0.9 + 0.2j, -0.3
    Yref = torch.empty_like(X)
    api.set_kernel_precision(ctx, "fp64_tc")
    try:
        api.k_heff(ctx, H, 20, L, R, X, Yref, alpha, Z, gamma)
    finally:
        api.set_kernel_precision(ctx, "fp64")
    ref = Yref - gamma * Z
    for precision in ("mixed_bf16", "mixed_tf32"):
        api.k_heff_lp_prepare(ctx, H, 20, L, R, precision)
        Y = torch.full_like(X, float("nan"))
        api.k_heff_lp_apply_n(ctx, H, 20, X, Y, alpha, Z, gamma, reps=2)
        err = (torch.linalg.vector_norm(Y - Yref) / torch.linalg.vector_norm(ref)).item()
        assert err <= 8 * U[precision], (model, chi, precision, err)
    del L, R, X, Z, Y, Yref


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_tf32"])
def test_refined_local_solve_matches_converged_gmres(api, ctx, precision):
    # a local problem of a saturated chi = 64 MPS: environments of the real
    # state, alpha = 1 - c s with a certified lower bound s, c = 0.3
    from tests.gpu_util import L_to_lib, R_to_lib, to_dev, to_host
    N, chi, i = 16, 64, 7
    Ws = ompo.heisenberg_mpo(N)
    A = inputs.random_isometric_mps(N, 2, chi, 2003)
    x = ls.right_canonicalize_svd(A)
    Rop = ls._build_right_envs(Ws, x, [("op", x)])[0]
    Lop = np.ones((1, 1, 1), complex)
    for k in range(i):                                   # move the centre to site i
        Xk = np.tensordot(x[k], x[k + 1], axes=([2], [0]))
        x[k], x[k + 1], _, _ = ls.split_two_site(Xk, 10 ** 6, 0.0, True)
        Lop = ls.left_env_update(Lop, x[k], Ws[k], x[k])
    L, R = Lop, Rop[i + 1]
    c, s = 0.3, -0.75 * (N - 1)
    alpha = 1.0 - c * s
    rng = np.random.default_rng(5)
    B = np.tensordot(x[i], x[i + 1], axes=([2], [0])) + 0.1 * (
        rng.standard_normal(x[i].shape[:2] + x[i + 1].shape[1:]) + 0j)
    X0 = np.tensordot(x[i], x[i + 1], axes=([2], [0]))
    mv = lambda V: alpha * V + c * ls.heff_apply(L, Ws[i], Ws[i + 1], R, V)
    want, (steps, res) = ls.gmres_restarted(mv, B, X0, 10, cycles=100, local_tol=1e-13)
    assert res <= 1e-13
    H = api.mpo_create(ctx, Ws)
    api.set_kernel_precision(ctx, precision)
    try:
        Xd = to_dev(X0)
        st, rel = api.k_local_solve(ctx, H, i, to_dev(L_to_lib(L)), to_dev(R_to_lib(R)), to_dev(B),
                                    Xd, alpha, c, krylov_dim=10, local_tol=1e-12)
    finally:
        api.set_kernel_precision(ctx, "fp64")
    got = to_host(Xd)
    assert rel <= 1e-12
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_tf32"])
@pytest.mark.parametrize("scheme", ["be", "tr"])
def test_mixed_step_matches_converged_oracle_chi128(api, ctx, precision, scheme):
    # N = 16, chi = 128 (bulk blocks 256 x 256): one step in a mixed mode
    # against the oracle with local GMRES converged to 1e-12 (reading c13);
    # shift = a certified lower bound, so every local system is positive
    # definite and the converged solve is well defined
    N, chi, cutoff, dt = 16, 128, 1e-10, 0.2
    Ws = ompo.heisenberg_mpo(N)
    H = api.mpo_create_heisenberg(ctx, N)
    A = inputs.random_isometric_mps(N, 2, chi, 2002)
    s = -0.75 * (N - 1)
    ost, oinfo = ostep.implicit_step(Ws, A, dt, scheme, s, chi, cutoff, local_tol=1e-12,
                                     max_cycles=100)
    psi = api.mps_create(ctx, A, chi)
    ginfo = api.implicit_step(ctx, H, psi, dt, scheme, s, chi, cutoff,
                              api.solver_opts(precision=precision, refine_tol=1e-11, refine_max=20))
    got = psi.tensors()
    rel = abs(ginfo["energy"] - oinfo.energy) / abs(oinfo.energy)
    assert rel <= 1e-8, rel
    ov = abs(omps.overlap(ost, got)) / (omps.norm(ost) * omps.norm(got))
    assert 1.0 - ov <= 1e-8
    assert ginfo["max_local_residual"] <= 1e-11


def test_mixed_step_at_the_benchmarked_configuration(api, ctx):
    # N = 64, chi_max = 256, cutoff 1e-10, the benchmark's start state and
    # first step (dtau = 1e-3, shift = the state's energy), mixed bf16 against
    # the oracle with converged local solves
    N, chi, cutoff, dt = 64, 256, 1e-10, 1e-3
    Ws = ompo.heisenberg_mpo(N)
    H = api.mpo_create_heisenberg(ctx, N)
    A = inputs.random_isometric_mps(N, 2, chi, 2000)
    s = omps.expect_mpo(A, Ws)
    ost, oinfo = ostep.implicit_step(Ws, A, dt, "be", s, chi, cutoff, local_tol=1e-12,
                                     max_cycles=100)
    psi = api.mps_create(ctx, A, chi)
    ginfo = api.implicit_step(ctx, H, psi, dt, "be", s, chi, cutoff,
                              api.solver_opts(precision="mixed_bf16", refine_tol=1e-11,
                                              refine_max=20))
    rel = abs(ginfo["energy"] - oinfo.energy) / abs(oinfo.energy)
    assert rel <= 1e-8, rel
    got = psi.tensors()
    ov = abs(omps.overlap(ost, got)) / (omps.norm(ost) * omps.norm(got))
    assert 1.0 - ov <= 1e-8
