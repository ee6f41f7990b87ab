"""GPU parity of each kernel-level step of the sweep against the oracle, at
small sizes (element by element, several tiles and ragged tails) and at the
workload sizes (sampled entries the oracle computes one by one).

Tolerance: all FP64.  A contraction over K terms has rounding error of order
K * 2^-53 relative to the largest partial sums; with K <= 4e4 that is below
1e-11, so element-wise checks use 1e-12 (small) / 1e-11 (workload sizes)
relative to the largest output magnitude."""
import numpy as np
import pytest

from oracle import linsolve as ls, mpo as ompo
from paper_2606_02930_gb300 import inputs

from tests.gpu_util import (L_from_lib, L_to_lib, R_from_lib, R_to_lib, crandn, rel_err,
                            to_dev, to_host)

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


def _models(n_sites_heis=8, n_bath=5):
    Wh = ompo.heisenberg_mpo(n_sites_heis)
    eps, V = inputs.flat_band_bath(n_bath)
    Wa = ompo.anderson_mpo(-0.15, 0.3, eps, V)
    return {"heisenberg": Wh, "anderson": Wa}


@pytest.mark.parametrize("model", ["heisenberg", "anderson"])
@pytest.mark.parametrize("dims", [(1, 1, 1, 1), (3, 3, 5, 5), (7, 5, 6, 9), (33, 40, 37, 35)])
def test_heff_matches_oracle(api, ctx, model, dims):
    Ws = _models()[model]
    H = api.mpo_create(ctx, Ws)
    rng = np.random.default_rng(hash((model, dims)) % 2**32)
    chlB, chlK, chrK, chrB = dims
    i = 2
    D0, D2, d = Ws[i].shape[0], Ws[i + 1].shape[3], Ws[i].shape[1]
    L = crandn(rng, chlB, D0, chlK)
    R = crandn(rng, chrB, D2, chrK)
    X = crandn(rng, chlK, d, d, chrK)
    Z = crandn(rng, chlB, d, d, chrB)
    want = 0.7 * ls.heff_apply(L, Ws[i], Ws[i + 1], R, X) + (0.2 - 0.1j) * Z
    Y = to_dev(np.zeros_like(Z))
    api.k_heff(ctx, H, i, to_dev(L_to_lib(L)), to_dev(R_to_lib(R)), to_dev(X), Y, alpha=0.7,
               Z=to_dev(Z), gamma=0.2 - 0.1j)
    assert rel_err(to_host(Y), want) < 1e-12


@pytest.mark.parametrize("model,dims", [("heisenberg", (128, 128, 128, 128)),
                                        ("heisenberg", (200, 136, 160, 190)),
                                        ("anderson", (96, 96, 80, 96))])
def test_heff_and_env_tensor_core_mode(api, model, dims):
    # kernel-level H_eff and environment update with the contractions on the
    # tensor cores (FP64-class slicing): same results as the oracle within
    # the emulation's bound K 2^-52 relative to the largest products
    kctx = api.ctx_create(0)
    api.set_kernel_precision(kctx, "fp64_tc")
    Ws = _models()[model]
    H = api.mpo_create(kctx, Ws)
    rng = np.random.default_rng(sum(dims) + len(model))
    chlB, chlK, chrK, chrB = dims
    i = 2
    D0, D2, d = Ws[i].shape[0], Ws[i + 1].shape[3], Ws[i].shape[1]
    L = crandn(rng, chlB, D0, chlK)
    R = crandn(rng, chrB, D2, chrK)
    X = crandn(rng, chlK, d, d, chrK)
    want = ls.heff_apply(L, Ws[i], Ws[i + 1], R, X)
    Y = to_dev(np.zeros((chlB, d, d, chrB), complex))
    api.k_heff(kctx, H, i, to_dev(L_to_lib(L)), to_dev(R_to_lib(R)), to_dev(X), Y)
    assert rel_err(to_host(Y), want) < 1e-10
    bra = crandn(rng, chlB, d, chrB)
    ket = crandn(rng, chlK, d, chrK)
    want_l = ls.left_env_update(L, bra, Ws[i], ket)
    Lout = to_dev(np.zeros((Ws[i].shape[3], chrB, chrK), complex))
    api.k_env_left(kctx, H, i, to_dev(L_to_lib(L)), to_dev(bra), to_dev(ket), Lout)
    assert rel_err(L_from_lib(to_host(Lout)), want_l) < 1e-10


@pytest.mark.parametrize("model,chi,nsamp", [("heisenberg", 256, 6), ("anderson", 512, 3)])
def test_heff_workload_size_sampled(api, ctx, model, chi, nsamp):
    # bulk two-site block of the N=64 chi=256 Heisenberg chain and of the
    # chi=512 Anderson chain
    Ws = _models()[model]
    H = api.mpo_create(ctx, Ws)
    rng = np.random.default_rng(chi)
    i = 2
    D0, D2, d = Ws[i].shape[0], Ws[i + 1].shape[3], Ws[i].shape[1]
    L = crandn(rng, chi, D0, chi)
    R = crandn(rng, chi, D2, chi)
    X = crandn(rng, chi, d, d, chi)
    Y = to_dev(np.zeros((chi, d, d, chi)))
    api.k_heff(ctx, H, i, to_dev(L_to_lib(L)), to_dev(R_to_lib(R)), to_dev(X), Y)
    Yh = to_host(Y)
    scale = None
    for k in range(nsamp):
        a, b = int(rng.integers(chi)), int(rng.integers(chi))
        want = ls.heff_entry(L, Ws[i], Ws[i + 1], R, X, a, b)
        scale = np.abs(want).max() if scale is None else max(scale, np.abs(want).max())
        assert np.abs(Yh[a, :, :, b] - want).max() < 1e-11 * scale
    assert np.isfinite(Yh).all()


@pytest.mark.parametrize("model", ["heisenberg", "anderson"])
@pytest.mark.parametrize("dims", [(1, 1, 2, 3), (4, 6, 5, 7), (31, 17, 40, 33)])
def test_env_updates_match_oracle(api, ctx, model, dims):
    Ws = _models()[model]
    H = api.mpo_create(ctx, Ws)
    rng = np.random.default_rng(7 + sum(dims))
    chlB, chlK, chrB, chrK = dims
    i = 3
    W = Ws[i]
    Dl, d, Dr = W.shape[0], W.shape[1], W.shape[3]
    bra = crandn(rng, chlB, d, chrB)
    ket = crandn(rng, chlK, d, chrK)
    Lin = crandn(rng, chlB, Dl, chlK)
    want = ls.left_env_update(Lin, bra, W, ket)
    Lout = to_dev(np.zeros((Dr, chrB, chrK)))
    api.k_env_left(ctx, H, i, to_dev(L_to_lib(Lin)), to_dev(bra), to_dev(ket), Lout)
    assert rel_err(L_from_lib(to_host(Lout)), want) < 1e-12
    Rin = crandn(rng, chrB, Dr, chrK)
    want = ls.right_env_update(Rin, bra, W, ket)
    Rout = to_dev(np.zeros((Dl, chlK, chlB)))
    api.k_env_right(ctx, H, i, to_dev(R_to_lib(Rin)), to_dev(bra), to_dev(ket), Rout)
    assert rel_err(R_from_lib(to_host(Rout)), want) < 1e-12


def _spectrum_matrix(rng, m, n, sv):
    U, _ = np.linalg.qr(crandn(rng, m, len(sv)))
    V, _ = np.linalg.qr(crandn(rng, n, len(sv)))
    return (U * sv[None, :]) @ V.conj().T


@pytest.mark.parametrize("m,n,kind", [(1, 7, "rand"), (9, 1, "rand"), (20, 33, "decay"),
                                      (40, 24, "decay"), (64, 64, "ties"), (30, 50, "lowrank"),
                                      (512, 512, "decay")])
def test_split_matches_oracle(api, ctx, m, n, kind):
    rng = np.random.default_rng(m * 1000 + n)
    p = min(m, n)
    if kind == "rand":
        X = crandn(rng, m, n)
    elif kind == "decay":
        X = _spectrum_matrix(rng, m, n, np.exp(-np.arange(p) / 6.0))
    elif kind == "ties":
        sv = np.repeat(np.exp(-np.arange(p // 4) / 3.0), 4)       # quadruplets
        X = _spectrum_matrix(rng, m, n, sv)
    else:
        sv = np.concatenate([np.exp(-np.arange(p // 3) / 4.0), np.zeros(p - p // 3)])
        X = _spectrum_matrix(rng, m, n, sv)
    S_ref = np.linalg.svd(X, compute_uv=False)
    for chi_max, cutoff in ((p, 0.0), (max(1, p // 2), 1e-10), (max(1, p // 3 + 1), 0.0)):
        r_ref, disc_ref = ls.choose_rank(S_ref, chi_max, cutoff)
        for centre_right in (True, False):
            left = to_dev(np.zeros(m * p))
            right = to_dev(np.zeros(p * n))
            sig = __import__("torch").zeros(p, dtype=__import__("torch").float64, device="cuda")
            r, disc = api.k_split(ctx, to_dev(X), m, n, chi_max, cutoff, centre_right, left, right,
                                  sig)
            assert r == r_ref
            assert abs(disc - disc_ref) <= 1e-12 * max(disc_ref, 1e-12) + 1e-15
            # singular values are resolved for the first chi_max entries down
            # to the skip weight 1e-3 max(cutoff, 1e-25) of the total; beyond
            # them only the total weight is exact
            sg = sig.cpu().numpy()
            tot = np.sum(S_ref ** 2)
            res = S_ref ** 2 > 1e-3 * max(cutoff, 1e-25) * tot * 10
            res[chi_max:] = False
            assert np.allclose(sg[res], S_ref[res], rtol=0, atol=1e-13 * S_ref[0])
            assert abs(np.sum(sg[~res] ** 2) - np.sum(S_ref[~res] ** 2)) <= 1e-13 * tot
            Lh = to_host(left)[: m * r].reshape(m, r)
            Rh = to_host(right)[: r * n].reshape(r, n)
            # the truncated product is gauge invariant: compare with the oracle split
            A1, A2, _, _ = ls.split_two_site(X.reshape(m, 1, 1, n), chi_max, cutoff, centre_right)
            want = A1.reshape(m, -1) @ A2.reshape(-1, n)
            assert rel_err(Lh @ Rh, want) < 1e-11
            iso = Lh if centre_right else Rh.conj().T
            assert np.abs(iso.conj().T @ iso - np.eye(r)).max() < 1e-12


def _canonical_envs(Ws, A, i):
    """Environments of a mixed-canonical random MPS around bond (i, i+1)."""
    from oracle import mps as omps
    B = ls.right_canonicalize_svd(A)
    for k in range(i):
        chl, d, chr_ = B[k].shape
        Q, Rm = np.linalg.qr(B[k].reshape(chl * d, chr_))
        B[k] = Q.reshape(chl, d, Q.shape[1])
        B[k + 1] = np.tensordot(Rm, B[k + 1], axes=([1], [0]))
    L = np.ones((1, 1, 1), complex)
    for k in range(i):
        L = ls.left_env_update(L, B[k], Ws[k], B[k])
    R = np.ones((1, 1, 1), complex)
    for k in range(len(B) - 1, i + 1, -1):
        R = ls.right_env_update(R, B[k], Ws[k], B[k])
    X0 = np.tensordot(B[i], B[i + 1], axes=([2], [0]))
    return L, R, X0


@pytest.mark.parametrize("model,N,chi,i", [("heisenberg", 10, 8, 4), ("heisenberg", 20, 64, 9),
                                           ("anderson", 6, 16, 2), ("heisenberg", 24, 256, 11)])
def test_local_solve_matches_oracle_gmres(api, ctx, model, N, chi, i):
    if model == "heisenberg":
        Ws = ompo.heisenberg_mpo(N)
        A = inputs.random_mps(N, 2, chi, 100 + N)
    else:
        eps, V = inputs.flat_band_bath(N - 1)
        Ws = ompo.anderson_mpo(-0.15, 0.3, eps, V)
        A = inputs.random_mps(N, 4, chi, 100 + N)
    H = api.mpo_create(ctx, Ws)
    L, R, X0 = _canonical_envs(Ws, A, i)
    rng = np.random.default_rng(N)
    B = X0 + 0.3 * crandn(rng, *X0.shape)
    for c, s, m in ((0.05, -1.0, 10), (30.0, 0.2, 10), (1.0, 0.0, 4)):
        alpha = 1.0 - c * s
        mv = lambda V: alpha * V + c * ls.heff_apply(L, Ws[i], Ws[i + 1], R, V)
        Xw, (k_ref, res_ref) = ls.gmres(mv, B, X0, m)
        X = to_dev(X0)
        k, res = api.k_local_solve(ctx, H, i, to_dev(L_to_lib(L)), to_dev(R_to_lib(R)), to_dev(B), X,
                                   alpha, c, m)
        assert k == k_ref
        assert rel_err(to_host(X), Xw) < 1e-10
        assert abs(res - res_ref) < 1e-8 * max(res_ref, 1e-6)


def test_bounded_grid_wait_ends_with_a_status(api, ctx):
    # A grid barrier that some blocks never reach: the waiting blocks give up
    # at the barrier's iteration limit, the call reports ITE_ETIMEOUT instead
    # of hanging, and the context keeps working (a split afterwards is exact).
    import torch
    from paper_2606_02930_gb300 import _lib as L
    assert api.k_barrier_selftest(ctx, 16, 0) == L.ITE_OK
    assert api.k_barrier_selftest(ctx, 16, 3) == L.ITE_ETIMEOUT
    assert b"wait ran out" in L.lib.ite_last_error(ctx.h)
    assert api.k_barrier_selftest(ctx, 16, 0) == L.ITE_OK
    rng = np.random.default_rng(5)
    X = _spectrum_matrix(rng, 64, 48, np.exp(-np.arange(48) / 6.0))
    left = to_dev(np.zeros(64 * 64))
    right = to_dev(np.zeros(64 * 48))
    sig = torch.zeros(48, dtype=torch.float64, device="cuda")
    r, _ = api.k_split(ctx, to_dev(X), 64, 48, 48, 0.0, True, left, right, sig)
    S = np.linalg.svd(X, compute_uv=False)
    assert r == 48
    assert np.max(np.abs(sig.cpu().numpy() - S) / S) < 1e-12


def test_local_solve_is_invariant_under_scaling(api, ctx):
    # (A, s B, s X0) gives s X in the same number of Krylov steps, also when
    # the scale makes |r0| tiny or huge next to |A v_j|
    N, chi, i = 8, 12, 3
    Ws = ompo.heisenberg_mpo(N)
    A = inputs.random_mps(N, 2, chi, 100 + N)
    H = api.mpo_create(ctx, Ws)
    L, R, X0 = _canonical_envs(Ws, A, i)
    B = X0 + 0.3 * crandn(np.random.default_rng(9), *X0.shape)
    Ld, Rd = to_dev(L_to_lib(L)), to_dev(R_to_lib(R))
    runs = {}
    for scale in (1.0, 1e-20, 1e20):
        X = to_dev(scale * X0)
        k, res = api.k_local_solve(ctx, H, i, Ld, Rd, to_dev(scale * B), X, 1.05, 0.05, 10)
        runs[scale] = (k, res, to_host(X) / scale)
    k1, r1, x1 = runs[1.0]
    assert k1 == 10
    for scale in (1e-20, 1e20):
        k, res, x = runs[scale]
        assert k == k1, scale
        assert rel_err(x, x1) < 1e-12
        assert abs(res - r1) < 1e-10


@pytest.mark.parametrize("m,n,chi_max,cutoff", [(1024, 1024, 256, 1e-10), (2048, 2048, 512, 1e-14)])
def test_split_workload_row_lengths(api, ctx, m, n, chi_max, cutoff):
    # The two-site blocks of the larger workloads: rows of 1024 (chi = 512
    # with d = 2, or chi = 256 with d = 4) and of 2048 (the chi = 512 impurity
    # chain, d = 4).  They take the Jacobi's 16-element register path and its
    # streamed path.  Same rank, singular values and truncated product as the
    # oracle's SVD, and an isometric left factor.
    import torch
    rng = np.random.default_rng(m + 1)
    p = min(m, n)
    X = _spectrum_matrix(rng, m, n, np.exp(-np.arange(p) / (p / 16)))
    S_ref = np.linalg.svd(X, compute_uv=False)
    r_ref, disc_ref = ls.choose_rank(S_ref, chi_max, cutoff)
    left = to_dev(np.zeros(m * p))
    right = to_dev(np.zeros(p * n))
    sig = torch.zeros(p, dtype=torch.float64, device="cuda")
    r, disc = api.k_split(ctx, to_dev(X), m, n, chi_max, cutoff, True, left, right, sig, tc=True)
    assert r == r_ref
    assert abs(disc - disc_ref) <= 1e-10 * max(disc_ref, 1e-12) + 1e-15
    sg = sig.cpu().numpy()[:r]
    assert np.max(np.abs(sg - S_ref[:r]) / S_ref[:r]) < 1e-10
    Lh = to_host(left)[: m * r].reshape(m, r)
    Rh = to_host(right)[: r * n].reshape(r, n)
    A1, A2, _, _ = ls.split_two_site(X.reshape(m, 1, 1, n), chi_max, cutoff, True)
    assert rel_err(Lh @ Rh, A1.reshape(m, -1) @ A2.reshape(-1, n)) < 1e-10
    assert np.abs(Lh.conj().T @ Lh - np.eye(r)).max() < 1e-12


@pytest.mark.parametrize("m,n,kind", [(128, 128, "decay"), (512, 512, "decay"), (200, 160, "ties"),
                                      (160, 200, "decay"), (256, 512, "decay")])
def test_split_tensor_core_mode(api, ctx, m, n, kind):
    # split with the projection GEMM on the tensor cores (FP64-class
    # emulation): same rank and truncated product as the oracle's SVD
    import torch
    rng = np.random.default_rng(m * 31 + n)
    p = min(m, n)
    if kind == "decay":
        X = _spectrum_matrix(rng, m, n, np.exp(-np.arange(p) / 20.0))
    else:
        sv = np.repeat(np.exp(-np.arange(p // 4) / 8.0), 4)
        X = _spectrum_matrix(rng, m, n, sv)
    S_ref = np.linalg.svd(X, compute_uv=False)
    for chi_max, cutoff in ((p, 1e-10), (max(1, p // 2), 1e-10), (max(1, p // 3 + 1), 0.0)):
        eff = cutoff
        r_ref, disc_ref = ls.choose_rank(S_ref, chi_max, eff)
        for centre_right in (True, False):
            left = to_dev(np.zeros(m * max(m, n)))
            right = to_dev(np.zeros(max(m, n) * n))
            r, disc = api.k_split(ctx, to_dev(X), m, n, chi_max, cutoff, centre_right, left, right,
                                  tc=True)
            assert r == r_ref
            assert abs(disc - disc_ref) <= 1e-10 * max(disc_ref, 1e-12) + 1e-15
            Lh = to_host(left)[: m * r].reshape(m, r)
            Rh = to_host(right)[: r * n].reshape(r, n)
            A1, A2, _, _ = ls.split_two_site(X.reshape(m, 1, 1, n), chi_max, eff, centre_right)
            want = A1.reshape(m, -1) @ A2.reshape(-1, n)
            assert rel_err(Lh @ Rh, want) < 1e-11
            iso = Lh if centre_right else Rh.conj().T
            assert np.abs(iso.conj().T @ iso - np.eye(r)).max() < 1e-12
