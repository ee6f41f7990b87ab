"""Pins for the MPS tier of the oracle: brute-force dense contractions on tiny
inputs, H_eff = P^dag H P for the isometry of a mixed-canonical MPS,
Hermiticity, GMRES against the explicit Krylov least-squares problem, the
truncation rule, and converged sweeps against the dense discrete propagator
(which the dense tier pins to closed forms)."""
import numpy as np
import pytest

from oracle import ed, grid, linsolve as ls, mpo, mps, step
from paper_2606_02930_gb300 import inputs


def dense_of_product(psi):
    v = psi[0]
    for k in range(1, len(psi)):
        v = np.kron(v, psi[k])
    return v


def test_dense_contractions_brute_force():
    N, d = 5, 2
    A = inputs.random_mps(N, d, 3, 21)
    v = mps.to_dense(A)
    # brute force amplitude by explicit matrix products
    for idx in (0, 7, 19, 31):
        digits = [(idx >> (N - 1 - k)) & 1 for k in range(N)]
        M = np.eye(1)
        for k, s in enumerate(digits):
            M = M @ A[k][:, s, :]
        assert abs(M[0, 0] - v[idx]) < 1e-14
    B = inputs.random_mps(N, d, 4, 22)
    assert abs(mps.overlap(B, A) - np.vdot(mps.to_dense(B), v)) < 1e-13
    H = ed.heisenberg_hamiltonian(N)
    assert abs(mps.expect_mpo(A, mpo.heisenberg_mpo(N)) - ed.energy(H, v)) < 1e-13


def test_correlators_against_dense_operators():
    N = 5
    A = inputs.random_mps(N, 2, 4, 31)
    v = mps.to_dense(A)
    v = v / np.linalg.norm(v)
    from tests.test_oracle_ed import kron_site, SZ, SX
    for i, j in ((0, 3), (1, 1), (2, 4)):
        Od = kron_site(SZ, i, N) @ kron_site(SX, j, N)
        want = np.vdot(v, Od @ v)
        got = mps.correlator(A, SZ, i, SX, j)
        assert abs(got - want) < 1e-13


def test_fermion_correlator_with_string_matches_fock_space():
    # <c^dag_{i,up} c_{j,up}> with the Jordan-Wigner string, against the Fock
    # space operator built by explicit sign counting.
    rng = np.random.default_rng(8)
    n_sites = 4
    A = inputs.random_mps(n_sites, 4, 6, 41)
    v = mps.to_dense(A)
    v = v / np.linalg.norm(v)
    for i, j in ((0, 2), (1, 3), (0, 3)):
        p, q = 2 * i, 2 * j
        dim = 4 ** n_sites
        Op = np.zeros((dim, dim))
        for idx in range(dim):
            r = ed._hop(idx, p, q, n_sites)
            if r is not None:
                Op[r[0], idx] += r[1]
        want = np.vdot(v, Op @ v)
        got = mps.correlator(A, mpo.C_UP.T @ mpo.F_PAR, i, mpo.C_UP, j, string=mpo.F_PAR)
        assert abs(got - want) < 1e-13


def test_right_canonicalize():
    A = inputs.random_mps(6, 2, 8, 51)
    B = mps.right_canonicalize(A)
    assert abs(abs(mps.overlap(A, B)) / (mps.norm(A) * mps.norm(B)) - 1) < 1e-14
    for T in B[1:]:
        M = T.reshape(T.shape[0], -1)
        assert np.abs(M @ M.conj().T - np.eye(M.shape[0])).max() < 1e-13


def _mixed_canonical(A, i):
    """Left-orthonormal sites < i, right-orthonormal sites > i+1 (via QR)."""
    B = mps.right_canonicalize(A)
    for k in range(i):
        chl, d, chr_ = B[k].shape
        Q, R = np.linalg.qr(B[k].reshape(chl * d, chr_))
        B[k] = Q.reshape(chl, d, Q.shape[1])
        B[k + 1] = np.tensordot(R, B[k + 1], axes=([1], [0]))
    return B


@pytest.mark.parametrize("model", ["heisenberg", "anderson"])
def test_heff_is_projected_hamiltonian_and_hermitian(model):
    if model == "heisenberg":
        N, d = 6, 2
        Ws = mpo.heisenberg_mpo(N)
        H = ed.heisenberg_hamiltonian(N)
        A = inputs.random_mps(N, d, 4, 61)
    else:
        N, d = 4, 4
        eps, V = inputs.flat_band_bath(3)
        Ws = mpo.anderson_mpo(-0.15, 0.3, eps, V)
        H = ed.anderson_hamiltonian(-0.15, 0.3, eps, V)
        A = inputs.random_mps(N, d, 6, 62)
    i = 2 if model == "heisenberg" else 1
    B = _mixed_canonical(A, i)
    L = np.ones((1, 1, 1), complex)
    for k in range(i):
        L = ls.left_env_update(L, B[k], Ws[k], B[k])
    R = np.ones((1, 1, 1), complex)
    for k in range(N - 1, i + 1, -1):
        R = ls.right_env_update(R, B[k], Ws[k], B[k])
    chl, chr_ = B[i].shape[0], B[i + 1].shape[2]
    n = chl * d * d * chr_
    Heff = np.zeros((n, n), complex)
    for col in range(n):
        e = np.zeros(n, complex)
        e[col] = 1.0
        Heff[:, col] = ls.heff_apply(L, Ws[i], Ws[i + 1], R, e.reshape(chl, d, d, chr_)).ravel()
    assert np.abs(Heff - Heff.conj().T).max() <= 1e-13 * np.abs(Heff).max()
    # isometry P: column (a, s, t, b) -> dense state with that two-site block
    P = np.zeros((d ** N, n), complex)
    for col in range(n):
        e = np.zeros(n, complex)
        e[col] = 1.0
        vec = e.reshape(chl, d, d, chr_)
        if i > 0:
            vec = np.tensordot(_left_block_matrix(B[:i]), vec, axes=([1], [0]))
        else:
            vec = vec[0]
        if i + 2 < N:
            vec = np.tensordot(vec, _right_block_matrix(B[i + 2:]), axes=([vec.ndim - 1], [0]))
        else:
            vec = vec[..., 0]
        P[:, col] = vec.ravel()
    assert np.abs(P.conj().T @ P - np.eye(n)).max() < 1e-12
    assert np.abs(P.conj().T @ H @ P - Heff).max() < 1e-12


def _left_block_matrix(sites):
    M = sites[0].reshape(sites[0].shape[1], sites[0].shape[2])
    for T in sites[1:]:
        M = np.tensordot(M, T, axes=([1], [0])).reshape(-1, T.shape[2])
    return M


def _right_block_matrix(sites):
    M = sites[-1].reshape(sites[-1].shape[0], sites[-1].shape[1])
    for T in reversed(sites[:-1]):
        M = np.tensordot(T, M, axes=([2], [0])).reshape(T.shape[0], -1)
    return M


def test_gmres_equals_krylov_least_squares():
    rng = np.random.default_rng(71)
    n = 40
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = np.eye(n) + 0.1 * (G + G.conj().T)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x0 = rng.standard_normal(n) + 0j
    for m in (1, 4, 10):
        x, (k, res) = ls.gmres(lambda v: A @ v, b, x0, m)
        r0 = b - A @ x0
        K = np.stack([np.linalg.matrix_power(A, j) @ r0 for j in range(m)], axis=1)
        Q, _ = np.linalg.qr(K)
        y = np.linalg.lstsq(A @ Q, r0, rcond=None)[0]
        want = x0 + Q @ y
        assert k == m
        assert np.linalg.norm(x - want) < 1e-10 * np.linalg.norm(want)
        assert abs(res - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) < 1e-10
    x, (k, _) = ls.gmres(lambda v: A @ v, b, x0, n + 5)
    assert np.linalg.norm(A @ x - b) < 1e-10 * np.linalg.norm(b)
    # happy breakdown: b in a 3-dimensional invariant subspace
    D = np.diag(np.arange(1.0, n + 1))
    bb = np.zeros(n, complex)
    bb[:3] = 1.0
    x, (k, _) = ls.gmres(lambda v: D @ v, bb, np.zeros(n, complex), 10)
    assert k == 3 and np.linalg.norm(D @ x - bb) < 1e-13


def test_gmres_is_invariant_under_scaling():
    # GMRES on (A, s b, s x0) returns s x in the same number of steps for any
    # scale s: the breakdown test compares h_{j+1,j} with |A v_j| (both of
    # the unit Krylov vectors), not with the scale of the residual
    rng = np.random.default_rng(73)
    n = 40
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = np.eye(n) + 0.1 * (G + G.conj().T)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x0 = rng.standard_normal(n) + 0j
    x1, (k1, r1) = ls.gmres(lambda v: A @ v, b, x0, 10)
    assert k1 == 10
    for scale in (1e-20, 1e-8, 1e8, 1e20):
        xs, (ks, rs) = ls.gmres(lambda v: A @ v, scale * b, scale * x0, 10)
        assert ks == k1, scale
        assert np.linalg.norm(xs / scale - x1) < 1e-12 * np.linalg.norm(x1)
        assert abs(rs - r1) < 1e-12


def test_restarted_gmres():
    # one cycle is plain GMRES; on a well-conditioned system restarted
    # GMRES(4) reaches the solution that a dense solve gives, with a
    # residual that never grows from cycle to cycle
    rng = np.random.default_rng(74)
    n = 40
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = 3.0 * np.eye(n) + 0.05 * (G + G.conj().T)             # spectrum in about [2, 4]
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x0 = np.zeros(n, complex)
    mv = lambda v: A @ v
    x1, (k1, r1) = ls.gmres_restarted(mv, b, x0, 4, 1)
    xg, (kg, rg) = ls.gmres(mv, b, x0, 4)
    assert k1 == kg == 4 and np.array_equal(x1, xg) and r1 == rg
    res = []
    for cycles in (1, 2, 4, 8, 60):
        _, (_, r) = ls.gmres_restarted(mv, b, x0, 4, cycles)
        res.append(r)
    assert all(b_ <= a_ * (1 + 1e-12) + 1e-14 for a_, b_ in zip(res, res[1:]))
    x, (k, r) = ls.gmres_restarted(mv, b, x0, 4, 60, local_tol=1e-13)
    want = np.linalg.solve(A, b)
    assert r <= 1e-13 and k < 4 * 60
    assert np.linalg.norm(x - want) < 1e-11 * np.linalg.norm(want)


def test_choose_rank_rules():
    S = np.array([1.0, 0.5, 0.25, 1e-3, 1e-6, 0.0])
    assert ls.choose_rank(S, 10, 0.0)[0] == 5          # exact zero dropped (weight floor)
    assert ls.choose_rank(S, 10, 1e-11)[0] == 4        # 1e-12 / total < 1e-11
    assert ls.choose_rank(S, 2, 0.0)[0] == 2           # chi_max cap
    S2 = np.array([1.0, 0.6, 0.3, 0.3 * (1 - 1e-12), 0.3 * (1 - 2e-12), 0.1])
    assert ls.choose_rank(S2, 4, 0.0)[0] == 2          # cap cuts a near-degenerate group
    S3 = np.array([0.5, 0.5, 0.5, 0.1])
    assert ls.choose_rank(S3, 2, 0.0)[0] == 2          # group from the top: left as is
    r, disc = ls.choose_rank(np.array([1.0, 1e-6]), 1, 0.0)
    assert r == 1 and abs(disc - 1e-12 / (1 + 1e-12)) < 1e-20


def _exact_run(model, N, chi, scheme, K, seed):
    if model == "heisenberg":
        Ws = mpo.heisenberg_mpo(N)
        H = ed.heisenberg_hamiltonian(N)
        psi = inputs.random_product_state(N, 2, seed)
    else:
        eps, V = inputs.flat_band_bath(N - 1)
        Ws = mpo.anderson_mpo(-0.15, 0.3, eps, V)
        H = ed.anderson_hamiltonian(-0.15, 0.3, eps, V)
        psi = inputs.random_product_state(N, 4, seed)
    v0 = dense_of_product(psi)
    e0 = np.linalg.eigvalsh(H)[0]
    nodes = grid.geometric_grid(1e-2, 1e2, 20)[: K + 1]
    dense, _, _ = ed.propagate_discrete(H, v0, grid.steps(nodes), scheme, shifts=e0)
    states, infos = step.evolve(Ws, mps.product_state(psi), nodes, scheme, chi, 0.0,
                                shift=e0, local_tol=1e-13, sweeps=12, sweep_tol=1e-15,
                                fit_sweeps=6, krylov_dim=20)
    return H, dense, states, infos


@pytest.mark.parametrize("scheme", ["be", "tr", "gl2", "gl3"])
def test_converged_linsolve_equals_dense_propagator(scheme):
    # Converged sweeps at full bond dimension solve each implicit step exactly,
    # so the MPS path must reproduce prod_k R(dtau_k (H - E0)) psi0.
    H, dense, states, infos = _exact_run("heisenberg", 8, 16, scheme, 6, 1000)
    for v, s, info in zip(dense, states, infos):
        w = mps.to_dense(s)
        assert ed.infidelity(v, w) < 1e-10
        assert abs(ed.energy(H, v) - info.energy) < 1e-10 * abs(ed.energy(H, v))
        assert info.norm_before <= 1.0 + 1e-12


def test_converged_linsolve_anderson_equals_dense():
    H, dense, states, infos = _exact_run("anderson", 4, 16, "be", 4, 1001)
    for v, s in zip(dense, states):
        assert ed.infidelity(v, mps.to_dense(s)) < 1e-10


def test_fixed_mode_backward_euler_energy_monotone():
    # Paper-faithful mode (one sweep, GMRES(10)); with s <= E0 the energy may
    # only drop, up to truncation/solve error.
    N = 10
    Ws = mpo.heisenberg_mpo(N)
    H = ed.heisenberg_hamiltonian(N)
    e0 = np.linalg.eigvalsh(H)[0]
    psi = inputs.random_product_state(N, 2, 1000)
    nodes = grid.geometric_grid(1e-2, 1e2, 20)
    states, infos = step.evolve(Ws, mps.product_state(psi), nodes, "be", 32, 0.0, shift=e0)
    es = [ed.energy(H, dense_of_product(psi))] + [i.energy for i in infos]
    assert all(b <= a + 1e-10 for a, b in zip(es, es[1:]))
    assert all(i.norm_before <= 1.0 + 1e-12 for i in infos)
    assert es[-1] - e0 < 1e-6 * abs(e0)


def test_trapezoid_fit_is_exact_at_full_bond_dimension():
    N = 6
    Ws = mpo.heisenberg_mpo(N)
    H = ed.heisenberg_hamiltonian(N)
    A = inputs.random_mps(N, 2, 8, 81)
    c, s = 0.37, -2.0
    f, _ = ls.fit_affine(Ws, A, 1 + c * s, -c, 8, 0.0, sweeps=4)
    v = mps.to_dense(A)
    want = (1 + c * s) * v - c * (H @ v)
    assert np.linalg.norm(mps.to_dense(f) - want) < 1e-11 * np.linalg.norm(want)


@pytest.mark.parametrize("scheme", ["fe", "heun"])
def test_explicit_steps_equal_dense_at_full_bond_dimension(scheme):
    # the fitted explicit steps are exact at full bond dimension
    N = 6
    Ws = mpo.heisenberg_mpo(N)
    H = ed.heisenberg_hamiltonian(N)
    psi = inputs.random_product_state(N, 2, 5)
    v0 = dense_of_product(psi)
    e0 = np.linalg.eigvalsh(H)[0]
    dts = [0.05, 0.1, 0.2]
    dense, _, _ = ed.propagate_discrete(H, v0, dts, scheme, shifts=e0)
    x = mps.product_state(psi)
    for v, dt in zip(dense, dts):
        x, info = step.implicit_step(Ws, x, dt, scheme, e0, 8, 0.0, fit_sweeps=4)
        assert ed.infidelity(v, mps.to_dense(x)) < 1e-12
        assert abs(ed.energy(H, v) - info.energy) < 1e-12 * abs(ed.energy(H, v))


def _evolve_long(Ws, psi, chi, steps):
    psi = mps.copy(psi)
    psi[0] = psi[0] / mps.norm(psi)
    s = mps.expect_mpo(psi, Ws)
    nodes = grid.geometric_grid(1e-1, 2e2, steps)
    for k in range(1, len(nodes)):
        psi, info = step.implicit_step(Ws, psi, nodes[k] - nodes[k - 1], "be", s, chi, 1e-12,
                                       local_tol=1e-12, sweeps=3, sweep_tol=1e-12, krylov_dim=16)
        s = info.energy
    return s


def test_long_time_limit_of_the_open_xx_chain_is_free_fermions():
    # J_z = 0 maps by Jordan-Wigner to free fermions hopping with amplitude
    # J/2: from the Neel state (S^z = 0, half filling) the evolution reaches
    # the sum of the negative single-particle energies
    N = 16
    hop = np.diag(np.full(N - 1, 0.5), 1)
    lev = np.linalg.eigvalsh(hop + hop.T)
    neel = np.zeros((N, 2))
    neel[np.arange(N), np.arange(N) % 2] = 1.0
    e = _evolve_long(mpo.heisenberg_mpo(N, 1.0, 0.0), mps.product_state(neel), 24, 14)
    assert abs(e - np.sum(lev[lev < 0])) < 1e-6 * abs(np.sum(lev[lev < 0]))


def _u0_levels(nb):
    eps, V = inputs.flat_band_bath(nb)
    h1 = np.diag(np.concatenate([[0.0], eps]))
    h1[0, 1:] = h1[1:, 0] = V
    return eps, V, np.linalg.eigvalsh(h1)


def test_long_time_limit_of_the_u0_impurity_is_free_fermions():
    # U = 0, eps_d = 0: the ground energy is twice the sum of the negative
    # levels of the one-body impurity + bath matrix (both spins); a generic
    # product state reaches it
    nb = 7
    eps, V, lev = _u0_levels(nb)
    Ws = mpo.anderson_mpo(0.0, 0.0, eps, V)
    psi = mps.product_state(inputs.random_product_state(nb + 1, 4, 7))
    e = _evolve_long(Ws, psi, 32, 14)
    assert abs(e - 2 * np.sum(lev[lev < 0])) < 1e-6 * abs(2 * np.sum(lev[lev < 0]))


def test_two_site_updates_keep_the_bond_sectors_of_an_occupation_product_state():
    # From a product of occupation states the one-sweep two-site evolution of
    # the star-geometry impurity cannot open the bond sectors that the ground
    # state of its particle sector needs: it settles far above that energy
    # (in exact arithmetic; rounding or a later seed may open them).
    nb = 7
    eps, V, lev = _u0_levels(nb)
    Ws = mpo.anderson_mpo(0.0, 0.0, eps, V)
    occ = np.zeros((nb + 1, 4))
    occ[np.arange(nb + 1), [1, 2] * ((nb + 1) // 2)] = 1.0            # 4 up, 4 down
    e = _evolve_long(Ws, mps.product_state(occ), 32, 8)
    assert e > 2 * np.sum(lev[: (nb + 1) // 2]) + 1.0
