"""Pins for the dense tier of the oracle (exact diagonalisation and the
discrete propagators), each against something other than the oracle itself:
closed forms, independent Kronecker-product constructions, free-fermion
spectra and the paper's printed numbers."""
import os
import json
import numpy as np
import pytest

from oracle import ed, grid, mpo
from paper_2606_02930_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SX = np.array([[0, 0.5], [0.5, 0]])
SY = np.array([[0, -0.5j], [0.5j, 0]])
SZ = np.diag([0.5, -0.5])


def kron_site(op, j, N):
    out = np.array([[1.0]])
    for k in range(N):
        out = np.kron(out, op if k == j else np.eye(2))
    return out


def heisenberg_kron(N, J=1.0, Jz=None):
    """Independent construction from Kronecker products of spin matrices."""
    Jz = J if Jz is None else Jz
    H = np.zeros((2 ** N, 2 ** N), complex)
    for j in range(N - 1):
        H += J * (kron_site(SX, j, N) @ kron_site(SX, j + 1, N)
                  + kron_site(SY, j, N) @ kron_site(SY, j + 1, N))
        H += Jz * kron_site(SZ, j, N) @ kron_site(SZ, j + 1, N)
    return H


def test_heisenberg_two_site_closed_form():
    # Heisenberg section: two spins form a singlet (-3J/4) and a triplet (+J/4).
    for J in (1.0, 0.7):
        w = np.linalg.eigvalsh(ed.heisenberg_hamiltonian(2, J))
        assert np.allclose(w, [-0.75 * J, 0.25 * J, 0.25 * J, 0.25 * J], atol=1e-14)
    H = ed.heisenberg_hamiltonian(2)
    singlet = np.array([0, 1, -1, 0]) / np.sqrt(2)          # (|up dn> - |dn up>)/sqrt 2
    assert np.allclose(H @ singlet, -0.75 * singlet, atol=1e-14)


def test_heisenberg_two_site_energy_curve():
    # E(tau) = (-3/4 |c_s|^2 f_s + 1/4 |c_t|^2 f_t) / (|c_s|^2 f_s + |c_t|^2 f_t)
    H = ed.heisenberg_hamiltonian(2)
    psi0 = inputs.random_product_state(2, 2, 7)
    v0 = np.kron(psi0[0], psi0[1])
    singlet = np.array([0, 1, -1, 0]) / np.sqrt(2)
    cs2 = abs(np.vdot(singlet, v0)) ** 2
    ct2 = 1.0 - cs2
    nodes = grid.geometric_grid(1e-2, 1e2, 12)
    dt = grid.steps(nodes)
    for scheme in ("be", "tr"):
        shift = -0.75
        states, _, _ = ed.propagate_discrete(H, v0, dt, scheme, shifts=shift)
        fs, ft = 1.0, 1.0
        for k in range(len(dt)):
            fs *= ed.amplification(dt[k] * (-0.75 - shift), scheme) ** 2
            ft *= ed.amplification(dt[k] * (0.25 - shift), scheme) ** 2
            want = (-0.75 * cs2 * fs + 0.25 * ct2 * ft) / (cs2 * fs + ct2 * ft)
            assert abs(ed.energy(H, states[k]) - want) < 1e-13
    for t, v in zip(nodes[1:], ed.propagate_exact(H, v0, nodes[1:])):
        fs, ft = np.exp(1.5 * t), np.exp(-0.5 * t)
        want = (-0.75 * cs2 * fs + 0.25 * ct2 * ft) / (cs2 * fs + ct2 * ft)
        assert abs(ed.energy(H, v) - want) < 1e-12


@pytest.mark.parametrize("N,Jz", [(3, None), (6, None), (5, 0.0), (4, 0.3)])
def test_heisenberg_matches_kron_construction(N, Jz):
    assert np.abs(ed.heisenberg_hamiltonian(N, 1.0, Jz) - heisenberg_kron(N, 1.0, Jz)).max() < 1e-14


def test_xx_chain_free_fermion_ground_energy():
    # Jz = 0: Jordan-Wigner maps the chain to free fermions with hopping J/2.
    N = 10
    e0 = np.linalg.eigvalsh(ed.heisenberg_hamiltonian(N, 1.0, 0.0))[0]
    t = np.diag(np.full(N - 1, 0.5), 1)
    sp = np.linalg.eigvalsh(t + t.T)
    assert abs(e0 - sp[sp < 0].sum()) < 1e-12


def _subset_sums(levels):
    sums = np.zeros(1)
    for e in levels:
        sums = np.concatenate([sums, sums + e])
    return sums


def test_anderson_u0_spectrum_is_free_fermion():
    # U = 0: every many-body level is a sum of occupied one-body levels, per
    # spin.  Any sign error in the hopping changes this spectrum.
    rng = np.random.default_rng(11)
    eps = rng.uniform(-1, 1, 3)
    V = rng.uniform(0.1, 0.5, 3)
    H = ed.anderson_hamiltonian(0.2, 0.0, eps, V)
    sp = np.linalg.eigvalsh(ed.single_particle_matrix(0.2, eps, V))
    one = _subset_sums(sp)
    want = np.sort((one[:, None] + one[None, :]).ravel())
    assert np.allclose(np.linalg.eigvalsh(H), want, atol=1e-12)


def test_anderson_atomic_limits():
    w = np.linalg.eigvalsh(ed.anderson_hamiltonian(-0.4, 1.3, [], []))
    assert np.allclose(w, sorted([0.0, -0.4, -0.4, 2 * -0.4 + 1.3]), atol=1e-14)
    H = ed.anderson_hamiltonian(-0.4, 1.3, [0.3, -0.2], [0.0, 0.0])
    assert np.abs(H - np.diag(np.diag(H))).max() == 0.0


def test_anderson_conserves_particle_number_and_spin():
    rng = np.random.default_rng(5)
    H = ed.anderson_hamiltonian(-0.15, 0.3, rng.uniform(-1, 1, 3), rng.uniform(0.1, 0.4, 3))
    n_sites = 4
    dim = 4 ** n_sites
    nup = np.zeros(dim)
    ndn = np.zeros(dim)
    for idx in range(dim):
        for k in range(n_sites):
            loc = (idx >> (2 * (n_sites - 1 - k))) & 3
            nup[idx] += loc & 1
            ndn[idx] += loc >> 1
    assert np.abs(H * (nup[:, None] - nup[None, :])).max() == 0.0
    assert np.abs(H * (ndn[:, None] - ndn[None, :])).max() == 0.0
    assert np.abs(H - H.T).max() == 0.0


def test_mpo_heisenberg_equals_ed():
    for N, Jz in ((2, None), (5, None), (7, 0.0), (6, 0.45)):
        Hm = mpo.mpo_to_dense(mpo.heisenberg_mpo(N, 1.0, Jz))
        assert np.abs(Hm - ed.heisenberg_hamiltonian(N, 1.0, Jz)).max() < 1e-14


def test_mpo_anderson_equals_ed():
    rng = np.random.default_rng(3)
    for nb in (1, 2, 4):
        eps, V = rng.uniform(-1, 1, nb), rng.uniform(0.05, 0.5, nb)
        Hm = mpo.mpo_to_dense(mpo.anderson_mpo(-0.2, 0.7, eps, V))
        assert np.abs(Hm - ed.anderson_hamiltonian(-0.2, 0.7, eps, V)).max() < 1e-14


def test_a_stability_and_forward_euler():
    # App. A: |R(z)| <= 1 on z >= 0 for the implicit schemes; forward Euler
    # leaves the unit disk once z > 2.
    z = np.concatenate([np.linspace(0, 10, 1001), np.logspace(1, 8, 200)])
    assert np.all(np.abs(ed.amplification(z, "be")) <= 1.0)
    assert np.all(np.abs(ed.amplification(z, "tr")) <= 1.0)
    fe = np.abs(ed.amplification(z, "fe"))
    assert np.all(fe[z <= 2.0] <= 1.0 + 1e-15) and np.all(fe[z > 2.0 + 1e-12] > 1.0)


def test_forward_euler_blows_up_on_log_grid():
    # App. A: once dtau * Lambda > 2 the explicit scheme amplifies the top
    # mode; the implicit schemes stay bounded on the same grid (shift = E0).
    N = 8
    H = ed.heisenberg_hamiltonian(N)
    w = np.linalg.eigvalsh(H)
    psi = inputs.random_product_state(N, 2, 1)
    v0 = psi[0]
    for k in range(1, N):
        v0 = np.kron(v0, psi[k])
    dt = grid.steps(grid.geometric_grid(1e-2, 1e2, 20))
    _, fe_norms, _ = ed.propagate_discrete(H, v0, dt, "fe", shifts=w[0], normalize=False)
    lam = w[-1] - w[0]
    crossed = dt * lam > 2.0
    assert crossed.any()
    assert fe_norms[-1] > 1e6
    for scheme in ("be", "tr"):
        _, norms, _ = ed.propagate_discrete(H, v0, dt, scheme, shifts=w[0], normalize=False)
        assert max(norms) <= 1.0 + 1e-12


def test_trapezoid_second_order_on_panel_grid():
    # Heisenberg section: doubling n (steps per panel) cuts the error ~4x.
    N = 8
    H = ed.heisenberg_hamiltonian(N)
    e0 = np.linalg.eigvalsh(H)[0]
    psi = inputs.random_product_state(N, 2, 2)
    v0 = psi[0]
    for k in range(1, N):
        v0 = np.kron(v0, psi[k])
    tau_max, P = 8.0, 8
    errs = []
    for n in (4, 8, 16):
        nodes = grid.panel_grid(tau_max, P, n)
        states, _, _ = ed.propagate_discrete(H, v0, grid.steps(nodes), "tr", shifts=e0)
        exact = ed.propagate_exact(H, v0, [tau_max])[0]
        errs.append(np.linalg.norm(states[-1] - exact * np.exp(1j * np.angle(np.vdot(exact, states[-1])))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5


def test_backward_euler_first_order():
    N = 6
    H = ed.heisenberg_hamiltonian(N)
    e0 = np.linalg.eigvalsh(H)[0]
    psi = inputs.random_product_state(N, 2, 4)
    v0 = psi[0]
    for k in range(1, N):
        v0 = np.kron(v0, psi[k])
    errs = []
    for n in (16, 32):
        nodes = grid.panel_grid(4.0, 6, n)
        states, _, _ = ed.propagate_discrete(H, v0, grid.steps(nodes), "be", shifts=e0)
        exact = ed.propagate_exact(H, v0, [4.0])[0]
        errs.append(np.linalg.norm(states[-1] - exact * np.exp(1j * np.angle(np.vdot(exact, states[-1])))))
    assert 1.8 < errs[0] / errs[1] < 2.2


def test_trapezoid_local_error_closed_form_and_paper_maximum():
    # App. A: with a = h = 2^k, b = 2^(k+1): E(mu) = e^{-3mu/2}(mu cosh(mu/2) - 2 sinh(mu/2)),
    # bounded, maximum ~0.04 near mu ~ 2.1, independent of k.
    with open(os.path.join(GOLDEN, "trapezoid_local_error.json")) as f:
        gold = json.load(f)
    mu = np.linspace(1e-3, 30, 300001)
    for k in (-3, 0, 4):
        h = 2.0 ** k
        lam = mu / h
        e = ed.trapezoid_local_error(lam, h, 2 * h)
        closed = np.exp(-1.5 * mu) * (mu * np.cosh(mu / 2) - 2 * np.sinh(mu / 2))
        assert np.allclose(e, closed, atol=1e-14)
        i = np.argmax(e)
        assert abs(e[i] - gold["max_value"]) <= gold["value_tol"]
        assert abs(mu[i] - gold["argmax_mu"]) <= gold["argmax_tol"]


def test_grids():
    nodes = grid.panel_grid(16.0, 4, 2)
    assert np.allclose(nodes, [0, 1, 2, 3, 4, 6, 8, 12, 16])
    g = grid.geometric_grid(1e-2, 1e2, 20)
    assert g[0] == 0.0 and abs(g[1] - 1e-2) < 1e-18 and abs(g[-1] - 1e2) < 1e-12
    r = g[2:] / g[1:-1]
    assert np.allclose(r, r[0]) and abs(r[0] - 10 ** (4 / 19)) < 1e-12


def test_backward_euler_energy_monotone_dense():
    # R_BE(lambda - s) is positive and decreasing on the spectrum when s <= E0,
    # so each step lowers the Rayleigh quotient.
    N = 8
    H = ed.heisenberg_hamiltonian(N)
    e0 = np.linalg.eigvalsh(H)[0]
    psi = inputs.random_product_state(N, 2, 9)
    v0 = psi[0]
    for k in range(1, N):
        v0 = np.kron(v0, psi[k])
    dt = grid.steps(grid.geometric_grid(1e-2, 1e2, 20))
    states, _, _ = ed.propagate_discrete(H, v0, dt, "be", shifts=e0)
    es = [ed.energy(H, v0)] + [ed.energy(H, v) for v in states]
    assert all(b <= a + 1e-13 for a, b in zip(es, es[1:]))


def _collocation_amplification(z, A, b):
    """Runge-Kutta stability function R(z) = 1 - z b^T (I + z A)^{-1} 1 of a
    Butcher tableau (A, b), for y' = -lambda y at z = lambda dtau."""
    A = np.asarray(A, float)
    one = np.ones(len(b))
    return np.array([1.0 - zz * np.asarray(b) @ np.linalg.solve(np.eye(len(b)) + zz * A, one)
                     for zz in np.atleast_1d(z)])


def test_gauss_legendre_amplification_equals_collocation_tableau():
    # 2- and 3-stage Gauss-Legendre collocation tableaux (nodes at the
    # Legendre roots on [0, 1]); their stability functions are the
    # diagonal Pade approximants of e^{-z}
    r3, r15 = np.sqrt(3.0), np.sqrt(15.0)
    A2 = [[0.25, 0.25 - r3 / 6], [0.25 + r3 / 6, 0.25]]
    b2 = [0.5, 0.5]
    A3 = [[5 / 36, 2 / 9 - r15 / 15, 5 / 36 - r15 / 30],
          [5 / 36 + r15 / 24, 2 / 9, 5 / 36 - r15 / 24],
          [5 / 36 + r15 / 30, 2 / 9 + r15 / 15, 5 / 36]]
    b3 = [5 / 18, 4 / 9, 5 / 18]
    z = np.array([1e-3, 0.1, 0.7, 2.0, 9.0, 60.0, 1e4])
    assert np.allclose(ed.amplification(z, "gl2"), _collocation_amplification(z, A2, b2),
                       rtol=1e-12, atol=1e-15)
    assert np.allclose(ed.amplification(z, "gl3"), _collocation_amplification(z, A3, b3),
                       rtol=1e-12, atol=1e-15)
    # one stage is the implicit midpoint rule, i.e. the trapezoid amplification
    assert np.allclose(ed.amplification(z, "gl1"), ed.amplification(z, "tr"), rtol=1e-15)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_gauss_legendre_order_and_a_stability(q):
    # local error e^{-z} - R_q(z) = O(z^{2q+1}): halving z divides it by 2^{2q+1}
    z = np.array([0.08, 0.04])
    err = np.abs(np.exp(-z) - ed.amplification(z, f"gl{q}"))
    assert abs(np.log2(err[0] / err[1]) - (2 * q + 1)) < 0.1
    # A-stability: |R| <= 1 on the closed right half plane, |R| = 1 on the axis
    x, y = np.meshgrid(np.linspace(0, 50, 41), np.linspace(-50, 50, 41))
    zz = x + 1j * y
    assert np.all(np.abs(ed.amplification(zz, f"gl{q}")) <= 1 + 1e-12)
    assert np.allclose(np.abs(ed.amplification(1j * np.linspace(-40, 40, 17), f"gl{q}")), 1.0)
    # partial fractions reproduce the rational function
    zp, a, r_inf = ed.pade_partial_fractions(q)
    t = np.array([0.3, 2.0, 17.0, 1e3])
    assert np.allclose(r_inf + sum(aj / (t - zj) for zj, aj in zip(zp, a)),
                       ed.amplification(t, f"gl{q}"), rtol=1e-12, atol=1e-14)


def test_heun_amplification_and_its_instability():
    # Heun's stability function from its two stages: predictor y* = y - z y,
    # corrector y_1 = y - (z/2)(y + y*)
    z = np.linspace(0.0, 5.0, 51)
    pred = 1.0 - z
    assert np.allclose(ed.amplification(z, "heun"), 1.0 - 0.5 * z * (1.0 + pred), rtol=1e-15)
    # second order, and unstable once z exceeds 2 (the critical step of the
    # stability section: dtau * E_max = 2)
    zz = np.array([0.02, 0.01])
    err = np.abs(np.exp(-zz) - ed.amplification(zz, "heun"))
    assert abs(np.log2(err[0] / err[1]) - 3.0) < 0.1
    r = np.abs(ed.amplification(z, "heun"))
    assert np.all(r[z <= 2.0] <= 1.0 + 1e-15) and np.all(r[z > 2.0] > 1.0)
