"""Pins of the METTS tier of the oracle: the sequential draw against the dense
probabilities |<sigma|psi>|^2 (exactly, and in frequency), the MPS chain
against the same chain on dense vectors, and the chain's energy average
against the thermal energy Tr(H e^{-beta H}) / Z."""
import numpy as np

from oracle import ed, grid, metts, mpo, mps, step
from paper_2606_02930_gb300 import inputs


def _dense_prob(psi, config, d):
    v = mps.to_dense(psi)
    idx = 0
    for s in config:
        idx = idx * d + s
    return abs(v[idx]) ** 2 / np.vdot(v, v).real


def test_sample_probability_is_the_born_weight():
    rng = np.random.default_rng(3)
    for N, d, chi in ((6, 2, 4), (4, 4, 6)):
        psi = inputs.random_mps(N, d, chi, 11 + N)
        for _ in range(20):
            config, p = metts.sample(psi, rng.random(N))
            assert abs(p - _dense_prob(psi, config, d)) < 1e-13


def test_sample_frequencies_follow_the_distribution():
    N, d = 4, 2
    psi = inputs.random_mps(N, d, 4, 5)
    v = mps.to_dense(psi)
    want = np.abs(v) ** 2 / np.vdot(v, v).real
    rng = np.random.default_rng(9)
    n = 20000
    counts = np.zeros(d ** N)
    for _ in range(n):
        config, _ = metts.sample(psi, rng.random(N))
        counts[int("".join(map(str, config)), 2)] += 1
    sigma = np.sqrt(want * (1 - want) / n)
    assert np.all(np.abs(counts / n - want) <= 5 * sigma + 1e-12)


def test_mps_chain_equals_dense_chain():
    # converged steps at full bond dimension: the MPS chain draws the same
    # configurations and measures the same energies as the dense chain
    N, d, beta = 6, 2, 2.0
    Ws = mpo.heisenberg_mpo(N)
    H = ed.heisenberg_hamiltonian(N)
    rng = np.random.default_rng(21)
    us = rng.random((6, N))
    config0 = [0, 1] * (N // 2)
    nodes = grid.geometric_grid(1e-2, 0.5 * beta, 5)
    e_mps, _, _ = metts.metts_chain(Ws, config0, d, nodes, 6, us, 8, 0.0,
                                    local_tol=1e-13, sweeps=12, sweep_tol=1e-15,
                                    krylov_dim=20)
    e_dense, _ = metts.dense_metts_chain(H, d, N, config0, beta, us, nodes=nodes, scheme="be")
    assert np.allclose(e_mps, e_dense, rtol=0, atol=1e-9)


def _thermal(evals, beta):
    w = np.exp(-beta * (evals - evals[0]))
    return np.sum(evals * w) / np.sum(w)


def _chain_mean_and_error(e, burn=100, block=100):
    e = np.array(e[burn:])
    blocks = e[: len(e) // block * block].reshape(-1, block).mean(axis=1)
    return e.mean(), blocks.std(ddof=1) / np.sqrt(len(blocks))


def test_chain_average_is_the_thermal_energy():
    # The chain samples the thermal ensemble: its energy average approaches
    # Tr(H e^{-beta H}) / Z (exact propagator, dense chain).  Collapsing in
    # the computational basis only, the chain keeps the total S^z of its
    # start state (the Heisenberg chain conserves it), so it samples that
    # sector's ensemble; alternating z and x collapses samples all of it.
    N, d, beta = 4, 2, 1.5
    H = ed.heisenberg_hamiltonian(N)
    rng = np.random.default_rng(33)
    us = rng.random((6000, N))
    sector = [i for i in range(d ** N) if bin(i).count("1") == N // 2]
    e_sector = _thermal(np.linalg.eigvalsh(H[np.ix_(sector, sector)]), beta)
    e, _ = metts.dense_metts_chain(H, d, N, [0, 1, 0, 1], beta, us)
    m, err = _chain_mean_and_error(e)
    assert abs(m - e_sector) < 5 * err
    e, _ = metts.dense_metts_chain(H, d, N, [0, 1, 0, 1], beta, us, alt_basis=metts.X_BASIS)
    m, err = _chain_mean_and_error(e)
    assert abs(m - _thermal(np.linalg.eigvalsh(H), beta)) < 5 * err


def test_mps_chain_with_alternating_basis_equals_dense_chain():
    N, d, beta = 6, 2, 2.0
    Ws = mpo.heisenberg_mpo(N)
    H = ed.heisenberg_hamiltonian(N)
    rng = np.random.default_rng(22)
    us = rng.random((6, N))
    config0 = [0, 1] * (N // 2)
    nodes = grid.geometric_grid(1e-2, 0.5 * beta, 5)
    e_mps, _, _ = metts.metts_chain(Ws, config0, d, nodes, 6, us, 8, 0.0,
                                    alt_basis=metts.X_BASIS, local_tol=1e-13, sweeps=12,
                                    sweep_tol=1e-15, krylov_dim=20)
    e_dense, _ = metts.dense_metts_chain(H, d, N, config0, beta, us, nodes=nodes, scheme="be",
                                         alt_basis=metts.X_BASIS)
    assert np.allclose(e_mps, e_dense, rtol=0, atol=1e-9)


def _in_sector_noise_chain(Ws, cfg, d, nodes, us, cutoff, amp, seed, obs):
    # the chain with every step's site tensors perturbed by amp relative
    # noise on their structurally non-zero entries (what rounding can touch)
    rng = np.random.default_rng(seed)
    orig = step.implicit_step

    def noisy(*a, **k):
        psi, info = orig(*a, **k)
        return [T + amp * np.linalg.norm(T) * (np.abs(T) > 0)
                * (rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape))
                for T in psi], info
    step.implicit_step = noisy
    try:
        return metts.metts_chain(Ws, cfg, d, nodes, len(us), us, 16, cutoff, obs=obs, obs_site=0,
                                 scheme="tr")
    finally:
        step.implicit_step = orig


def _paper_grid(tau_max, first=0.01, n=4):
    P = int(np.ceil(np.log2(tau_max / first))) + 1
    return grid.panel_grid(tau_max, P, n)


def test_anderson_chain_conditioning():
    # The one-sweep two-site evolution of a computational-basis product state
    # of the impurity model can be ill-conditioned: a sector enters the bond
    # spaces only once a seed below the truncation passes it, and the step at
    # which that happens can flip under rounding-size changes of the state.
    # (a) the chain the GPU parity test compares at 1e-10 moves by far less
    # than that under 1e-14 noise per step; (b) a chain with such a birth
    # moves by orders of magnitude more, so element-wise parity is not
    # defined there (the GPU test checks it step by step instead).
    docc = np.diag([0.0, 0.0, 0.0, 1.0]).astype(complex)
    eps, V = inputs.flat_band_bath(2)
    Ws = mpo.anderson_mpo(-0.15, 0.3, eps, V)
    us = np.random.default_rng(13).random((4, 3))
    nodes = _paper_grid(2.0)
    e0, v0, c0 = metts.metts_chain(Ws, [3, 0, 1], 4, nodes, 4, us, 16, 0.0, obs=docc, obs_site=0,
                                   scheme="tr")
    e1, v1, c1 = _in_sector_noise_chain(Ws, [3, 0, 1], 4, nodes, us, 0.0, 1e-14, 1, docc)
    assert c0 == c1
    assert np.max(np.abs(np.array(e1) - e0) / np.abs(e0)) < 1e-10
    eps, V = inputs.flat_band_bath(3)
    Ws = mpo.anderson_mpo(-0.15, 0.3, eps, V)
    us = np.random.default_rng(13).random((4, 4))
    e0, _, _ = metts.metts_chain(Ws, [1, 2, 1, 2], 4, nodes, 4, us, 16, 1e-14, obs=docc,
                                 obs_site=0, scheme="tr")
    e1, _, _ = _in_sector_noise_chain(Ws, [1, 2, 1, 2], 4, nodes, us, 1e-14, 1e-14, 1, docc)
    assert np.max(np.abs(np.array(e1) - e0) / np.abs(e0)) > 1e-6


def test_draw_never_takes_a_state_of_zero_probability():
    # Amplitudes (a, b, c, 0) whose normalised cumulative probabilities round
    # to 1 - 2^-53 in total: with u the largest double below 1 no cumulative
    # probability exceeds u, and the draw must still take a state of nonzero
    # probability (the last one, c), never the empty state 3.
    amp = np.array([1.0486494471372438, 0.41183145201048543, 0.5233264489725756, 0.0])
    psi = [amp.astype(complex).reshape(1, 4, 1)]
    config, p = metts.sample(psi, [1.0 - 2.0 ** -53])
    assert config == [2]
    assert abs(p - amp[2] ** 2 / np.sum(amp ** 2)) < 1e-15


def test_impurity_chain_samples_its_sector_thermal_state():
    # The dense METTS chain of the impurity model (2 bath sites) with
    # collapses in the occupation basis keeps N_up and N_down of its start
    # state; its energy and impurity double occupancy (the paper's METTS
    # observable) average to that sector's thermal values at beta = 8.
    eps, V = inputs.flat_band_bath(2)
    H = ed.anderson_hamiltonian(-0.15, 0.3, eps, V)
    d, N = 4, 3

    def n_up_down(i):
        digits = [(i // d ** (N - 1 - k)) % d for k in range(N)]
        return sum(s in (1, 3) for s in digits), sum(s in (2, 3) for s in digits)

    sector = [i for i in range(d ** N) if n_up_down(i) == (2, 1)]         # start state up, down, up
    docc = np.diag([1.0 if (i // d ** (N - 1)) % d == 3 else 0.0 for i in range(d ** N)])
    beta = 8.0
    ev, U = np.linalg.eigh(H[np.ix_(sector, sector)])
    w = np.exp(-beta * (ev - ev[0]))
    e_th = np.sum(w * ev) / np.sum(w)
    Dsec = docc[np.ix_(sector, sector)]
    d_th = np.sum(w * np.real(np.einsum("ij,ik,kj->j", U.conj(), Dsec, U))) / np.sum(w)
    us = np.random.default_rng(41).random((30000, N))
    e, dd = metts.dense_metts_chain(H, d, N, [1, 2, 1], beta, us, obs_dense=docc)
    m, err = _chain_mean_and_error(e, burn=200, block=500)
    assert abs(m - e_th) < 5 * err and err < 1e-3
    m, err = _chain_mean_and_error(dd, burn=200, block=500)
    assert abs(m - d_th) < 5 * err and err < 1e-3
