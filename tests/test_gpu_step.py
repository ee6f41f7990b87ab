"""GPU parity of whole implicit steps and evolutions against the oracle, and
the measurements (energy, overlap, correlators).

FP64 mode bar: relative energy error <= 1e-10 and infidelity <= 1e-10 against
the oracle run with identical options (same algorithm, same truncation rule)."""
import numpy as np
import pytest

from oracle import ed, grid as ogrid, linsolve as ls, mpo as ompo, mps as omps, step as ostep
from paper_2606_02930_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02930_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def ctx(api):
    return api.ctx_create(0)


def infid(a_tensors, b_tensors):
    ov = omps.overlap(a_tensors, b_tensors)
    return 1.0 - abs(ov) / (omps.norm(a_tensors) * omps.norm(b_tensors))


def run_pair(api, ctx, Ws, H, psi0_tensors, nodes, scheme, chi, cutoff, shift_mode="fixed",
             shift=0.0, opts=None, okw=None):
    """Step the oracle and the library side by side; yield per-step pairs."""
    okw = okw or {}
    psi = api.mps_create(ctx, psi0_tensors, chi)
    ost = omps.copy(psi0_tensors)
    nrm = omps.norm(ost)
    ost[0] = ost[0] / nrm
    psi.set(ost)
    s_o = omps.expect_mpo(ost, Ws) if shift_mode == "energy" else shift
    s_g = api.energy(ctx, H, psi) if shift_mode == "energy" else shift
    out = []
    for k in range(1, len(nodes)):
        dt = nodes[k] - nodes[k - 1]
        ost, oinfo = ostep.implicit_step(Ws, ost, dt, scheme, s_o, chi, cutoff, **okw)
        ginfo = api.implicit_step(ctx, H, psi, dt, scheme, s_g, chi, cutoff, opts)
        out.append((ost, oinfo, psi.tensors(), ginfo))
        if shift_mode == "energy":
            s_o, s_g = oinfo.energy, ginfo["energy"]
    return out


def test_heisenberg_n10_backward_euler_fixed_mode(api, ctx):
    # N=10, J=1, chi_max=32 (exact), cutoff 0, backward Euler on the geometric
    # grid 1e-2 -> 1e2 with 20 steps, shift = exact E0
    N = 10
    Ws = ompo.heisenberg_mpo(N)
    e0 = np.linalg.eigvalsh(ed.heisenberg_hamiltonian(N))[0]
    H = api.mpo_create_heisenberg(ctx, N)
    psi0 = omps.product_state(inputs.random_product_state(N, 2, 1000))
    nodes = ogrid.geometric_grid(1e-2, 1e2, 20)
    pairs = run_pair(api, ctx, Ws, H, psi0, nodes, "be", 32, 0.0, shift=e0)
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * abs(oinfo.energy)
        assert infid(ost, gst) <= TOL
        assert abs(ginfo["norm_before"] - oinfo.norm_before) <= 1e-10
        assert ginfo["max_chi"] == oinfo.max_chi
        assert ginfo["gmres_steps"] == oinfo.gmres_steps
    es = [g["energy"] for _, _, _, g in pairs]
    assert all(b <= a + 1e-10 for a, b in zip(es, es[1:]))


def test_restarted_gmres_steps_match_oracle(api, ctx):
    # three GMRES(4) cycles per local solve, each restarted from the last
    # iterate, on N = 10 with the trapezoid rule: the same states, energies
    # and Arnoldi step counts as the oracle's restarted solve
    N = 10
    Ws = ompo.heisenberg_mpo(N)
    e0 = np.linalg.eigvalsh(ed.heisenberg_hamiltonian(N))[0]
    H = api.mpo_create_heisenberg(ctx, N)
    psi0 = omps.product_state(inputs.random_product_state(N, 2, 1001))
    nodes = ogrid.geometric_grid(1e-2, 1e1, 6)
    opts = api.solver_opts(krylov_dim=4, max_cycles=3)
    pairs = run_pair(api, ctx, Ws, H, psi0, nodes, "tr", 32, 0.0, shift=e0, opts=opts,
                     okw=dict(krylov_dim=4, max_cycles=3))
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * abs(oinfo.energy)
        assert infid(ost, gst) <= TOL
        assert ginfo["gmres_steps"] == oinfo.gmres_steps
    assert max(o.gmres_steps for _, o, _, _ in pairs) > 2 * (N - 1) * 4   # restarts ran


def test_heisenberg_n10_evolve_loggrid_equals_steps(api, ctx):
    N = 10
    e0 = np.linalg.eigvalsh(ed.heisenberg_hamiltonian(N))[0]
    H = api.mpo_create_heisenberg(ctx, N)
    vecs = inputs.random_product_state(N, 2, 1000)
    psi = api.mps_create_product(ctx, vecs, 32)
    nodes, infos = api.evolve_loggrid(ctx, H, psi, 1e-2, 1e2, 20, "be", 32, 0.0, shift0=e0)
    assert np.allclose(nodes, ogrid.geometric_grid(1e-2, 1e2, 20), rtol=1e-15)
    Ws = ompo.heisenberg_mpo(N)
    states, oinfos = ostep.evolve(Ws, omps.product_state(vecs), nodes, "be", 32, 0.0, shift=e0)
    for g, o in zip(infos, oinfos):
        assert abs(g["energy"] - o.energy) <= TOL * abs(o.energy)
    assert infid(states[-1], psi.tensors()) <= TOL


def test_converged_mode_equals_dense_propagator(api, ctx):
    # converged sweeps at full bond dimension solve each step exactly:
    # prod_k R_BE(dtau_k (H - E0)) psi0 from exact diagonalisation
    N = 8
    Hd = ed.heisenberg_hamiltonian(N)
    e0 = np.linalg.eigvalsh(Hd)[0]
    H = api.mpo_create_heisenberg(ctx, N)
    vecs = inputs.random_product_state(N, 2, 1001)
    v0 = omps.to_dense(omps.product_state(vecs))
    nodes = ogrid.geometric_grid(1e-2, 1e2, 20)[:8]
    for scheme in ("be", "tr"):
        dense, _, _ = ed.propagate_discrete(Hd, v0, ogrid.steps(nodes), scheme, shifts=e0)
        psi = api.mps_create_product(ctx, vecs, 16)
        opts = api.solver_opts(krylov_dim=20, sweeps=12, local_tol=1e-13, sweep_tol=1e-15,
                               fit_sweeps=6)
        for k in range(1, len(nodes)):
            api.implicit_step(ctx, H, psi, nodes[k] - nodes[k - 1], scheme, e0, 16, 0.0, opts)
            assert ed.infidelity(dense[k - 1], omps.to_dense(psi.tensors())) <= TOL


def test_heisenberg_trapezoid_fixed_mode(api, ctx):
    N = 10
    Ws = ompo.heisenberg_mpo(N)
    H = api.mpo_create_heisenberg(ctx, N)
    psi0 = omps.product_state(inputs.random_product_state(N, 2, 1002))
    nodes = ogrid.geometric_grid(1e-2, 1e2, 20)[:10]
    pairs = run_pair(api, ctx, Ws, H, psi0, nodes, "tr", 32, 1e-10, shift_mode="energy")
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * abs(oinfo.energy)
        assert infid(ost, gst) <= TOL


@pytest.mark.parametrize("scheme", ["be", "tr"])
def test_anderson_fixed_mode(api, ctx, scheme):
    nb = 5
    eps, V = inputs.flat_band_bath(nb)
    Ws = ompo.anderson_mpo(-0.15, 0.3, eps, V)
    H = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15)
    psi0 = omps.product_state(inputs.random_product_state(nb + 1, 4, 3000))
    nodes = ogrid.geometric_grid(1e-2, 1e4, 50)[:12]
    pairs = run_pair(api, ctx, Ws, H, psi0, nodes, scheme, 64, 1e-14, shift_mode="energy")
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * abs(oinfo.energy)
        assert infid(ost, gst) <= TOL


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("scheme", ["be", "tr"])
def test_saturated_input_one_step(api, ctx, scheme, precision):
    # a full-bond-dimension random input (chi = 64 in the bulk of N = 20); in
    # fp64_tc mode the bulk contractions run on the tensor cores
    N, chi = 20, 64
    Ws = ompo.heisenberg_mpo(N)
    H = api.mpo_create_heisenberg(ctx, N)
    A = inputs.random_isometric_mps(N, 2, chi, 2001)
    pairs = run_pair(api, ctx, Ws, H, A, np.array([0.0, 0.5, 3.0]), scheme, chi, 1e-10,
                     shift_mode="energy", opts=api.solver_opts(precision=precision))
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * abs(oinfo.energy)
        assert infid(ost, gst) <= TOL


@pytest.mark.parametrize("scheme", ["be", "tr"])
def test_tensor_core_mode_matches_oracle_chi128(api, ctx, scheme):
    # N = 16, chi = 128 (the bulk two-site blocks are 256 x 256): one step in
    # fp64_tc mode against the oracle, FP64 bar
    N, chi = 16, 128
    Ws = ompo.heisenberg_mpo(N)
    H = api.mpo_create_heisenberg(ctx, N)
    A = inputs.random_isometric_mps(N, 2, chi, 2002)
    pairs = run_pair(api, ctx, Ws, H, A, np.array([0.0, 0.2]), scheme, chi, 1e-10,
                     shift_mode="energy", opts=api.solver_opts(precision="fp64_tc"))
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * abs(oinfo.energy)
        assert infid(ost, gst) <= TOL


@pytest.mark.parametrize("scheme", ["be", "tr"])
def test_tensor_core_mode_anderson(api, ctx, scheme):
    nb = 5
    eps, V = inputs.flat_band_bath(nb)
    Ws = ompo.anderson_mpo(-0.15, 0.3, eps, V)
    H = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15)
    A = inputs.random_isometric_mps(nb + 1, 4, 64, 3001)
    pairs = run_pair(api, ctx, Ws, H, A, np.array([0.0, 0.1, 1.0]), scheme, 64, 1e-14,
                     shift_mode="energy", opts=api.solver_opts(precision="fp64_tc"))
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * abs(oinfo.energy)
        assert infid(ost, gst) <= TOL


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_workload_size_step_invariants(api, ctx, precision):
    # N = 64, chi_max = 256, cutoff 1e-10, saturated random input: one backward
    # Euler step with a certified lower bound s <= E0 must not raise the energy
    # (R_BE positive and decreasing on the spectrum) and must not grow the norm.
    N, chi = 64, 256
    H = api.mpo_create_heisenberg(ctx, N)
    A = inputs.random_isometric_mps(N, 2, chi, 2000)
    psi = api.mps_create(ctx, A, chi)
    e_in = api.energy(ctx, H, psi)
    s = -0.75 * (N - 1)
    info = api.implicit_step(ctx, H, psi, 0.1, "be", s, chi, 1e-10,
                             api.solver_opts(precision=precision))
    assert info["energy"] < e_in
    assert abs(info["energy"] - api.energy(ctx, H, psi)) < 1e-10 * abs(info["energy"])
    chis, _ = psi.bond_dims()
    assert chis.max() <= chi and chis[0] == 1 and chis[-1] == 1


def test_measurements_match_oracle(api, ctx):
    N = 9
    A = inputs.random_mps(N, 2, 8, 55)
    psi = api.mps_create(ctx, A, 8)
    H = api.mpo_create_heisenberg(ctx, N, 1.0, 0.6)
    Ws = ompo.heisenberg_mpo(N, 1.0, 0.6)
    assert abs(api.energy(ctx, H, psi) - omps.expect_mpo(A, Ws)) < 1e-12 * N
    B = inputs.random_mps(N, 2, 5, 56)
    phi = api.mps_create(ctx, B, 8)
    assert abs(api.overlap(ctx, phi, psi) - omps.overlap(B, A)) < 1e-12 * abs(omps.overlap(B, A)) + 1e-15
    for (i, j) in ((0, 5), (3, 3), (2, 8)):
        got = api.correlator(ctx, psi, ompo.SZ, i, ompo.SP, j)
        want = omps.correlator(A, ompo.SZ, i, ompo.SP, j)
        assert abs(got - want) < 1e-12
    # fermions: <c^dag_up,i c_up,j> with the Jordan-Wigner string, and <n_up n_down>
    Af = inputs.random_mps(5, 4, 6, 57)
    pf = api.mps_create(ctx, Af, 16)
    O = ompo.C_UP.T @ ompo.F_PAR
    got = api.correlator(ctx, pf, O, 1, ompo.C_UP, 4, ompo.F_PAR)
    want = omps.correlator(Af, O, 1, ompo.C_UP, 4, string=ompo.F_PAR)
    assert abs(got - want) < 1e-12
    got = api.correlator(ctx, pf, ompo.N_UP, 0, ompo.N_DN, 0)
    want = omps.correlator(Af, ompo.N_UP, 0, ompo.N_DN, 0)
    assert abs(got - want) < 1e-12


def test_mpo_builders_match_oracle_dense(api, ctx):
    # the library's built-in MPOs give the oracle's energies on random states
    A = inputs.random_mps(6, 4, 10, 58)
    eps, V = inputs.flat_band_bath(5)
    Ha = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15)
    psi = api.mps_create(ctx, A, 16)
    want = omps.expect_mpo(A, ompo.anderson_mpo(-0.15, 0.3, eps, V))
    assert abs(api.energy(ctx, Ha, psi) - want) < 1e-12 * max(1.0, abs(want))


def test_edge_cases(api, ctx):
    from paper_2606_02930_gb300._lib import IteError
    # two sites: a single bond, swept twice
    Ws = ompo.heisenberg_mpo(2)
    H = api.mpo_create_heisenberg(ctx, 2)
    psi0 = omps.product_state(inputs.random_product_state(2, 2, 5))
    pairs = run_pair(api, ctx, Ws, H, psi0, np.array([0.0, 0.1, 1.0, 10.0]), "be", 2, 0.0,
                     shift=-0.75)
    for ost, oinfo, gst, ginfo in pairs:
        assert infid(ost, gst) <= TOL
    # N = 2 closed form: singlet -3/4, triplet +1/4, each weighted by the
    # squared product of backward-Euler factors 1/(1 + dtau (lambda - s))
    v0 = omps.to_dense(psi0)
    singlet = np.array([0, 1, -1, 0]) / np.sqrt(2)
    cs2 = abs(np.vdot(singlet, v0)) ** 2 / np.vdot(v0, v0).real
    fs = ft = 1.0
    for k, dt in enumerate((0.1, 0.9, 9.0)):
        fs /= (1.0 + dt * (-0.75 + 0.75)) ** 2
        ft /= (1.0 + dt * (0.25 + 0.75)) ** 2
        want = (-0.75 * cs2 * fs + 0.25 * (1 - cs2) * ft) / (cs2 * fs + (1 - cs2) * ft)
        assert abs(pairs[k][3]["energy"] - want) < 1e-12
    # chi_max = 1 keeps a product state
    N = 6
    H6 = api.mpo_create_heisenberg(ctx, N)
    psi = api.mps_create_product(ctx, inputs.random_product_state(N, 2, 6), 4)
    api.implicit_step(ctx, H6, psi, 0.5, "be", 0.0, 1, 0.0)
    assert psi.bond_dims()[0].max() == 1
    # invalid requests fail cleanly and leave the state unchanged
    before = psi.tensors()
    with pytest.raises(IteError):
        api.implicit_step(ctx, H6, psi, 0.5, "be", 0.0, 99, 0.0)   # above capacity
    with pytest.raises(IteError):
        api.implicit_step(ctx, H6, psi, -1.0, "be", 0.0, 2, 0.0)
    with pytest.raises(IteError):
        api.implicit_step(ctx, H, psi, 0.5, "be", 0.0, 2, 0.0)     # MPO length mismatch
    after = psi.tensors()
    assert all(np.array_equal(a, b) for a, b in zip(before, after))
    # non-finite input is reported, not propagated silently
    bad = [T.copy() for T in before]
    bad[2][0, 0, 0] = np.nan
    psi_bad = api.mps_create(ctx, bad, 4)
    with pytest.raises(IteError) as ei:
        api.implicit_step(ctx, H6, psi_bad, 0.5, "be", 0.0, 4, 0.0)
    assert ei.value.status in (3, 6)

@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_rank_deficient_start_takes_the_svd_gauge(api, ctx, precision):
    # A start state whose bond 3 carries two identical directions (rank 1 on
    # a bond of dimension 2) and whose bond 5 carries an exactly zero
    # direction: the gauge move must drop them as the oracle's SVD does (the
    # LQ fast path cannot certify full rank there), and the fixed-mode step
    # must then match the oracle.  Full-rank bonds take the LQ path.
    N = 8
    rng = np.random.default_rng(77)
    chis = [1, 2, 4, 2, 4, 2, 4, 2, 1]
    A = []
    for i in range(N):
        g = rng.standard_normal((chis[i], 2, chis[i + 1], 2))
        A.append(g[..., 0] + 1j * g[..., 1])
    A[2][:, :, 1] = A[2][:, :, 0]
    A[4][:, :, 1] = 0.0
    Ws = ompo.heisenberg_mpo(N)
    H = api.mpo_create_heisenberg(ctx, N)
    opts = api.solver_opts(precision=precision)
    nodes = ogrid.geometric_grid(1e-1, 1e1, 3)
    pairs = run_pair(api, ctx, Ws, H, A, nodes, "be", 16, 0.0, shift_mode="energy", opts=opts)
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * abs(oinfo.energy)
        assert infid(ost, gst) <= TOL
        assert ginfo["max_chi"] == oinfo.max_chi


@pytest.mark.parametrize("scheme,precision", [("gl2", "fp64"), ("gl3", "fp64"), ("gl2", "fp64_tc")])
def test_gauss_legendre_fixed_mode(api, ctx, scheme, precision):
    # the paper's Gauss-Legendre step (q complex-shifted solves and the fit of
    # their combination), fixed effort, against the oracle step by step
    N = 10
    Ws = ompo.heisenberg_mpo(N)
    H = api.mpo_create_heisenberg(ctx, N)
    psi0 = omps.product_state(inputs.random_product_state(N, 2, 1000))
    nodes = ogrid.geometric_grid(1e-2, 1e2, 8)
    pairs = run_pair(api, ctx, Ws, H, psi0, nodes, scheme, 24, 1e-12, shift_mode="energy",
                     opts=api.solver_opts(precision=precision))
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * abs(oinfo.energy)
        assert infid(ost, gst) <= TOL
        assert abs(ginfo["norm_before"] - oinfo.norm_before) <= 1e-10
        assert ginfo["max_chi"] == oinfo.max_chi
        assert ginfo["gmres_steps"] == oinfo.gmres_steps


def test_gauss_legendre_converged_equals_dense_propagator(api, ctx):
    # converged solves and fit at full bond dimension: the step is exactly
    # R_q(dtau (H - E0)) with R_q the (q, q) Pade approximant of e^{-z}
    N = 8
    H = api.mpo_create_heisenberg(ctx, N)
    Hd = ed.heisenberg_hamiltonian(N)
    e0 = np.linalg.eigvalsh(Hd)[0]
    sv = inputs.random_product_state(N, 2, 1000)
    v0 = sv[0]
    for k in range(1, N):
        v0 = np.kron(v0, sv[k])
    nodes = ogrid.geometric_grid(1e-2, 1e2, 6)
    for scheme in ("gl2", "gl3"):
        dense, _, _ = ed.propagate_discrete(Hd, v0, ogrid.steps(nodes), scheme, shifts=e0)
        psi = api.mps_create(ctx, omps.product_state(sv), 16)
        opts = api.solver_opts(local_tol=1e-13, sweeps=12, sweep_tol=1e-15, fit_sweeps=6,
                               krylov_dim=20)
        _, infos = api.evolve_loggrid(ctx, H, psi, 1e-2, 1e2, 6, scheme, 16, 0.0,
                                      shift0=e0, opts=opts)
        for v, info in zip(dense, infos):
            assert abs(ed.energy(Hd, v) - info["energy"]) <= 1e-10 * abs(ed.energy(Hd, v))
        assert ed.infidelity(dense[-1], omps.to_dense(psi.tensors())) <= 1e-10


@pytest.mark.parametrize("scheme", ["fe", "heun"])
def test_explicit_steps_match_oracle_and_blow_up(api, ctx, scheme):
    # the explicit counter-examples on a growing log grid: parity with the
    # oracle step by step, and growth of the norm (|R| > 1) once the step
    # passes the critical size dtau (E_max - s) = 2
    N = 8
    Ws = ompo.heisenberg_mpo(N)
    Hd = ed.heisenberg_hamiltonian(N)
    ev = np.linalg.eigvalsh(Hd)
    H = api.mpo_create_heisenberg(ctx, N)
    psi0 = omps.product_state(inputs.random_product_state(N, 2, 1002))
    nodes = ogrid.geometric_grid(1e-2, 2.0, 8)
    pairs = run_pair(api, ctx, Ws, H, psi0, nodes, scheme, 16, 0.0, shift=ev[0],
                     opts=api.solver_opts(fit_sweeps=2), okw=dict(fit_sweeps=2))
    grew = False
    amp = 1.0      # bound on how much an unstable step can amplify rounding differences
    for k, (ost, oinfo, gst, ginfo) in enumerate(pairs):
        dt = nodes[k + 1] - nodes[k]
        z_max = dt * (ev[-1] - ev[0])
        amp *= max(1.0, abs(float(ed.amplification(z_max, scheme))))
        assert abs(ginfo["energy"] - oinfo.energy) <= TOL * amp * max(abs(oinfo.energy), 1.0)
        assert infid(ost, gst) <= TOL * amp ** 2
        assert abs(ginfo["norm_before"] - oinfo.norm_before) <= 1e-10 * amp * max(oinfo.norm_before, 1.0)
        if z_max > 2.5:
            grew = grew or ginfo["norm_before"] > 1.0
        elif z_max <= 2.0:
            assert ginfo["norm_before"] <= 1.0 + 1e-12
    assert grew


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc", "mixed_bf16"])
def test_anderson_reduced_bath_saturated_step(api, ctx, precision):
    # the impurity workload on a reduced bath: impurity + 10 bath sites
    # (N = 11, d = 4, MPO bond dimension 6), flat band Gamma = 0.05,
    # U = 0.3, eps_d = -U/2, cutoff 1e-14, chi = 64 saturated (random
    # isometries), backward Euler dtau = 0.05 with the energy shift; the fixed
    # modes against the oracle's fixed-effort step (1e-10), the mixed mode
    # against its converged step (1e-8)
    nb, chi, cutoff, dt = 10, 64, 1e-14, 0.05
    eps, V = inputs.flat_band_bath(nb)
    Ws = ompo.anderson_mpo(-0.15, 0.3, eps, V)
    H = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15)
    A = inputs.random_isometric_mps(nb + 1, 4, chi, 3002)
    mixed = precision.startswith("mixed")
    okw = dict(local_tol=1e-12, max_cycles=100) if mixed else {}
    opts = (api.solver_opts(precision=precision, refine_tol=1e-11, refine_max=20) if mixed
            else api.solver_opts(precision=precision))
    pairs = run_pair(api, ctx, Ws, H, A, np.array([0.0, dt]), "be", chi, cutoff,
                     shift_mode="energy", opts=opts, okw=okw)
    bar = 1e-8 if mixed else TOL
    for ost, oinfo, gst, ginfo in pairs:
        assert abs(ginfo["energy"] - oinfo.energy) <= bar * abs(oinfo.energy)
        assert infid(ost, gst) <= bar
        assert ginfo["max_chi"] == oinfo.max_chi
