"""METTS on the GPU against the oracle: the Born-rule collapse (same
configuration and probability from the same uniforms, in the computational
and in a rotated basis) and whole chains (energies, observable and drawn
configurations), for the Heisenberg chain and the Anderson impurity (whose
double occupancy is the paper's METTS observable)."""
import numpy as np
import pytest

from oracle import metts as ometts, mpo as ompo, mps as omps, step as ostep
from paper_2606_02930_gb300 import inputs
from paper_2606_02930_gb300._lib import IteError

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


@pytest.mark.parametrize("N,d,chi,rotated", [(10, 2, 16, False), (10, 2, 16, True),
                                             (5, 4, 12, False)])
def test_collapse_matches_oracle(api, ctx, N, d, chi, rotated):
    A = inputs.random_mps(N, d, chi, 70 + N + d)
    basis = ometts.X_BASIS if rotated else None
    rng = np.random.default_rng(5 + d)
    for _ in range(8):
        u = rng.random(N)
        psi = api.mps_create(ctx, A, chi)
        cfg, p = api.mps_sample(ctx, psi, u, basis)
        cfg_o, p_o = ometts.sample(A, u, basis)
        assert cfg == cfg_o
        assert abs(p - p_o) <= 1e-12 * p_o


def _paper_grid(api, tau_max, first=0.01, n=4):
    # the paper's METTS grid: doubling panels of n steps from a first panel of
    # at most [0, first] up to beta/2
    P = int(np.ceil(np.log2(tau_max / first))) + 1
    return api.grid_panels(tau_max, P, n)


def test_collapse_never_takes_a_state_of_zero_probability(api, ctx):
    # amplitudes (a, b, c, 0) on the first site and u the largest double
    # below 1: whether or not rounding leaves the cumulative total below u,
    # the draw takes c (the last state of nonzero probability), never 3
    amp = np.array([1.0486494471372438, 0.41183145201048543, 0.5233264489725756, 0.0])
    A = [amp.astype(complex).reshape(1, 4, 1), np.eye(4)[0].astype(complex).reshape(1, 4, 1)]
    u = [1.0 - 2.0 ** -53, 0.5]
    psi = api.mps_create(ctx, A, 4)
    cfg, p = api.mps_sample(ctx, psi, u)
    cfg_o, p_o = ometts.sample(A, u)
    assert cfg == cfg_o == [2, 0]
    assert abs(p - p_o) <= 1e-12 * p_o


def test_heisenberg_chain_matches_oracle(api, ctx):
    # trapezoid rule on the paper's panel grid with the current-energy shift;
    # the steps keep dtau (s - E0) / 2 <= 0.33 for every product start state,
    # so every local solve is well conditioned
    N, beta = 8, 2.0
    Ws = ompo.heisenberg_mpo(N)
    H = api.mpo_create_heisenberg(ctx, N)
    us = np.random.default_rng(12).random((5, N))
    cfg0 = [0, 1] * (N // 2)
    sz = np.diag([0.5, -0.5]).astype(complex)
    nodes = _paper_grid(api, 0.5 * beta)
    e, vals, cfgs = api.metts(ctx, H, cfg0, nodes, 16, 1e-12, us, alt_basis=ometts.X_BASIS,
                              obs=sz, obs_site=3)
    e_o, vals_o, cfgs_o = ometts.metts_chain(Ws, cfg0, 2, nodes, 5, us, 16, 1e-12, obs=sz,
                                             obs_site=3, scheme="tr", alt_basis=ometts.X_BASIS)
    assert np.allclose(e, e_o, rtol=1e-10, atol=0)
    assert np.allclose(vals, vals_o, rtol=0, atol=1e-10)
    assert cfgs.tolist() == cfgs_o


def test_anderson_chain_double_occupancy_matches_oracle(api, ctx):
    # the paper's METTS setting for the impurity: trapezoid rule, panel grid
    # from [0, 0.01] with 4 steps per panel, shift = the current energy, all
    # non-zero singular values kept below the cap, double occupancy of the
    # impurity as the observable.  This chain is well conditioned (the oracle
    # tests show that 1e-14 noise per step moves it by far less than 1e-10).
    n_bath, beta = 2, 4.0
    eps, V = inputs.flat_band_bath(n_bath)
    Ws = ompo.anderson_mpo(-0.15, 0.3, eps, V)
    H = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15)
    us = np.random.default_rng(13).random((4, n_bath + 1))
    cfg0 = [3, 0, 1]             # doubly occupied impurity, empty, up
    docc = np.diag([0.0, 0.0, 0.0, 1.0]).astype(complex)
    nodes = _paper_grid(api, 0.5 * beta)
    e, vals, cfgs = api.metts(ctx, H, cfg0, nodes, 16, 0.0, us, obs=docc, obs_site=0)
    e_o, vals_o, cfgs_o = ometts.metts_chain(Ws, cfg0, 4, nodes, 4, us, 16, 0.0, obs=docc,
                                             obs_site=0, scheme="tr")
    assert cfgs.tolist() == cfgs_o
    assert np.allclose(e, e_o, rtol=1e-10, atol=0)
    assert np.allclose(vals, vals_o, rtol=0, atol=1e-10)


def _dense(ts):
    v = ts[0]
    for T in ts[1:]:
        v = np.tensordot(v, T, axes=([v.ndim - 1], [0]))
    v = v.reshape(-1)
    return v / np.linalg.norm(v)


def test_anderson_sector_birth_stepwise_parity(api, ctx):
    # An evolution in which sectors enter the bonds from seeds near the
    # truncation cutoff: whole evolutions are ill-conditioned (the step at
    # which a sector enters can flip under rounding), so each GPU step is
    # compared with the oracle's step from the same (GPU) tensors and shift.
    eps, V = inputs.flat_band_bath(3)
    Ws = ompo.anderson_mpo(-0.15, 0.3, eps, V)
    H = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15)
    nodes = _paper_grid(api, 2.0)
    psi0 = ometts.product_tensors([0, 3, 1, 2], 4)
    g = api.mps_create(ctx, psi0, 16)
    s = omps.expect_mpo(psi0, Ws) / omps.norm(psi0) ** 2
    for k in range(1, len(nodes)):
        dt = nodes[k] - nodes[k - 1]
        before = g.tensors()
        ig = api.implicit_step(ctx, H, g, dt, "tr", s, 16, 1e-14)
        o, io = ostep.implicit_step(Ws, before, dt, "tr", s, 16, 1e-14)
        assert abs(ig["energy"] - io.energy) <= 1e-10 * abs(io.energy), k
        assert ig["max_chi"] == max(T.shape[2] for T in o[:-1]), k
        vg, vo = _dense(g.tensors()), _dense(o)
        assert 1.0 - abs(np.vdot(vo, vg)) <= 1e-10, k
        s = ig["energy"]


def test_metts_rejects_invalid_grid(api, ctx):
    H = api.mpo_create_heisenberg(ctx, 4)
    us = np.full((1, 4), 0.5)
    for bad in ([0.1, 0.2, 0.5], [0.0, 0.3, 0.2], [0.0]):
        with pytest.raises(IteError):
            api.metts(ctx, H, [0, 1, 0, 1], bad, 8, 1e-12, us)
