"""METTS on the GPU against the oracle: the Born-rule collapse (same
configuration and probability from the same uniforms, in the computational
and in a rotated basis) and whole chains (energies, observable and drawn
configurations), for the Heisenberg chain and the Anderson impurity (whose
double occupancy is the paper's METTS observable)."""
import numpy as np
import pytest

from oracle import ed, metts as ometts, mpo as ompo
from paper_2606_02930_gb300 import inputs

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


def test_heisenberg_chain_matches_oracle(api, ctx):
    N, beta = 8, 2.0
    Ws = ompo.heisenberg_mpo(N)
    H = api.mpo_create_heisenberg(ctx, N)
    us = np.random.default_rng(12).random((5, N))
    cfg0 = [0, 1] * (N // 2)
    sz = np.diag([0.5, -0.5]).astype(complex)
    # a fixed shift at the ground energy keeps every solve positive definite
    e0 = np.linalg.eigvalsh(ed.heisenberg_hamiltonian(N))[0]
    e, vals, cfgs = api.metts(ctx, H, cfg0, beta, 1e-2, 4, 16, 1e-12, us,
                              alt_basis=ometts.X_BASIS, obs=sz, obs_site=3, shift0=e0)
    e_o, vals_o, cfgs_o = ometts.metts_chain(Ws, cfg0, 2, beta, 5, us, 1e-2, 4, 16, 1e-12,
                                             obs=sz, obs_site=3, alt_basis=ometts.X_BASIS,
                                             shift_mode="fixed", shift=e0)
    assert np.allclose(e, e_o, rtol=1e-10, atol=0)
    assert np.allclose(vals, vals_o, rtol=0, atol=1e-10)
    assert cfgs.tolist() == cfgs_o


def test_anderson_chain_double_occupancy_matches_oracle(api, ctx):
    n_bath, beta = 3, 4.0
    eps, V = inputs.flat_band_bath(n_bath)
    Ws = ompo.anderson_mpo(-0.15, 0.3, eps, V)
    H = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15)
    us = np.random.default_rng(13).random((4, n_bath + 1))
    cfg0 = [1, 2, 1, 2]          # up, down on alternating sites
    docc = np.diag([0.0, 0.0, 0.0, 1.0]).astype(complex)
    e0 = np.linalg.eigvalsh(ed.anderson_hamiltonian(-0.15, 0.3, eps, V))[0]
    e, vals, cfgs = api.metts(ctx, H, cfg0, beta, 1e-2, 4, 16, 1e-14, us, obs=docc, obs_site=0,
                              shift0=e0)
    e_o, vals_o, cfgs_o = ometts.metts_chain(Ws, cfg0, 4, beta, 4, us, 1e-2, 4, 16, 1e-14,
                                             obs=docc, obs_site=0, shift_mode="fixed", shift=e0)
    assert np.allclose(e, e_o, rtol=1e-10, atol=0)
    assert np.allclose(vals, vals_o, rtol=0, atol=1e-10)
    assert cfgs.tolist() == cfgs_o
