"""MPS checkpoints and dense read-out on the GPU: a checkpoint taken in the
middle of an evolution, loaded into a new context, continues exactly as the
original does; malformed images are refused; the dense vector equals the
oracle's contraction of the same tensors."""
import numpy as np
import pytest

from oracle import mps as omps
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


def test_checkpoint_resumes_an_evolution_exactly(api, ctx):
    N, chi = 10, 16
    H = api.mpo_create_heisenberg(ctx, N)
    psi = api.mps_create_product(ctx, inputs.random_product_state(N, 2, 31), chi)
    s = -4.0
    for dt in (0.05, 0.1, 0.2):
        s = api.implicit_step(ctx, H, psi, dt, "tr", s, chi, 1e-12)["energy"]
    data = psi.save()
    assert data[:8] == b"ITEMPS01"
    same = api.mps_load(ctx, data)
    for a, b in zip(psi.tensors(), same.tensors()):
        assert np.array_equal(a, b)
    ctx2 = api.ctx_create(0)
    H2 = api.mpo_create_heisenberg(ctx2, N)
    other = api.mps_load(ctx2, data)
    s1 = s2 = s
    for dt in (0.4, 0.8):
        s1 = api.implicit_step(ctx, H, psi, dt, "tr", s1, chi, 1e-12)["energy"]
        s2 = api.implicit_step(ctx2, H2, other, dt, "tr", s2, chi, 1e-12)["energy"]
        assert s1 == s2
    for a, b in zip(psi.tensors(), other.tensors()):
        assert np.array_equal(a, b)
    # malformed images: wrong magic, truncated header, truncated tensors
    for bad in (b"XXXXXXXX" + data[8:], data[:20], data[:-8]):
        with pytest.raises(IteError):
            api.mps_load(ctx, bad)


@pytest.mark.parametrize("N,d,chi", [(8, 2, 8), (5, 4, 12)])
def test_to_dense_equals_oracle(api, ctx, N, d, chi):
    A = inputs.random_mps(N, d, chi, 50 + N)
    psi = api.mps_create(ctx, A, chi)
    v = psi.to_dense()
    want = omps.to_dense(A)
    assert np.abs(v - want).max() <= 1e-13 * np.abs(want).max()
