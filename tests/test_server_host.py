"""CPU checks of the served-execution runtime's host logic (include/ite_server.h):
the admission estimate and argument validation, with no GPU call."""
import numpy as np

from paper_2606_02930_gb300 import _lib as L, inputs
from paper_2606_02930_gb300.api import Job, lib


def _heis(N, chi, precision="fp64"):
    from paper_2606_02930_gb300.api import solver_opts
    return Job("heisenberg", N, inputs.random_product_state(N, 2, 1), chi, 1e-10, 1e-2, 1e1, 5,
               opts=solver_opts(precision=precision))


def test_device_bytes_grow_with_chi_and_n():
    b = [_heis(32, chi).device_bytes() for chi in (8, 16, 32, 64, 128)]
    assert all(x < y for x, y in zip(b, b[1:]))
    assert _heis(16, 64).device_bytes() < _heis(64, 64).device_bytes()
    # saturated chi: the bulk two-site block dominates; chi^2 scaling
    r = _heis(64, 256).device_bytes() / _heis(64, 128).device_bytes()
    assert 3.0 < r < 4.5
    assert _heis(64, 256, "fp64_tc").device_bytes() > _heis(64, 256).device_bytes()


def test_anderson_estimate_and_invalid_jobs():
    eps, V = inputs.flat_band_bath(9)
    ja = Job("anderson", 9, inputs.random_product_state(10, 4, 2), 64, 1e-14, 1e-2, 1e2, 4,
             U=0.3, eps_d=-0.15, eps=eps, V=V)
    assert ja.device_bytes() > 0
    bad = _heis(8, 16)
    bad.c.n_steps = 0
    assert bad.device_bytes() == 0
    bad = _heis(8, 16)
    bad.c.tau_max = bad.c.tau0
    assert bad.device_bytes() == 0
    bad = _heis(8, 16)
    bad.c.model = 7
    assert bad.device_bytes() == 0


def test_server_calls_reject_invalid_arguments():
    import ctypes as C
    t = C.c_longlong()
    assert lib.ite_server_submit(None, C.byref(_heis(8, 16).c), C.byref(t)) == L.ITE_EINVAL
    assert lib.ite_server_create(0, 0, 0, C.byref(C.c_void_p())) == L.ITE_EINVAL
    assert lib.ite_server_create(0, 65, 0, C.byref(C.c_void_p())) == L.ITE_EINVAL
    # an invalid job is refused before any device work
    bad = _heis(8, 16)
    bad.c.chi_max = 0
    arr = (L.ite_job * 1)(bad.c)
    res = (L.ite_job_result * 1)()
    assert lib.ite_evolve_batch(0, 2, 0, 1, arr, res, None) == L.ITE_EINVAL
    assert lib.ite_server_drain(None) == L.ITE_EINVAL
    assert np.isfinite(_heis(8, 16).device_bytes())


def test_metts_and_panel_job_validation():
    from paper_2606_02930_gb300.api import MettsJob
    us = np.full((3, 6), 0.5)
    ok = MettsJob("heisenberg", 6, [0, 1] * 3, 16, 1e-12, 1.0, 8, 4, us)
    assert ok.device_bytes() > 0
    bad = MettsJob("heisenberg", 6, [0, 1, 0, 1, 0, 2], 16, 1e-12, 1.0, 8, 4, us)
    assert bad.device_bytes() == 0                     # state 2 of a spin
    bad = MettsJob("heisenberg", 6, [0, 1] * 3, 16, 1e-12, 1.0, 0, 4, us)
    assert bad.device_bytes() == 0                     # no panels
    bad = MettsJob("heisenberg", 6, [0, 1] * 3, 16, 1e-12, 1.0, 8, 4, us,
                   obs=np.eye(2), obs_site=6)
    assert bad.device_bytes() == 0                     # observable site out of range
    pj = Job("heisenberg", 8, inputs.random_product_state(8, 2, 1), 16, 1e-10, 0.0, 4.0, 3,
             panels=5)
    assert pj.device_bytes() > 0 and len(pj.energies) == 15
    pj.c.grid = 5
    assert pj.device_bytes() == 0


def test_mixed_modes_estimate_their_refinement_buffers():
    # the mixed modes hold the FP64-class slice scratch, the refinement's four
    # vectors and the low-precision operands on top of the FP64 state
    for prec in ("mixed_bf16", "mixed_tf32"):
        assert _heis(64, 256, prec).device_bytes() > _heis(64, 256, "fp64_tc").device_bytes()


def test_serve_stream_draws():
    # the served stream's requests: fixed by the seed, parameters in their
    # ranges, steps from the grid length rule, bath arrays of the drawn size
    a = inputs.serve_stream(12, baths=(9, 19), chis=(16, 32))
    b = inputs.serve_stream(12, baths=(9, 19), chis=(16, 32))
    assert all(np.array_equal(x["site_vecs"], y["site_vecs"]) and x["U"] == y["U"] for x, y in zip(a, b))
    for r in a:
        assert 0.05 <= r["U"] <= 0.6 and 0.02 <= r["Gamma"] <= 0.1 and r["eps_d"] == -0.5 * r["U"]
        assert r["n_bath"] in (9, 19) and r["chi_max"] in (16, 32) and r["gap_s"] >= 0.0
        assert r["tau_max"] in (1e2, 1e3, 1e4)
        assert r["n_steps"] == int(np.ceil(10 * np.log10(r["tau_max"] / 1e-2)))
        assert r["eps"].shape == (r["n_bath"],) and r["V"].shape == (r["n_bath"],)
        assert r["site_vecs"].shape == (r["n_bath"] + 1, 4)
