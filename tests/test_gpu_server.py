"""Served execution on the GPU (include/ite_server.h): jobs of different
models, sizes, schemes and precisions run side by side on several streams, and
each job's energies and final state equal those of the same evolution run
alone through ite_evolve_loggrid.  The kernels are deterministic and the jobs
share no data, so the comparison is at 1e-12."""
import numpy as np
import pytest

from oracle import mps as omps
from paper_2606_02930_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02930_gb300 import api as a
    return a


def _jobs(api):
    specs = []
    for k, (N, chi, scheme, prec) in enumerate([(8, 16, "be", "fp64"), (10, 32, "tr", "fp64"),
                                                (12, 32, "be", "fp64"), (16, 64, "be", "fp64_tc"),
                                                (12, 24, "tr", "fp64_tc")]):
        specs.append(dict(model="heisenberg", n=N, site_vecs=inputs.random_product_state(N, 2, 40 + k),
                          chi_max=chi, cutoff=1e-10, tau0=1e-2, tau_max=1e1, n_steps=5,
                          scheme=scheme, opts=api.solver_opts(precision=prec)))
    eps, V = inputs.flat_band_bath(4)
    specs.append(dict(model="anderson", n=4, site_vecs=inputs.random_product_state(5, 4, 50),
                      chi_max=24, cutoff=1e-14, tau0=1e-2, tau_max=1e2, n_steps=4, scheme="be",
                      U=0.3, eps_d=-0.15, eps=eps, V=V, opts=api.solver_opts()))
    return specs


def _alone(api, spec):
    ctx = api.ctx_create(0)
    if spec["model"] == "heisenberg":
        H = api.mpo_create_heisenberg(ctx, spec["n"])
    else:
        H = api.mpo_create_anderson(ctx, spec["eps"], spec["V"], spec["U"], spec["eps_d"])
    psi = api.mps_create_product(ctx, spec["site_vecs"], spec["chi_max"])
    _, infos = api.evolve_loggrid(ctx, H, psi, spec["tau0"], spec["tau_max"], spec["n_steps"],
                                  spec["scheme"], spec["chi_max"], spec["cutoff"],
                                  shift_mode=api.SHIFT_CURRENT_ENERGY, opts=spec["opts"])
    return np.array([i["energy"] for i in infos]), psi.tensors()


def _check_against_alone(api, jobs, results, specs):
    for job, res, spec in zip(jobs, results, specs):
        assert res["status"] == 0
        assert res["steps_done"] == spec["n_steps"]
        e_alone, t_alone = _alone(api, spec)
        assert np.max(np.abs(job.energies - e_alone)) <= 1e-12 * np.max(np.abs(e_alone))
        t_mix = job.tensors()
        ov = omps.overlap(t_alone, t_mix)
        assert 1.0 - abs(ov) / (omps.norm(t_alone) * omps.norm(t_mix)) <= 1e-12
        assert res["latency_ms"] >= res["run_ms"] >= 0.0


def test_jobs_in_the_mix_equal_jobs_alone(api):
    specs = _jobs(api)
    jobs = [api.Job(want_state=True, **s) for s in specs]
    server = api.Server(0, n_slots=3)
    tickets = [server.submit(j) for j in jobs]
    results = [server.wait(t) for t in tickets]
    st = server.stats()
    server.close()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["peak_running"] >= 2          # the jobs did overlap
    assert 0.0 < st["p50_latency_ms"] <= st["p99_latency_ms"]
    assert st["tau_steps"] == sum(s["n_steps"] for s in specs)
    _check_against_alone(api, jobs, results, specs)


def test_admission_by_device_bytes(api):
    # a budget that holds the two largest estimates but not three: at most two
    # run at once, all finish, results unchanged
    specs = _jobs(api)
    jobs = [api.Job(want_state=True, **s) for s in specs]
    sizes = sorted(j.device_bytes() for j in jobs)
    budget = sizes[-1] + sizes[-2] + 1
    results, st = api.evolve_batch(jobs, n_slots=4, mem_budget=budget)
    assert st["completed"] == len(jobs)
    assert st["peak_running"] <= 2 or sum(sizes[:3]) <= budget
    _check_against_alone(api, jobs, results, specs)
    # a job larger than the whole budget is refused at submission
    server = api.Server(0, n_slots=1, mem_budget=sizes[0] - 1)
    with pytest.raises(Exception):
        server.submit(jobs[-1])
    server.close()
