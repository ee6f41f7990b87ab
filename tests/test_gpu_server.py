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


def _metts_specs(api):
    X = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)
    sz = np.diag([0.5, -0.5]).astype(complex)
    docc = np.diag([0.0, 0.0, 0.0, 1.0]).astype(complex)
    specs = []
    for k, N in enumerate((6, 8, 8)):
        specs.append(dict(model="heisenberg", n=N, config0=[0, 1] * (N // 2), chi_max=16,
                          cutoff=1e-12, tau_max=1.0, panels=8, steps_per_panel=4,
                          uniforms=np.random.default_rng(60 + k).random((4, N)), alt_basis=X,
                          obs=sz, obs_site=2))
    eps, V = inputs.flat_band_bath(2)
    specs.append(dict(model="anderson", n=2, config0=[3, 0, 1], chi_max=16, cutoff=0.0,
                      tau_max=2.0, panels=9, steps_per_panel=4,
                      uniforms=np.random.default_rng(13).random((4, 3)), obs=docc, obs_site=0,
                      U=0.3, eps_d=-0.15, eps=eps, V=V))
    return specs


def _metts_alone(api, spec):
    ctx = api.ctx_create(0)
    if spec["model"] == "heisenberg":
        H = api.mpo_create_heisenberg(ctx, spec["n"])
    else:
        H = api.mpo_create_anderson(ctx, spec["eps"], spec["V"], spec["U"], spec["eps_d"])
    nodes = api.grid_panels(spec["tau_max"], spec["panels"], spec["steps_per_panel"])
    return api.metts(ctx, H, spec["config0"], nodes, spec["chi_max"], spec["cutoff"],
                     spec["uniforms"], alt_basis=spec.get("alt_basis"), obs=spec["obs"],
                     obs_site=spec["obs_site"])


def test_metts_and_panel_jobs_in_the_mix_equal_calls_alone(api):
    # METTS chains (ite_metts) and a panel-grid evolution (ite_evolve_panels)
    # served side by side give what the same calls give alone
    specs = _metts_specs(api)
    jobs = [api.MettsJob(**s) for s in specs]
    sv = inputs.random_product_state(10, 2, 77)
    evo = api.Job("heisenberg", 10, sv, 24, 1e-10, 0.0, 4.0, 3, scheme="tr", panels=6,
                  want_state=True)
    results, st = api.evolve_batch(jobs + [evo], n_slots=3)
    assert st["completed"] == len(jobs) + 1 and st["failed"] == 0
    for job, res, spec in zip(jobs, results, specs):
        assert res["status"] == 0
        assert res["steps_done"] == len(spec["uniforms"]) * spec["panels"] * spec["steps_per_panel"]
        e, vals, cfgs = _metts_alone(api, spec)
        assert np.array_equal(job.configs, cfgs)
        assert np.max(np.abs(job.energies - e)) <= 1e-12 * np.max(np.abs(e))
        assert np.max(np.abs(job.obs_values - vals)) <= 1e-12
    ctx = api.ctx_create(0)
    H = api.mpo_create_heisenberg(ctx, 10)
    psi = api.mps_create_product(ctx, sv, 24)
    _, infos = api.evolve_panels(ctx, H, psi, 4.0, 6, 3, "tr", 24, 1e-10,
                                 shift_mode=api.SHIFT_CURRENT_ENERGY)
    e_alone = np.array([i["energy"] for i in infos])
    assert results[-1]["steps_done"] == 18
    assert np.max(np.abs(evo.energies - e_alone)) <= 1e-12 * np.max(np.abs(e_alone))
    t_mix, t_alone = evo.tensors(), psi.tensors()
    ov = omps.overlap(t_alone, t_mix)
    assert 1.0 - abs(ov) / (omps.norm(t_alone) * omps.norm(t_mix)) <= 1e-12


def _energies_and_states(api, specs, n_slots, grouping, window_ms):
    jobs = [api.Job(want_state=True, **s) for s in specs]
    results, st = api.evolve_batch(jobs, n_slots=n_slots, grouping=grouping, window_ms=window_ms)
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert all(r["status"] == 0 for r in results)
    return jobs, results, st


@pytest.mark.parametrize("which", ["same_shapes", "mixed_shapes"])
def test_grouped_jacobi_launches_change_no_result(api, which):
    # the splits of the running jobs go to the device as grouped launches
    # (k_jacobi_grouped); every job ends bit for bit as with grouping off, and
    # as the same evolution alone
    if which == "same_shapes":
        specs = [dict(model="heisenberg", n=12, site_vecs=inputs.random_product_state(12, 2, 90 + k),
                      chi_max=32, cutoff=1e-10, tau0=1e-2, tau_max=1e1, n_steps=3, scheme="be",
                      opts=api.solver_opts(precision="fp64"))
                 for k in range(4)]
    else:
        specs = _jobs(api)
    # mode 2 (gather) makes the grouping certain: every running job's post
    g_jobs, g_res, g_st = _energies_and_states(api, specs, len(specs), 2, 200.0)
    u_jobs, _, u_st = _energies_and_states(api, specs, len(specs), 0, 20.0)
    assert u_st["group_launches"] == 0
    assert g_st["group_items"] > g_st["group_launches"] > 0     # launches carried several splits
    for gj, uj in zip(g_jobs, u_jobs):
        assert np.array_equal(gj.energies, uj.energies)
        assert all(np.array_equal(a, b) for a, b in zip(gj.tensors(), uj.tensors()))
    _check_against_alone(api, g_jobs, g_res, specs)
