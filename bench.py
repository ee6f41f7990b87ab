"""Benchmark: tau-steps/s of the implicit MPS imaginary-time step on GB300.

Workload (the configuration the headline metric is quoted on): Heisenberg XXX
chain, N = 64, J = 1, open boundaries, MPO bond dimension 5, chi_max = 256,
SVD cutoff 1e-10, backward Euler (implicit Euler) on the geometric tau grid
1e-3 -> 1e3 with 40 steps, shift = energy of the current state.  The start
state is a seeded synthetic MPS at the saturated bond dimension (chi = 256 in
the bulk: random isometries with bond weights exp(-b/64), so the cap of 256
binds rather than the cutoff), standing in for the evolved random product
state once chi has saturated, where the evolution spends its time.  One benchmark step = one
implicit tau-step (gauge move, environments, a full L->R->R->L sweep of
GMRES(10) local solves with truncated SVD splits, normalisation, energy) on
the next node of the grid.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs independent replicas (one chain per rank, no data-path
collective), launched with torch.distributed.run.  --impl reference times the
CPU oracle on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SITES, CHI, CUTOFF, D_MPO, D_SITE = 64, 256, 1e-10, 5, 2
TAU0, TAU_MAX, K_GRID = 1e-3, 1e3, 40
SEED = 2000
METRIC = "H_eff matvec TFLOP/s; τ-steps/s vs plain FP64 at equal ΔE; p50/p99 latency"
UNIT = "tau-steps/s"
# FP64 pipe of GB300 (no measured FP64 peak exists for this machine): 152 SMs x
# 2 DFMA/clk x 2 FLOP x 2.07 GHz = 1.26 TFLOP/s, in line with the nominal
# 1.25 TFLOP/s (a DFMA probe measured 1.19 at 1995 MHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) of one k_jacobi_persistent launch on the bulk
# 512 x 512 split from the ncu capture of this kernel source summarised in
# profiles/k_jacobi_persistent_split512.md (None once the kernel changes).
JACOBI_TRAFFIC_BYTES = 4.268544e6 + 1.094656e6
JACOBI_TRAFFIC_NOTE = ("dram bytes per launch on the 512 x 512 bulk split (ncu, "
                       "profiles/k_jacobi_persistent_split512.md); the matrix is L2-resident, "
                       "the kernel is FP64-bound")
WORKLOAD = ("heisenberg_bulk: XXX chain N=64 J=1 OBC, D=5, chi_max=256, cutoff 1e-10, "
            "backward Euler on geometric grid 1e-3->1e3 (40 steps), shift=current energy, "
            "saturated synthetic start (chi=256 bulk)")


SCHEME_NAMES = {"be": "backward_euler", "tr": "trapezoid", "gl2": "gauss_legendre_2",
                "gl3": "gauss_legendre_3"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--bonds", type=int, default=6, help="bulk bonds in the CPU sample")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="steps of the timed sequence replayed in plain FP64 for comparison")
    ap.add_argument("--mixed-steps", type=int, default=3,
                    help="steps of the sequence replayed with converged local solves, mixed bf16 "
                         "against plain FP64 (equal accuracy)")
    ap.add_argument("--precision", choices=["fp64", "fp64_tc", "mixed_bf16", "mixed_tf32"],
                    default="fp64_tc",
                    help="fp64: FP64 pipes; fp64_tc: FP64-class contractions on the tensor cores; "
                         "mixed_*: local solves converged by refinement with bf16/tf32 inner "
                         "matvecs")
    ap.add_argument("--only", choices=["heff", "split", "heff_lp"], default=None,
                    help="time one kernel-level call at the bulk shape (for profiler captures)")
    ap.add_argument("--scheme", choices=["be", "tr", "gl2", "gl3"], default="be",
                    help="time stepper of the chain workload (the headline runs backward Euler)")
    ap.add_argument("--workload", choices=["chain", "batch", "chi_study", "metts", "anderson",
                                           "serve"],
                    default="chain",
                    help="batch: a bounded sample of the batched workload served side by side; "
                         "chi_study: bond-dimension growth and step cost of an evolution; "
                         "metts: independent METTS chains served side by side; "
                         "anderson: the first steps of the impurity-model evolution; "
                         "serve: a Poisson stream of impurity evolutions through the server")
    ap.add_argument("--lp-shape", default="all",
                    help="--only heff_lp: all, heisenberg512, heisenberg1024 or anderson512")
    ap.add_argument("--jobs", type=int, default=16, help="jobs in the batch sample")
    ap.add_argument("--no-single", action="store_true", help="batch: skip the one-at-a-time arm")
    ap.add_argument("--no-grouped", action="store_true", help="batch: skip the grouped arm")
    ap.add_argument("--batch-ns", default="16,24,32,48,64", help="batch: chain lengths drawn from")
    ap.add_argument("--grouping-mode", type=int, default=1, choices=[1, 2],
                    help="batch: grouping mode of the grouped arm (1 continuous, 2 gather)")
    ap.add_argument("--batch-chis", default="32,64,128,256", help="batch: bond caps drawn from")
    ap.add_argument("--anderson-start", choices=["product", "saturated"], default="product",
                    help="anderson: start from a product state or at the saturated chi")
    ap.add_argument("--anderson-bath", type=int, default=99, help="anderson: bath sites")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: mean arrivals per second")
    ap.add_argument("--serve-baths", default="9,19,29", help="serve: bath sizes drawn from")
    ap.add_argument("--serve-chis", default="16,32,64", help="serve: bond caps drawn from")
    ap.add_argument("--slots", type=int, default=4, help="concurrent jobs in the batch sample")
    ap.add_argument("--study-n", type=int, default=100, help="chain length of the chi study")
    ap.add_argument("--study-m", type=int, default=8, help="chi study runs to tau_max = 2^m")
    ap.add_argument("--study-chi", type=int, default=128, help="bond-dimension cap of the chi study")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def bond_weights():
    """Cost of each of the 2(N-1) two-site updates of a sweep relative to a
    bulk update, by the algorithmic H_eff FLOP count (chi profile of the
    saturated state)."""
    from paper_2606_02930_gb300 import inputs
    cap = [1] + inputs.bond_profile(N_SITES, D_SITE, CHI) + [1]
    d, D = D_SITE, D_MPO

    def fl(chl, chr_):
        return D * d * d * chl * chr_ * (chl + chr_) + 2 * D * D * d ** 3 * chl * chr_

    bulk = fl(CHI, CHI)
    w = [fl(cap[i], cap[i + 2]) / bulk for i in range(N_SITES - 1)]
    return 2.0 * sum(w)


def oracle_bond_sample(n_bonds):
    """Time the oracle on the start of one tau-step of the real workload: the
    gauge move and right environments of the start state, then the first
    two-site updates of the left-to-right pass up to and including n_bonds
    bulk (chi = 256) bonds (projection of the right-hand side, GMRES(10) on
    (1 - c s) X + c H_eff X, truncated SVD split, environment updates), with
    the first step's dtau and shift = the state's energy.  Returns (seconds
    of the setup, seconds per bulk update, updates timed)."""
    from oracle import linsolve as ls, mpo as ompo, mps as omps
    from paper_2606_02930_gb300 import inputs
    Ws = ompo.heisenberg_mpo(N_SITES)
    A = inputs.random_isometric_mps(N_SITES, D_SITE, CHI, SEED)
    s = omps.expect_mpo(A, Ws)
    c = TAU0                               # backward Euler, first grid step
    t0 = time.perf_counter()
    x = ls.right_canonicalize_svd(A)
    b = A
    Rop, Rov = ls._build_right_envs(Ws, x, [("op", x), ("ov", b)])
    Lop = np.ones((1, 1, 1), complex)
    Lov = np.ones((1, 1), complex)
    t_setup = time.perf_counter() - t0
    alpha = 1.0 - c * s
    first_bulk = int(np.ceil(np.log2(CHI))) if D_SITE == 2 else 0
    t_bulk, n_done, i = 0.0, 0, 0
    while n_done < n_bonds:
        t1 = time.perf_counter()
        B = ls.project_two_site(Lov, b[i], b[i + 1], Rov[i + 1])
        X0 = np.tensordot(x[i], x[i + 1], axes=([2], [0]))
        mv = lambda V: alpha * V + c * ls.heff_apply(Lop, Ws[i], Ws[i + 1], Rop[i + 1], V)
        X, _ = ls.gmres(mv, B, X0, 10)
        x[i], x[i + 1], _, _ = ls.split_two_site(X, CHI, CUTOFF, True)
        Lop = ls.left_env_update(Lop, x[i], Ws[i], x[i])
        Lov = ls.left_overlap_update(Lov, x[i], b[i])
        if i >= first_bulk:
            t_bulk += time.perf_counter() - t1
            n_done += 1
        i += 1
    return t_setup, t_bulk / n_bonds, i


def cpu_baseline_line(n_bonds):
    t_setup, t_bond, done = oracle_bond_sample(n_bonds)
    per_step = t_setup + t_bond * bond_weights()
    return {"value": 1.0 / per_step, "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle, extrapolated",
            "sample": (f"the oracle's gauge move and environments of the start state "
                       f"({t_setup:.1f} s) and the first {done} two-site updates of its sweep "
                       f"({n_bonds} bulk chi=256 updates timed: {t_bond:.2f} s each), the step "
                       f"extrapolated as setup + {bond_weights():.1f} bulk-equivalent updates")}


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            work = os.path.join(ROOT, "_build", "clocks")           # git-ignored scratch
            os.makedirs(work, exist_ok=True)
            fd, self.path = tempfile.mkstemp(prefix=f"rank{self.index}_", suffix=".csv", dir=work)
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ replicas
def replica_seed(rank):
    """Seed of rank's chain: replicas evolve different synthetic states."""
    return SEED + rank


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest x over all ranks of the process group (x without one)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, t_max_s):
    """tau-steps/s of the whole job: every rank's steps over the slowest rank's time."""
    return world * steps / t_max_s


# ------------------------------------------------------------------ arms
def run_reference(args, rank, world):
    if rank != 0:
        return
    W, K = args.warmup, args.steps
    for _ in range(W):
        oracle_bond_sample(1)
    vals = []
    t0 = time.perf_counter()
    for _ in range(K):
        t_setup, t_bond, _ = oracle_bond_sample(args.bonds)
        vals.append(t_setup + t_bond * bond_weights())
    tot = time.perf_counter() - t0
    value = 1.0 / statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * statistics.mean(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{args.bonds} bulk bonds per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle, extrapolated",
                             "sample": (f"each step: the oracle's gauge move and environments "
                                        f"of the start state and its sweep up to {args.bonds} "
                                        f"bulk chi=256 two-site updates, extrapolated to "
                                        f"{bond_weights():.1f} bulk-equivalent updates per "
                                        f"tau-step; wall {tot:.1f} s")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def heff_kernel_rates(api, ctx, H, precision, reps=5):
    """Kernel-level H_eff TFLOP/s (algorithmic FLOP count) at the bulk shapes
    chi = 256 and chi = 512 (d = 2, D = 5), CUDA events on the context stream."""
    import torch
    from paper_2606_02930_gb300 import inputs  # noqa: F401  (same module set as the step)
    rng = np.random.default_rng(SEED)
    out = {}
    api.set_kernel_precision(ctx, precision)
    stream = torch.cuda.current_stream()
    try:
        for chi in (256, 512):
            def dev(*shape):
                a = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(shape[-1])
                return torch.from_numpy(a).to("cuda")
            L, R, X = dev(D_MPO, chi, chi), dev(D_MPO, chi, chi), dev(chi, D_SITE, D_SITE, chi)
            Y = torch.empty_like(X)
            flops = 8.0 * (2 * D_MPO * D_SITE ** 2 * chi ** 3 + 2 * D_MPO ** 2 * D_SITE ** 3 * chi ** 2)
            for _ in range(2):
                api.k_heff(ctx, H, 20, L, R, X, Y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                api.k_heff(ctx, H, 20, L, R, X, Y)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out[f"chi{chi}"] = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12}
    finally:
        api.set_kernel_precision(ctx, "fp64")
    return out


def measured_peaks():
    """(bf16 burst TFLOP/s, sustained, source) from MEASURED_PEAKS.json, else
    the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, 1700.0, "fallback"


LP_SHAPES = (("heisenberg", 2, 5, 512), ("heisenberg", 2, 5, 1024), ("anderson", 4, 6, 512))


def heff_lp_rates(api, ctx, precisions=("mixed_bf16",), reps=10, shapes=LP_SHAPES):
    """Kernel-level TFLOP/s of the low-precision H_eff matvec (operands
    prepared once, as in a local solve) at bulk shapes with chi >= 512, by the
    algorithmic FLOP count, CUDA events on the context stream; fraction of the
    measured bf16 burst peak (tf32: half of it, the nominal tf32/bf16 ratio)."""
    import torch
    from paper_2606_02930_gb300 import inputs
    peak_bf16, _, src = measured_peaks()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(SEED)
    out = {}
    for model, d, D, chi in shapes:
        if model == "heisenberg":
            H = api.mpo_create_heisenberg(ctx, 40)
            i = 20
        else:
            eps, V = inputs.flat_band_bath(39)
            H = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15)
            i = 20

        def dev(*shape):
            a = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(shape[-1])
            return torch.from_numpy(a).to("cuda")
        L, R, X = dev(D, chi, chi), dev(D, chi, chi), dev(chi, d, d, chi)
        Y = torch.empty_like(X)
        flops = 8.0 * (2 * D * d ** 2 * chi ** 3 + 2 * D ** 2 * d ** 3 * chi ** 2)
        for prec in precisions:
            api.k_heff_lp_prepare(ctx, H, i, L, R, prec)
            for _ in range(3):
                api.k_heff_lp_apply(ctx, H, i, X, Y, 1.0, X, 0.5)
            # back-to-back matvecs (one host synchronisation), as in a Krylov cycle
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            api.k_heff_lp_apply_n(ctx, H, i, X, Y, 1.0, X, 0.5, reps=reps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            tf = flops / (ms * 1e-3) / 1e12
            peak = peak_bf16 if prec == "mixed_bf16" else 0.5 * peak_bf16
            out[f"{model}_d{d}_D{D}_chi{chi}_{prec}"] = {
                "ms": ms, "tflops": tf, "peak": peak, "frac": tf / peak,
                "peak_note": (f"{src} bf16 burst" if prec == "mixed_bf16"
                              else f"{src} bf16 burst x 1/2 (nominal tf32 ratio)")}
        del L, R, X, Y
    return out


def reference_energies(converged=False):
    """Oracle energies of the first steps of the timed sequence (backward
    Euler from the start state; fixed effort or converged local solves),
    written by tests/golden/make_bench_reference.py; None when absent."""
    name = "bench_reference_energies" + ("_converged" if converged else "") + ".json"
    path = os.path.join(ROOT, "tests", "golden", name)
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2606_02930_gb300 import api, inputs
    from paper_2606_02930_gb300 import _lib as L
    import ctypes as C
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    ctx = api.ctx_create(local_rank)
    stream = torch.cuda.current_stream()
    H = api.mpo_create_heisenberg(ctx, N_SITES)
    A0 = inputs.random_isometric_mps(N_SITES, D_SITE, CHI, replica_seed(rank))
    psi = api.mps_create(ctx, A0, CHI)
    start = api.mps_create(ctx, A0, CHI)       # the start state, kept on the device
    nodes = api.grid_geometric(TAU0, TAU_MAX, K_GRID)
    s0 = api.energy(ctx, H, start)
    opts = api.solver_opts(precision=args.precision)

    # Every measured sequence is the same: K steps k = 0..K-1 of the grid from
    # the start state, shift = the energy of the current state.
    def run(n, o, events=None, host_io=None):
        api.mps_copy(ctx, start, psi)
        s, infos = s0, []
        for k in range(n):
            if host_io is not None:
                host_io.before()
            kk = k % K_GRID
            info = api.implicit_step(ctx, H, psi, nodes[kk + 1] - nodes[kk], args.scheme, s, CHI,
                                     CUTOFF, o)
            if host_io is not None:
                host_io.after()
            if events is not None:
                events[k].record(stream)
            s = info["energy"]
            infos.append(info)
        return infos

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    run(args.warmup, opts)

    # ---- device-timed region: state resident in HBM
    clocks = ClockSampler(local_rank)
    api.mps_copy(ctx, start, psi)
    barrier()
    clocks.start()
    launches0 = api.kernel_launches()
    api.svd_stats(ctx)
    api.profile_start(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e0.record(stream)
    # run() copies the start state in first; that device copy (134 MB) is
    # timed with the steps
    infos = run(args.steps, opts, events=ev)
    barrier()
    prof = api.profile_stop(ctx)
    svd = api.svd_stats(ctx)
    launches = api.kernel_launches() - launches0
    clk = clocks.stop()
    ms = e0.elapsed_time(ev[-1])
    step_ms = [e0.elapsed_time(ev[0])] + [ev[k - 1].elapsed_time(ev[k]) for k in range(1, args.steps)]
    t_max = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(world, args.steps, t_max * 1e-3)

    # ---- end to end through the C ABI with host buffers (pinned): the same
    # K steps from the same start state; every step uploads the state from
    # host memory and reads the new state back
    cap = [1] + inputs.bond_profile(N_SITES, D_SITE, CHI) + [1]
    cap_doubles = sum(2 * cap[i] * D_SITE * cap[i + 1] for i in range(N_SITES))
    host = torch.empty(cap_doubles, dtype=torch.float64, pin_memory=True)
    lib = L.lib
    hptr = C.cast(C.c_void_p(host.data_ptr()), C.POINTER(C.c_double))

    class HostIO:
        def __init__(self):
            self.chi = np.zeros(N_SITES + 1, np.int32)
            self.n = C.c_size_t()
            self.h2d = self.d2h = 0
            L.check(lib.ite_mps_bond_dims(start.h, self.chi.ctypes.data_as(C.POINTER(C.c_int)),
                                          C.byref(self.n)))
            L.check(lib.ite_mps_get(ctx.h, start.h, hptr, cap_doubles), ctx.h)

        def before(self):
            L.check(lib.ite_mps_set(ctx.h, psi.h, self.chi.ctypes.data_as(C.POINTER(C.c_int)),
                                    hptr), ctx.h)
            self.h2d += 8 * self.n.value

        def after(self):
            L.check(lib.ite_mps_bond_dims(psi.h, self.chi.ctypes.data_as(C.POINTER(C.c_int)),
                                          C.byref(self.n)))
            L.check(lib.ite_mps_get(ctx.h, psi.h, hptr, cap_doubles), ctx.h)
            self.d2h += 8 * self.n.value

    hio = HostIO()
    barrier()
    t0 = time.perf_counter()
    e2e_infos = run(args.steps, opts, host_io=hio)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_same = all(a["energy"] == b["energy"] for a, b in zip(infos, e2e_infos))

    # ---- plain FP64 arm on the first steps of the same sequence
    n64 = min(args.steps, args.fp64_steps)
    fp64 = None
    if n64 > 0 and args.precision != "fp64":
        ev64 = [torch.cuda.Event(enable_timing=True) for _ in range(n64)]
        f0 = torch.cuda.Event(enable_timing=True)
        barrier()
        f0.record(stream)
        infos64 = run(n64, api.solver_opts(precision="fp64"), events=ev64)
        barrier()
        ms64 = f0.elapsed_time(ev64[-1])
        ms_same = sum(step_ms[:n64])
        fp64 = {"steps": n64, "ms_per_step": ms64 / n64,
                "tau_steps_per_s": n64 / (ms64 * 1e-3),
                "this_precision_ms_per_step_same_steps": ms_same / n64,
                "speedup_over_fp64": ms64 / ms_same,
                "max_rel_energy_diff_vs_this_precision": max(
                    abs(a["energy"] - b["energy"]) / abs(b["energy"]) for a, b in zip(infos64, infos))}

    # ---- equal accuracy: local solves converged, mixed bf16 refinement
    # against plain FP64 GMRES restarted to the same relative residual
    mixed = None
    nmx = min(args.steps, args.mixed_steps)
    if nmx > 0 and rank == 0:
        arms = {}
        for name, o in (("mixed_bf16", api.solver_opts(precision="mixed_bf16", refine_tol=1e-10,
                                                        refine_max=20)),
                        ("fp64_converged", api.solver_opts(precision="fp64", local_tol=1e-10,
                                                           max_cycles=200))):
            evx = [torch.cuda.Event(enable_timing=True) for _ in range(nmx)]
            x0 = torch.cuda.Event(enable_timing=True)
            barrier()
            x0.record(stream)
            inf_x = run(nmx, o, events=evx)
            barrier()
            msx = x0.elapsed_time(evx[-1])
            arms[name] = {"steps": nmx, "ms_per_step": msx / nmx, "tau_steps_per_s": nmx / (msx * 1e-3),
                          "energies": [i["energy"] for i in inf_x],
                          "max_local_residual": max(i["max_local_residual"] for i in inf_x)}
        ref_c = reference_energies(converged=True)
        if ref_c is not None:
            e_ref = ref_c["energies"]
            for name, a in arms.items():
                n = min(len(e_ref), nmx)
                a["delta_e_vs_converged_oracle"] = max(abs(a["energies"][k] - e_ref[k]) / abs(e_ref[k])
                                                       for k in range(n))
        mixed = {"what": ("the same steps with every local solve converged: mixed bf16 "
                          "(refinement to |r| <= 1e-10 |B|, bf16 inner GMRES(10), FP64-class "
                          "residuals) against plain FP64 GMRES(10) restarted to |r| <= 1e-10 |B|"),
                 **arms,
                 "speedup_mixed_over_fp64": arms["fp64_converged"]["ms_per_step"]
                 / arms["mixed_bf16"]["ms_per_step"],
                 "max_rel_energy_diff": max(abs(a - b) / abs(b) for a, b in
                                            zip(arms["mixed_bf16"]["energies"],
                                                arms["fp64_converged"]["energies"]))}

    ref = reference_energies()
    delta_e = None
    if ref is not None and ref.get("scheme") == args.scheme and rank == 0:
        e_ref = ref["energies"]
        nref = min(len(e_ref), args.steps)
        delta_e = {"reference": ref["what"], "steps": nref,
                   args.precision: max(abs(infos[k]["energy"] - e_ref[k]) / abs(e_ref[k])
                                       for k in range(nref))}
        if fp64 is not None:
            n = min(nref, n64)
            delta_e["fp64"] = max(abs(infos64[k]["energy"] - e_ref[k]) / abs(e_ref[k])
                                  for k in range(n))
            delta_e["fp64_steps"] = n

    heff_rates = heff_kernel_rates(api, ctx, H, args.precision) if rank == 0 else None
    lp_rates = heff_lp_rates(api, ctx, ("mixed_bf16", "mixed_tf32")) if rank == 0 else None

    heff = prof["heff"]
    heff_tf = heff["flops"] / (heff["ms"] * 1e-3) / 1e12 if heff["ms"] > 0 else 0.0
    jac, lq = prof["jacobi"], prof["lq"]
    jac_dev_tf = svd["jacobi_fp64_flops"] / (jac["ms"] * 1e-3) / 1e12 if jac["ms"] > 0 else 0.0
    jac_alg = svd["svd_alg_flops"]
    jac_tf = jac_alg / (jac["ms"] * 1e-3) / 1e12 if jac["ms"] > 0 else 0.0
    lq_tf = lq["flops"] / (lq["ms"] * 1e-3) / 1e12 if lq["ms"] > 0 else 0.0
    breakdown = {k: round(v["ms"] / args.steps, 3) for k, v in prof.items()}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_SITES, "chi_max": CHI, "cutoff": CUTOFF,
                       "scheme": SCHEME_NAMES[args.scheme], "precision": args.precision,
                       "steps_timed": f"grid steps 0..{args.steps - 1} from the start state",
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (state 134 MB + environments 0.7 GB per chain)"},
            "e2e": {"value": whole_job_rate(world, args.steps, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": hio.h2d // args.steps,
                    "d2h_bytes_per_step": hio.d2h // args.steps,
                    "same_steps_as_value": True, "same_energies_as_value": e2e_same},
            "gpu_launches": int(launches),
            "roofline": {"kernel": "k_jacobi_persistent (one-sided Jacobi of the SVD splits)",
                         "bound": "alu", "achieved": jac_tf, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": jac_tf / FP64_PEAK_TFLOPS,
                         "traffic": JACOBI_TRAFFIC_BYTES,
                         "traffic_note": JACOBI_TRAFFIC_NOTE,
                         "achieved_note": ("algorithmic SVD work (22 n^3-class count: 8.7 GFLOP "
                                           "per 512 x 512 split, scaled by m n min(m,n)) over "
                                           "the Jacobi kernel's CUDA-event time"),
                         "device_counted_tflops": jac_dev_tf,
                         "launches": jac["count"], "ms_per_launch": jac["ms"] / max(1, jac["count"]),
                         "peak_note": ("derived, not measured: FP64 pipe from unit counts and "
                                       "clocks (152 SMs x 4 FLOP/clk x 2.07 GHz)"),
                         "share_of_step": jac["ms"] / max(1e-9, prof["step"]["ms"])},
            "roofline_other": {
                "lq": {"kernel": "k_lq_persistent (Householder LQ of the SVD splits)", "bound": "alu",
                       "achieved": lq_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": lq_tf / FP64_PEAK_TFLOPS,
                       "share_of_step": lq["ms"] / max(1e-9, prof["step"]["ms"])},
                "heff": {"kernel": "two-site H_eff in the step", "precision": args.precision,
                         "achieved": heff_tf, "unit": "TFLOP/s",
                         "share_of_step": heff["ms"] / max(1e-9, prof["step"]["ms"])}},
            "heff_kernel": {"precision": args.precision, "shapes": "d=2, D=5, chi_l=chi_r=chi",
                            **(heff_rates or {})},
            "fp64_arm": fp64,
            "equal_accuracy": mixed,
            "heff_lp_kernel": lp_rates,
            "delta_e_vs_oracle": delta_e,
            "stage_ms_per_step": breakdown,
            "step_ms": [round(x, 3) for x in step_ms],
            "heff_calls_per_step": heff["count"] // max(1, args.steps),
            "svd_jacobi": svd,
            "energies": [i["energy"] for i in infos],
            "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(args.bonds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_batch(args):
    """Served execution of the batched workload: --jobs Heisenberg chains (64
    at the full specification) with N drawn from {16, 24, 32, 48, 64} and
    chi_max from {32, 64, 128, 256} (seed 4000), random product starts (seed
    4000 + i), backward Euler on the geometric grid 1e-2 -> 1e2 in --steps steps
    (30 at the full specification), shift = the current energy, in
    --precision (mixed_bf16: bf16 contractions with fp32 accumulation, FP64
    SVD and Krylov, local solves refined to 1e-10).  The same jobs run served
    on --slots workers with the splits' Jacobi grouped across jobs, served
    without grouping, and (unless --no-single) one at a time.  Prints one JSON
    line (not the benchmark line): tau-steps/s, p50/p99 latency, the grouped
    launches, and the speed-ups."""
    import torch
    from paper_2606_02930_gb300 import api, inputs
    torch.cuda.init()
    rng = np.random.default_rng(4000)
    Ns = rng.choice([int(x) for x in args.batch_ns.split(",")], size=args.jobs)
    chis = rng.choice([int(x) for x in args.batch_chis.split(",")], size=args.jobs)
    prec = args.precision
    if prec.startswith("mixed"):
        opts = api.solver_opts(precision=prec, refine_tol=1e-10, refine_max=20)
    else:
        opts = api.solver_opts(precision=prec)

    def make():
        return [api.Job("heisenberg", int(N), inputs.random_product_state(int(N), 2, 4000 + i),
                        int(chi), 1e-10, 1e-2, 1e2, args.steps, scheme="be", opts=opts)
                for i, (N, chi) in enumerate(zip(Ns, chis))]

    api.evolve_batch(make()[:2], n_slots=2)          # warm-up: build caches, page in kernels
    out = {"workload": "batch", "metric": "tau-steps/s and p50/p99 latency of served jobs",
           "jobs": int(args.jobs), "steps_per_job": args.steps, "precision": prec,
           "sample": (f"Heisenberg N in {{{args.batch_ns}}}, chi_max in {{{args.batch_chis}}} "
                      "(seed 4000), BE 1e-2 -> 1e2, shift = current energy"),
           "chi_max_drawn": [int(c) for c in chis], "N_drawn": [int(n) for n in Ns]}
    arms = [] if args.no_grouped else [("grouped", args.slots, args.grouping_mode)]
    arms.append(("ungrouped", args.slots, 0))
    if not args.no_single:
        arms.append(("one_at_a_time", 1, 0))
    energies = {}
    for name, slots, grouping in arms:
        jobs = make()
        res, st = api.evolve_batch(jobs, n_slots=slots, grouping=grouping)
        assert all(r["status"] == 0 for r in res)
        energies[name] = [float(r["energy"]) for r in res]
        out[name] = {"slots": slots, "grouping_mode": grouping,
                     **{k: st[k] for k in ("tau_steps_per_s", "p50_latency_ms",
                                                           "p99_latency_ms", "wall_ms",
                                                           "peak_running", "group_launches",
                                                           "group_items")}}
    out["same_energies"] = all(energies[a] == energies["ungrouped"] for a in energies)
    if "grouped" in out:
        out["speedup_grouped_over_ungrouped"] = (out["grouped"]["tau_steps_per_s"]
                                                 / out["ungrouped"]["tau_steps_per_s"])
    if "one_at_a_time" in out:
        out["speedup_served_over_one_at_a_time"] = (out["ungrouped"]["tau_steps_per_s"]
                                                     / out["one_at_a_time"]["tau_steps_per_s"])
    print(json.dumps(out), flush=True)


def run_metts(args):
    """Independent METTS chains of the impurity model served side by side: the
    paper's METTS setting (trapezoid rule, panel grid from [0, 0.01] with 4
    steps per panel, shift = the current energy, all non-zero singular values
    kept below the cap, double occupancy of the impurity measured) on a
    flat-band bath of 9 sites (Gamma = 0.05, U = 0.3), chi cap 64, beta = 16,
    --jobs chains of 2 samples each from seeded configurations (seed 5000),
    tensor-core mode.  Runs the chains one at a time (1 slot) and side by side
    (--slots) and prints one JSON line (not the benchmark line): METTS
    samples/s, tau-steps/s and p50/p99 chain latency."""
    import torch
    from paper_2606_02930_gb300 import api, inputs
    torch.cuda.init()
    n_bath, beta, samples = 9, 16.0, 2
    eps, V = inputs.flat_band_bath(n_bath)
    P = int(np.ceil(np.log2(0.5 * beta / 0.01))) + 1
    docc = np.diag([0.0, 0.0, 0.0, 1.0]).astype(complex)
    rng = np.random.default_rng(5000)
    cfgs = rng.integers(0, 4, size=(args.jobs, n_bath + 1))
    us = rng.random((args.jobs, samples, n_bath + 1))
    opts = api.solver_opts(precision=args.precision)

    def make():
        return [api.MettsJob("anderson", n_bath, cfgs[i], 64, 0.0, 0.5 * beta, P, 4, us[i],
                             obs=docc, obs_site=0, U=0.3, eps_d=-0.15, eps=eps, V=V, opts=opts)
                for i in range(args.jobs)]

    api.evolve_batch(make()[:2], n_slots=2)          # warm-up: caches, kernel images
    out = {"workload": "metts", "metric": "METTS samples/s and p50/p99 chain latency, served",
           "chains": int(args.jobs), "samples_per_chain": samples, "steps_per_sample": 4 * P,
           "precision": args.precision,
           "config": {"model": "Anderson impurity, flat-band bath of 9 sites, U=0.3, eps_d=-U/2",
                      "beta": beta, "chi_cap": 64, "cutoff": 0.0, "scheme": "trapezoid",
                      "grid": f"panels from [0, {0.5 * beta / 2 ** (P - 1):.4g}], 4 steps/panel",
                      "start": "seeded configurations (seed 5000)"}}
    for slots in (1, args.slots):
        res, st = api.evolve_batch(make(), n_slots=slots)
        assert all(r["status"] == 0 for r in res)
        out[f"slots{slots}"] = {"samples_per_s": args.jobs * samples / (st["wall_ms"] * 1e-3),
                                **{k: st[k] for k in ("tau_steps_per_s", "p50_latency_ms",
                                                      "p99_latency_ms", "wall_ms",
                                                      "peak_running")}}
    out["speedup"] = (out[f"slots{args.slots}"]["samples_per_s"]
                      / out["slots1"]["samples_per_s"])
    print(json.dumps(out), flush=True)


def run_chi_study(args):
    """Bond-dimension growth and step cost of the paper's Heisenberg run (App.
    C): XXX chain of --study-n spins (J = 1, open ends) from the Neel state,
    trapezoid rule on the panel grid (first panel [0, 2^-5], 4 steps per
    panel) up to tau_max = 2^--study-m, discarded weight 1e-10 per bond, chi
    capped at --study-chi, shift = the current energy, tensor-core mode.  Every
    step is one synchronous library call, timed by the host clock around it.
    Fits the step cost t(chi) = a chi^p and the growth chi(tau) (logarithmic
    and power laws), and sets the measured cost of the logarithmic grid
    against uniform steps of 0.1 (the paper's TDVP step) predicted from the
    fit on the same evolution.  Prints one JSON line (not the benchmark line)."""
    import torch
    from paper_2606_02930_gb300 import api, costmodel
    torch.cuda.init()
    N, m, cap = args.study_n, args.study_m, args.study_chi
    opts = api.solver_opts(precision=args.precision)
    ctx = api.ctx_create(0)
    neel = np.zeros((N, 2))
    neel[np.arange(N), np.arange(N) % 2] = 1.0
    # warm-up on a short chain: kernel images, caches
    Hw = api.mpo_create_heisenberg(ctx, 8)
    pw = api.mps_create_product(ctx, neel[:8], 8)
    for dt in (0.01, 0.02, 0.04):
        api.implicit_step(ctx, Hw, pw, dt, "tr", 0.0, 8, CUTOFF, opts)
    H = api.mpo_create_heisenberg(ctx, N)
    psi = api.mps_create_product(ctx, neel, cap)
    P = m + 5 + 1
    nodes = api.grid_panels(2.0 ** m, P, 4)
    s = api.energy(ctx, H, psi)
    taus, chis, secs, energies = [], [], [], []
    for k in range(1, len(nodes)):
        t0 = time.perf_counter()
        info = api.implicit_step(ctx, H, psi, nodes[k] - nodes[k - 1], "tr", s, cap, CUTOFF, opts)
        secs.append(time.perf_counter() - t0)
        s = info["energy"]
        taus.append(float(nodes[k]))
        chis.append(int(info["max_chi"]))
        energies.append(float(s))
    taus, chis_a, secs_a = np.array(taus), np.array(chis), np.array(secs)
    big = chis_a >= 16
    a, p = costmodel.fit_power_law(chis_a[big], secs_a[big])
    grow = chis_a < cap
    growth = costmodel.fit_growth(taus[grow & (taus >= 0.1)], chis_a[grow & (taus >= 0.1)])
    t_fit = lambda c: a * np.maximum(c, 16.0) ** p
    ratios = {}
    for j in range(0, m + 1):
        tmax = 2.0 ** j
        c_log = float(np.sum(secs_a[taus <= tmax + 1e-12]))
        c_uni = costmodel.uniform_cost(tmax, 0.1, nodes, chis, t_fit)
        ratios[str(int(tmax))] = {"log_grid_s": c_log, "uniform_0.1_s": c_uni,
                                  "ratio": c_uni / c_log}
    at_cap = secs_a[chis_a == cap]
    out = {"workload": "chi_study", "metric": "chi(tau), step cost t(chi), App. C cost sums",
           "config": {"model": f"Heisenberg XXX N={N} J=1 OBC, Neel start", "scheme": "trapezoid",
                      "grid": f"panels, first [0, 2^-5], 4 steps/panel, tau_max 2^{m}",
                      "cutoff": CUTOFF, "chi_cap": cap, "shift": "current energy",
                      "precision": args.precision},
           "steps": len(taus), "total_s": float(np.sum(secs_a)),
           "step_cost_fit": {"a": a, "p": p, "over": "steps with chi >= 16"},
           "growth_fit": growth,
           "cost_vs_tau_max": ratios,
           "at_cap": ({"steps": int(at_cap.size), "mean_s": float(at_cap.mean()),
                       "min_s": float(at_cap.min()), "max_s": float(at_cap.max()),
                       "dtau_range": [float(np.min(np.diff(nodes)[chis_a == cap])),
                                      float(np.max(np.diff(nodes)[chis_a == cap]))]}
                      if at_cap.size else None),
           "trace": {"tau": taus.tolist(), "chi": chis, "s": [round(x, 4) for x in secs],
                     "energy": energies}}
    print(json.dumps(out), flush=True)


def oracle_anderson_sample(chi, n_bonds):
    """The oracle on the impurity workload at a saturated bond dimension chi
    (random isometries, seed 3000): seconds per bulk two-site update of the
    first step (gauge move and environments untimed; backward Euler, dtau =
    1e-2, shift = the state's energy), over n_bonds updates from the
    impurity end; and the number of bulk-equivalent updates of a step."""
    from oracle import linsolve as ls, mpo as ompo, mps as omps
    from paper_2606_02930_gb300 import inputs
    n_bath, d = 99, 4
    eps, V = inputs.flat_band_bath(n_bath)
    Ws = ompo.anderson_mpo(-0.15, 0.3, eps, V)
    N = n_bath + 1
    A = inputs.random_isometric_mps(N, d, chi, 3000)
    s = omps.expect_mpo(A, Ws)
    c = 1e-2
    x = ls.right_canonicalize_svd(A)
    Rop, Rov = ls._build_right_envs(Ws, x, [("op", x), ("ov", A)])
    Lop, Lov = np.ones((1, 1, 1), complex), np.ones((1, 1), complex)
    alpha = 1.0 - c * s
    cap = [1] + inputs.bond_profile(N, d, chi) + [1]
    first_bulk = next(i for i in range(N - 1) if cap[i] == chi and cap[i + 2] == chi)
    t_bulk, n_done, i = 0.0, 0, 0
    while n_done < n_bonds:
        t1 = time.perf_counter()
        B = ls.project_two_site(Lov, A[i], A[i + 1], Rov[i + 1])
        X0 = np.tensordot(x[i], x[i + 1], axes=([2], [0]))
        mv = lambda V: alpha * V + c * ls.heff_apply(Lop, Ws[i], Ws[i + 1], Rop[i + 1], V)
        X, _ = ls.gmres(mv, B, X0, 10)
        x[i], x[i + 1], _, _ = ls.split_two_site(X, chi, 1e-14, True)
        Lop = ls.left_env_update(Lop, x[i], Ws[i], x[i])
        Lov = ls.left_overlap_update(Lov, x[i], A[i])
        if i >= first_bulk:
            t_bulk += time.perf_counter() - t1
            n_done += 1
        i += 1

    def fl(chl, chr_):
        return 6 * d * d * chl * chr_ * (chl + chr_) + 2 * 36 * d ** 3 * chl * chr_
    bulk = fl(chi, chi)
    equiv = 2.0 * sum(fl(cap[j], cap[j + 2]) / bulk for j in range(N - 1))
    return t_bulk / n_bonds, equiv


def run_anderson(args):
    """The first --steps steps of the Anderson-impurity evolution: impurity plus
    99 bath sites (N = 100, d = 4, MPO bond dimension 6), flat band of
    half-bandwidth 1 linearly discretised, Gamma = 0.05, U = 0.3, eps_d = -U/2,
    chi_max = 512, cutoff 1e-14, backward Euler on the geometric grid
    1e-2 -> 1e4 (50 steps), shift = the current energy (App. D), from a seeded
    random product state (seed 3000), in --precision.  Every step is one
    synchronous call timed by CUDA events on the context stream, with the
    library's stage timers.  Prints one JSON line (not the benchmark line)."""
    import torch
    from paper_2606_02930_gb300 import api, inputs
    torch.cuda.init()
    n_bath, chi, cutoff = args.anderson_bath, 512, 1e-14
    eps, V = inputs.flat_band_bath(n_bath)
    ctx = api.ctx_create(0)
    H = api.mpo_create_anderson(ctx, eps, V, 0.3, -0.15)
    if args.anderson_start == "saturated":
        # the bond dimension the evolution saturates at: random isometries with
        # slowly decaying bond weights, chi = 512 in the bulk (seed 3000).  The
        # norm of such a state falls geometrically with N (about 1e-74 at N =
        # 100 already at chi = 32), and squared norms of its partial
        # contractions would underflow, so every site is scaled by the same
        # factor that makes the norm 1 (transfer matrices on the host, each
        # renormalised by its trace, the logarithms summed).
        A = inputs.random_isometric_mps(n_bath + 1, 4, chi, 3000)
        E, log_norm2 = np.ones((1, 1), complex), 0.0
        for a in A:
            E = np.tensordot(a.conj(), np.tensordot(E, a, axes=([1], [0])), axes=([0, 1], [0, 1]))
            t = float(np.trace(E).real)
            E /= t
            log_norm2 += np.log(t)
        f = np.exp(-0.5 * log_norm2 / len(A))
        psi = api.mps_create(ctx, [a * f for a in A], chi)
    else:
        vecs = inputs.random_product_state(n_bath + 1, 4, 3000)
        psi = api.mps_create_product(ctx, vecs, chi)
    nodes = api.grid_geometric(1e-2, 1e4, 50)
    opts = api.solver_opts(precision=args.precision)
    s = api.energy(ctx, H, psi)
    stream = torch.cuda.current_stream()
    steps = []
    api.svd_stats(ctx)
    for k in range(args.steps):
        api.profile_start(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = api.implicit_step(ctx, H, psi, nodes[k + 1] - nodes[k], "be", s, chi, cutoff, opts)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = api.profile_stop(ctx)
        svd = api.svd_stats(ctx)
        ms = e0.elapsed_time(e1)
        s = info["energy"]
        steps.append({"k": k, "dtau": float(nodes[k + 1] - nodes[k]), "ms": ms,
                      "energy": info["energy"], "max_chi": info["max_chi"],
                      "max_discarded_weight": info["max_discarded_weight"],
                      "gmres_steps": info["gmres_steps"],
                      "max_local_residual": info["max_local_residual"],
                      "stage_shares": {kk: round(v["ms"] / ms, 4) for kk, v in prof.items()
                                       if kk != "step" and v["ms"] > 0},
                      "svd_sweeps_mean": svd["sweeps_mean"]})
    out = {"workload": "anderson", "metric": "tau-steps/s of the first steps, stage shares",
           "config": {"model": (f"Anderson impurity + {n_bath} bath sites (N={n_bath + 1}, d=4, "
                                f"D=6), flat band D=1, Gamma=0.05, U=0.3, eps_d=-U/2"),
                      "chi_max": chi, "cutoff": cutoff, "scheme": "backward_euler",
                      "grid": "geometric 1e-2 -> 1e4, 50 steps", "shift": "current energy",
                      "start": ("saturated synthetic state (random isometries, chi = 512 in "
                                "the bulk), seed 3000" if args.anderson_start == "saturated"
                                else "random product state, seed 3000"),
                      "precision": args.precision},
           "steps": steps,
           "tau_steps_per_s": len(steps) / (sum(x["ms"] for x in steps) * 1e-3)}
    if not args.no_cpu_baseline:
        t64, eq64 = oracle_anderson_sample(64, 2)
        t128, eq128 = oracle_anderson_sample(128, 2)
        out["cpu_baseline"] = {
            "kind": "oracle, extrapolated", "cores": os.cpu_count(),
            "seconds_per_bulk_update": {"chi64": t64, "chi128": t128},
            "bulk_equivalent_updates": {"chi64": eq64, "chi128": eq128},
            "seconds_per_step": {"chi64": t64 * eq64, "chi128": t128 * eq128},
            "measured_exponent_64_to_128": float(np.log2(t128 / t64)),
            "seconds_per_step_chi512_extrapolated": t128 * eq128 * (512 / 128) ** 3,
            "sample": ("the oracle's first two bulk two-site updates of a step at a saturated "
                       "chi = 64 and chi = 128 (random isometries, seed 3000), times the step's "
                       "bulk-equivalent updates, then the chi^3 law from chi = 128 to 512")}
    print(json.dumps(out), flush=True)


def run_serve(args):
    """A Poisson stream of impurity evolutions through the server, after the
    served workload's arrival process and parameter draws
    (inputs.serve_stream: mean rate --rate per second, seed 5000, U ~ U[0.05,
    0.6], Gamma ~ U[0.02, 0.1], tau_max from {1e2, 1e3, 1e4}, geometric grids
    from 1e-2 with ceil(10 log10(tau_max / 1e-2)) steps, random product
    starts), with the bath sizes and bond caps scaled down to --serve-baths and
    --serve-chis so that the stream finishes in minutes.  The same requests run
    served (--slots workers, mixed bf16) and one at a time in plain FP64 (1
    worker); both arms converge every local solve (refinement / restarted
    GMRES to 1e-8), and each arm's final energies are compared with the
    oracle's converged evolutions (tests/golden/serve_reference_energies.json,
    when it holds this stream).  Prints one JSON line (not the benchmark
    line)."""
    import torch
    from paper_2606_02930_gb300 import api, inputs
    torch.cuda.init()
    n = args.jobs
    baths = tuple(int(x) for x in args.serve_baths.split(","))
    chis = tuple(int(x) for x in args.serve_chis.split(","))
    reqs = inputs.serve_stream(n, args.rate, baths, chis)

    def make(prec):
        if prec == "fp64":
            o = api.solver_opts(precision="fp64", local_tol=1e-8, max_cycles=200)
        else:
            o = api.solver_opts(precision=prec, refine_tol=1e-8, refine_max=20)
        return [api.Job("anderson", r["n_bath"], r["site_vecs"], r["chi_max"], 1e-14, 1e-2,
                        r["tau_max"], r["n_steps"], scheme="be", U=r["U"], eps_d=r["eps_d"],
                        eps=r["eps"], V=r["V"], opts=o) for r in reqs]

    def stream(jobs, slots):
        srv = api.Server(0, n_slots=slots)
        tickets = []
        for j, r in zip(jobs, reqs):
            time.sleep(r["gap_s"])
            tickets.append(srv.submit(j))
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
        srv.close()
        assert all(r["status"] == 0 for r in res), [r["status"] for r in res]
        lat = np.array([r["latency_ms"] for r in res])
        return {"tau_steps_per_s": st["tau_steps_per_s"], "wall_ms": st["wall_ms"],
                "p50_latency_ms": float(np.percentile(lat, 50)),
                "p99_latency_ms": float(np.percentile(lat, 99)),
                "peak_running": st["peak_running"],
                "energies": [float(r["energy"]) for r in res]}

    warm = make("mixed_bf16")[:2]
    api.evolve_batch(warm, n_slots=2)
    served = stream(make("mixed_bf16"), args.slots)
    single = stream(make("fp64"), 1)
    dE = max(abs(a - b) / abs(b) for a, b in zip(served["energies"], single["energies"]))
    out = {"workload": "serve", "metric": "p50/p99 latency and tau-steps/s of a served stream",
           "config": {"requests": n, "rate_per_s": args.rate, "seed": 5000,
                      "bath_sites": list(baths), "chi_max": list(chis),
                      "tau_max": [1e2, 1e3, 1e4], "U": [0.05, 0.6], "Gamma": [0.02, 0.1],
                      "cutoff": 1e-14,
                      "scaled": "bath sizes and bond caps scaled down from the served "
                                "workload's {49,99,199} and {128,...,1024}"},
           "served_mixed_bf16": {k: v for k, v in served.items() if k != "energies"},
           "one_at_a_time_fp64": {k: v for k, v in single.items() if k != "energies"},
           "max_rel_energy_diff_between_arms": dE,
           "throughput_ratio": served["tau_steps_per_s"] / single["tau_steps_per_s"],
           "p99_ratio": single["p99_latency_ms"] / served["p99_latency_ms"]}
    try:
        with open(os.path.join(ROOT, "tests", "golden", "serve_reference_energies.json")) as f:
            ref = json.load(f)
        if ref["n"] == n and tuple(ref["baths"]) == baths and tuple(ref["chis"]) == chis:
            e = ref["energies"]
            for name, arm in (("served_mixed_bf16", served), ("one_at_a_time_fp64", single)):
                out[name]["max_rel_energy_error_vs_oracle"] = max(
                    abs(a - b) / abs(b) for a, b in zip(arm["energies"], e))
    except (OSError, ValueError, KeyError):
        pass
    print(json.dumps(out), flush=True)


def run_only(args):
    """Time one kernel-level entry point at the workload's bulk shape: the
    two-site H_eff (chi = 256, d = 2, D = 5) or the truncated SVD split of a
    512 x 512 two-site block.  Prints one JSON line (not a benchmark line)."""
    import torch
    from paper_2606_02930_gb300 import api, inputs
    ctx = api.ctx_create(0)
    rng = np.random.default_rng(SEED)

    def dev(*shape):
        a = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(shape[-1])
        return torch.from_numpy(a).to("cuda")

    if args.only == "heff_lp":
        prec = args.precision if args.precision.startswith("mixed") else "mixed_bf16"
        shapes = tuple(sh for sh in LP_SHAPES if args.lp_shape in ("all", f"{sh[0]}{sh[3]}"))
        print(json.dumps({"only": "heff_lp", **heff_lp_rates(api, ctx, (prec,), args.steps,
                                                             shapes)}), flush=True)
        return
    H = api.mpo_create_heisenberg(ctx, N_SITES)
    api.set_kernel_precision(ctx, args.precision)
    if args.only == "heff":
        L, R, X = dev(D_MPO, CHI, CHI), dev(D_MPO, CHI, CHI), dev(CHI, D_SITE, D_SITE, CHI)
        Y = torch.empty_like(X)
        call = lambda: api.k_heff(ctx, H, 20, L, R, X, Y)
        flops = 8.0 * (2 * D_MPO * D_SITE ** 2 * CHI ** 3 + 2 * D_MPO ** 2 * D_SITE ** 3 * CHI ** 2)
    else:
        A = inputs.random_isometric_mps(20, D_SITE, CHI, SEED)
        X = torch.from_numpy(np.tensordot(A[9], A[10], axes=([2], [0])).reshape(512, 512)).to("cuda")
        left = torch.empty(512 * 512, dtype=torch.complex128, device="cuda")
        right = torch.empty_like(left)
        tc = args.precision == "fp64_tc"
        call = lambda: api.k_split(ctx, X, 512, 512, CHI, CUTOFF, True, left, right, tc=tc)
        flops = 0.0
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        call()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    out = {"only": args.only, "ms_per_call": ms}
    if flops:
        out["tflops"] = flops / (ms * 1e-3) / 1e12
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.only:
        run_only(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "chi_study":
        run_chi_study(args)
        return
    if args.workload == "metts":
        run_metts(args)
        return
    if args.workload == "anderson":
        run_anderson(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
