"""Writes the oracle's energies along the benchmark's timed sequence, so that
the benchmark can state each precision mode's energy error against the oracle
without running it: bench_reference_energies.json (the paper's fixed effort,
one GMRES(10) cycle per local solve) and, with --converged,
bench_reference_energies_converged.json (local GMRES restarted until the
relative residual is below 1e-12: the reference of the mixed-precision modes,
whose refinement converges every local solve).

The sequence: Heisenberg chain N = 64 (J = 1, open ends), chi_max = 256,
cutoff 1e-10, start state random_isometric_mps(64, 2, 256, seed 2000),
backward Euler on the geometric grid 1e-3 -> 1e3 (40 steps) from its first
step, shift = the energy of the current state (App. D), one sweep of
GMRES(10) local solves per step (App. B, App. D).  Calls only the oracle and
the seeded input generator.

    python tests/golden/make_bench_reference.py [n_steps] [--converged]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import grid, mpo, mps, step  # noqa: E402
from paper_2606_02930_gb300 import inputs  # noqa: E402

N, CHI, CUTOFF, SEED = 64, 256, 1e-10, 2000


def main(n_steps, converged=False):
    kw = dict(local_tol=1e-12, max_cycles=100) if converged else {}
    Ws = mpo.heisenberg_mpo(N)
    psi = inputs.random_isometric_mps(N, 2, CHI, SEED)
    nodes = grid.geometric_grid(1e-3, 1e3, 40)
    s = mps.expect_mpo(psi, Ws)
    energies, norms, secs = [], [], []
    name = "bench_reference_energies" + ("_converged" if converged else "") + ".json"
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    for k in range(n_steps):
        t0 = time.perf_counter()
        psi, info = step.implicit_step(Ws, psi, nodes[k + 1] - nodes[k], "be", s, CHI, CUTOFF, **kw)
        secs.append(time.perf_counter() - t0)
        s = info.energy
        energies.append(info.energy)
        norms.append(info.norm_before)
        doc = {"what": ("oracle energies after steps 1..n of the benchmark sequence: Heisenberg "
                        "N=64, chi_max=256, cutoff 1e-10, random_isometric_mps seed 2000, backward "
                        "Euler on the geometric grid 1e-3 -> 1e3 (40 steps) from its first step, "
                        "shift = current energy, one sweep of GMRES(10)"
                        + (" cycles restarted to a relative residual of 1e-12" if converged
                           else ", one cycle per local solve")),
               "scheme": "be", "local_solves": "converged" if converged else "fixed",
               "energies": energies, "norms_before": norms,
               "oracle_seconds_per_step": secs}
        with open(out, "w") as f:
            json.dump(doc, f, indent=1)
        print(k + 1, info.energy, f"{secs[-1]:.1f} s", flush=True)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    main(int(args[0]) if args else 8, "--converged" in sys.argv)
