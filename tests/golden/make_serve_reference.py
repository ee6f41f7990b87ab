"""Writes the oracle's final energies of the served impurity stream's
requests, so that the served benchmark can state each arm's energy error
against the oracle without running it: serve_reference_energies.json.

The requests are inputs.serve_stream(n, rate, baths, chis) (seed 5000): the
impurity model with a flat-band bath (App. D, reading c10), backward Euler on
the geometric grid 1e-2 -> tau_max, shift = the energy of the current state
(App. D), bond cap chi_max, cutoff 1e-14, one sweep per step with every local
GMRES(10) solve restarted until its relative residual is below 1e-12 (the
converged reference of reading c13).  Calls only the oracle and the seeded
input generator; requests run in parallel worker processes.

    python tests/golden/make_serve_reference.py [n] [baths] [chis] [workers]
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def final_energy(args):
    n, baths, chis, i = args
    from oracle import grid, mpo, mps, step
    from paper_2606_02930_gb300 import inputs
    r = inputs.serve_stream(n, baths=baths, chis=chis)[i]
    Ws = mpo.anderson_mpo(r["eps_d"], r["U"], r["eps"], r["V"])
    psi = mps.product_state(r["site_vecs"])
    nodes = grid.geometric_grid(1e-2, r["tau_max"], r["n_steps"])
    s = mps.expect_mpo(psi, Ws)
    t0 = time.perf_counter()
    for k in range(r["n_steps"]):
        psi, info = step.implicit_step(Ws, psi, nodes[k + 1] - nodes[k], "be", s, r["chi_max"],
                                       1e-14, local_tol=1e-12, max_cycles=200)
        s = info.energy
    return i, s, time.perf_counter() - t0


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 10
    baths = tuple(int(x) for x in (sys.argv[2] if len(sys.argv) > 2 else "9,19").split(","))
    chis = tuple(int(x) for x in (sys.argv[3] if len(sys.argv) > 3 else "16,32").split(","))
    workers = int(sys.argv[4]) if len(sys.argv) > 4 else min(n, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(workers) as pool:
        res = sorted(pool.map(final_energy, [(n, baths, chis, i) for i in range(n)]))
    doc = {"what": ("oracle final energies of the served impurity stream's requests "
                    "(inputs.serve_stream, seed 5000): backward Euler on the geometric grid "
                    "1e-2 -> tau_max, shift = current energy, cutoff 1e-14, local GMRES(10) "
                    "restarted to a relative residual of 1e-12"),
           "n": n, "baths": list(baths), "chis": list(chis),
           "energies": [e for _, e, _ in res], "oracle_seconds": [t for _, _, t in res]}
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "serve_reference_energies.json")
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps(doc))


if __name__ == "__main__":
    main()
