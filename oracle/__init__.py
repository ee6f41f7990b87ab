"""CPU oracle for implicit imaginary-time stepping of matrix product states.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute anything in this package: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code with the CUDA library under
``paper_2606_02930_gb300/``; both sides receive the same seeded inputs from
``paper_2606_02930_gb300/inputs.py``, which holds no arithmetic of the method.

Everything here is plain NumPy in complex128 (FP64), written for a reader to
check against the paper by eye.  Citations name the paper's sections and
equations ("Method", "Eq. 4", "App. A", ...).

Tiers:

* ``ed``       -- exact dense references: Hamiltonians built by bit
                  operations / explicit fermionic sign counting, the exact
                  propagator of Eq. 1 and the discrete propagators of the
                  backward-Euler and trapezoid steppers (Eq. 4, App. A).
* ``grid``     -- the logarithmic tau grids (Method, panel grid; geometric grid).
* ``mpo``      -- finite-state-machine MPOs for the Heisenberg chain and the
                  Anderson impurity model (star geometry, Jordan-Wigner).
* ``mps``      -- MPS helpers: product states, canonical forms, overlaps,
                  energies and two-point correlators.
* ``linsolve`` -- the two-site DMRG-style MPO-MPS linear solve with GMRES
                  local solves (Method, App. B) and the two-site fit used to
                  form the trapezoid right-hand side.
* ``step``     -- one implicit step and evolution over a tau grid.

Parity status: the pins live in ``tests/test_oracle_*.py``.  The paper-faithful
fixed-effort mode (one sweep, one GMRES(10) cycle per bond) has no closed form;
it is pinned only through its converged limit (equal to the dense discrete
propagator) and invariants.  That mode is therefore "parity unpinned" beyond
those checks.
"""
