"""One implicit imaginary-time step and evolution over a tau grid (oracle).
Test infrastructure only.

Schemes (H' = H - s):
* 'tr' -- implicit trapezoid rule, Eq. 4: (I + c H') psi_k = (I - c H') psi_{k-1}
          with c = dtau/2.  The right-hand side MPS b is a two-site fit of
          (I - c H') psi_{k-1} and is also the initial guess (App. B).
* 'be' -- backward Euler: (I + c H') psi_k = psi_{k-1} with c = dtau; b = psi_{k-1}
          and the initial guess is psi_{k-1}.
* 'fe', 'heun' -- the explicit forward Euler and Heun (predictor-corrector)
          steps, psi_k = (I - dtau H') psi_{k-1} and psi_k = psi_{k-1}/2 +
          (I - dtau H') psi*/2 with psi* the Euler predictor, each product formed
          by two-site fits: the unstable counter-examples of the stability
          section (|1 - z + z^2/2| > 1 once z > 2).
* 'gl<q>' -- q-stage Gauss-Legendre collocation (Method: the spectral panel
          method), which for this linear ODE is psi_k = R_q(dtau H') psi_{k-1}
          with R_q the (q, q) Pade approximant of e^{-z}.  By partial fractions
          R_q(z) = r_inf + sum_j a_j / (z - z_j), so psi_k = r_inf psi_{k-1} +
          sum_j w_j x_j with (I + c_j H') x_j = psi_{k-1}, c_j = -dtau / z_j,
          w_j = -a_j / z_j: q independent shifted solves with complex c_j (each
          from the initial guess psi_{k-1}), then a two-site fit of the sum.
After the solve the state is normalised (Heisenberg section, App. D).  The
shift s is either fixed or, in 'energy' mode, the energy of the current state
(App. D moves the spectrum by the energy of the state the last step produced).
"""
import numpy as np

from . import linsolve as ls
from . import mps as mpsmod


class StepInfo:
    def __init__(self):
        self.energy = 0.0
        self.norm_before = 0.0
        self.max_discarded = 0.0
        self.max_local_residual = 0.0
        self.max_chi = 0
        self.gmres_steps = 0
        self.shift = 0.0


def implicit_step(Ws, psi, dtau, scheme, shift, chi_max, cutoff, krylov_dim=10,
                  local_tol=0.0, sweeps=1, sweep_tol=0.0, fit_sweeps=1, max_cycles=1):
    """Advance the MPS psi (assumed normalised) by one step of size dtau.
    Returns (new normalised MPS, StepInfo)."""
    info = StepInfo()
    info.shift = shift
    if scheme == "be":
        c = dtau
        b = mpsmod.copy(psi)
        x0 = mpsmod.copy(psi)
    elif scheme == "tr":
        c = 0.5 * dtau
        b, finfo = ls.fit_affine(Ws, psi, 1.0 + c * shift, -c, chi_max, cutoff, fit_sweeps)
        info.max_discarded = finfo.max_discarded
        x0 = mpsmod.copy(b)
    elif scheme in ("fe", "heun"):
        # explicit steps (the stability counter-examples): forward Euler
        # psi* = (I - dtau H') psi as a two-site fit; Heun adds the corrector
        # psi_k = psi/2 + (I - dtau H') psi* / 2
        a, b = 1.0 + dtau * shift, -dtau
        y, finfo = ls.fit_affine(Ws, psi, a, b, chi_max, cutoff, fit_sweeps)
        info.max_discarded = finfo.max_discarded
        if scheme == "heun":
            y2, finfo = ls.fit_affine(Ws, y, a, b, chi_max, cutoff, fit_sweeps)
            info.max_discarded = max(info.max_discarded, finfo.max_discarded)
            y, finfo = ls.fit_combination([psi, y2], [0.5, 0.5], chi_max, cutoff, fit_sweeps)
            info.max_discarded = max(info.max_discarded, finfo.max_discarded)
        return _finish(y, info, Ws)
    elif str(scheme).startswith("gl"):
        from .ed import pade_partial_fractions, gl_stages
        z, a, r_inf = pade_partial_fractions(gl_stages(scheme))
        xs, ws = [], []
        for zj, aj in zip(z, a):
            cj = -dtau / zj
            xj, sinfo = ls.linsolve(Ws, mpsmod.copy(psi), psi, cj, shift, chi_max, cutoff,
                                    krylov_dim, local_tol, sweeps, sweep_tol, max_cycles)
            info.max_discarded = max(info.max_discarded, sinfo.max_discarded)
            info.max_local_residual = max(info.max_local_residual, sinfo.max_local_residual)
            info.gmres_steps += sinfo.gmres_steps
            xs.append(xj)
            ws.append(-aj / zj)
        x, finfo = ls.fit_combination([psi] + xs, [r_inf] + ws, chi_max, cutoff, fit_sweeps)
        info.max_discarded = max(info.max_discarded, finfo.max_discarded)
        return _finish(x, info, Ws)
    else:
        raise ValueError(scheme)
    x, sinfo = ls.linsolve(Ws, x0, b, c, shift, chi_max, cutoff, krylov_dim,
                           local_tol, sweeps, sweep_tol, max_cycles)
    info.max_discarded = max(info.max_discarded, sinfo.max_discarded)
    info.max_local_residual = sinfo.max_local_residual
    info.gmres_steps = sinfo.gmres_steps
    return _finish(x, info, Ws)


def _finish(x, info, Ws):
    """Normalise (centre on site 1, the rest right-orthonormal), energy."""
    nrm = float(np.linalg.norm(x[0]))
    x[0] = x[0] / nrm
    info.norm_before = nrm
    info.max_chi = max(mpsmod.bond_dims(x) + [1])
    info.energy = mpsmod.expect_mpo(x, Ws)
    return x, info


def evolve(Ws, psi0, nodes, scheme, chi_max, cutoff, shift_mode="fixed", shift=0.0,
           **kw):
    """Evolve psi0 over the grid `nodes` (t_0 = 0 < t_1 < ...).  Returns
    (list of MPS after each step, list of StepInfo)."""
    psi = mpsmod.copy(psi0)
    nrm = mpsmod.norm(psi)
    psi[0] = psi[0] / nrm
    s = mpsmod.expect_mpo(psi, Ws) if shift_mode == "energy" else shift
    states, infos = [], []
    for k in range(1, len(nodes)):
        psi, info = implicit_step(Ws, psi, nodes[k] - nodes[k - 1], scheme, s, chi_max,
                                  cutoff, **kw)
        states.append(psi)
        infos.append(info)
        if shift_mode == "energy":
            s = info.energy
    return states, infos
