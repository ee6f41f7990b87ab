"""Exact dense references (oracle tier O1).  Test infrastructure only.

* Heisenberg chain H = J sum_j (Sx_j Sx_{j+1} + Sy_j Sy_{j+1}) + Jz sum_j Sz_j Sz_{j+1}
  (Heisenberg-chain section; Jz = J is the isotropic model of the paper).
  Basis: site 1 is the most significant digit of the dense index; local
  index 0 = spin up (Sz = +1/2), 1 = spin down.
* Anderson impurity model (Anderson-impurity section): impurity at site 0,
  bath sites 1..N_b, local basis {|0>, |up>, |down>, |up down>} with local
  index n_up + 2 n_down.  Built in Fock space with explicit fermionic sign
  counting over the mode order (0 up, 0 down, 1 up, 1 down, ...), which is
  independent of any Jordan-Wigner string construction.
* Propagators: the exact evolution of Eq. 1, and the discrete steppers whose
  one-step amplification factors are R_BE(z) = 1/(1+z) (backward Euler) and
  R_TR(z) = (1 - z/2)/(1 + z/2) (implicit trapezoid rule, Eq. 4 and App. A),
  applied through the eigendecomposition of H.
"""
import numpy as np


# ---------------------------------------------------------------- Heisenberg
def heisenberg_hamiltonian(N, J=1.0, Jz=None):
    """Dense Heisenberg Hamiltonian on N sites, open boundaries, by bit operations."""
    Jz = J if Jz is None else Jz
    dim = 1 << N
    H = np.zeros((dim, dim))
    for state in range(dim):
        for j in range(N - 1):
            pj, pk = N - 1 - j, N - 2 - j          # bit positions of sites j, j+1
            bj, bk = (state >> pj) & 1, (state >> pk) & 1   # 1 means spin down
            H[state, state] += Jz * (0.5 - bj) * (0.5 - bk)
            if bj != bk:                            # (S+S- + S-S+)/2 flips the pair
                H[state ^ (1 << pj) ^ (1 << pk), state] += 0.5 * J
    return H


# ---------------------------------------------------------------- Anderson
def _occ(idx, mode, n_sites):
    site, spin = divmod(mode, 2)
    return (idx >> (2 * (n_sites - 1 - site) + spin)) & 1


def _flip(idx, mode, n_sites):
    site, spin = divmod(mode, 2)
    return idx ^ (1 << (2 * (n_sites - 1 - site) + spin))


def _sign_before(idx, mode, n_sites):
    """(-1)^(number of occupied modes preceding `mode` in the mode order)."""
    s = 0
    for m in range(mode):
        s += _occ(idx, m, n_sites)
    return -1.0 if (s & 1) else 1.0


def _hop(idx, p, q, n_sites):
    """Apply c_p^dagger c_q to basis state idx.  Returns (new_idx, amplitude) or None."""
    if not _occ(idx, q, n_sites):
        return None
    s1 = _sign_before(idx, q, n_sites)
    mid = _flip(idx, q, n_sites)
    if _occ(mid, p, n_sites):
        return None
    s2 = _sign_before(mid, p, n_sites)
    return _flip(mid, p, n_sites), s1 * s2


def anderson_hamiltonian(eps_d, U, eps, V):
    """Dense single-impurity Anderson Hamiltonian (Anderson-impurity section):

        H = eps_d n_d + U n_d,up n_d,down + sum_{j,s} eps_j n_{j,s}
            + sum_{j,s} V_j (d^dag_s c_{j,s} + c^dag_{j,s} d_s)
    """
    eps = np.asarray(eps, float)
    V = np.asarray(V, float)
    n_sites = 1 + len(eps)
    dim = 1 << (2 * n_sites)
    H = np.zeros((dim, dim))
    for idx in range(dim):
        nu, nd = _occ(idx, 0, n_sites), _occ(idx, 1, n_sites)
        diag = eps_d * (nu + nd) + U * nu * nd
        for j in range(1, n_sites):
            diag += eps[j - 1] * (_occ(idx, 2 * j, n_sites) + _occ(idx, 2 * j + 1, n_sites))
        H[idx, idx] += diag
        for j in range(1, n_sites):
            for spin in range(2):
                d_mode, c_mode = spin, 2 * j + spin
                for p, q in ((d_mode, c_mode), (c_mode, d_mode)):
                    r = _hop(idx, p, q, n_sites)
                    if r is not None:
                        H[r[0], idx] += V[j - 1] * r[1]
    return H


def single_particle_matrix(eps_d, eps, V):
    """One-body (per spin) matrix of the U=0 Anderson model: impurity level,
    bath levels and hybridisations V_j (star geometry)."""
    nb = len(eps)
    h = np.zeros((nb + 1, nb + 1))
    h[0, 0] = eps_d
    h[np.arange(1, nb + 1), np.arange(1, nb + 1)] = eps
    h[0, 1:] = V
    h[1:, 0] = V
    return h


# ---------------------------------------------------------------- propagators
def pade_denominator(q):
    """Coefficients p_0..p_q of the denominator of the (q, q) Pade approximant
    of e^{-z}: P_q(z) = sum_k (2q-k)! q! / ((2q)! k! (q-k)!) z^k, so that
    e^{-z} ~ P_q(-z) / P_q(z) with error O(z^{2q+1})."""
    from math import factorial
    return np.array([factorial(2 * q - k) * factorial(q)
                     / (factorial(2 * q) * factorial(k) * factorial(q - k)) for k in range(q + 1)])


def gl_stages(scheme):
    """Number of Gauss-Legendre stages q of a scheme name 'gl<q>'."""
    return int(scheme[2:])


def pade_partial_fractions(q):
    """R_q(z) = P_q(-z)/P_q(z) = r_inf + sum_j a_j / (z - z_j): the poles z_j
    (roots of P_q), the residues a_j = P_q(-z_j) / P_q'(z_j) and r_inf =
    (-1)^q.  For a linear ODE the q-stage Gauss-Legendre collocation step is
    this rational function of z = dtau (H - s) (Method: Gauss-Legendre
    collocation on each panel)."""
    p = pade_denominator(q)
    poly = np.polynomial.Polynomial(p)
    num = np.polynomial.Polynomial(p * (-1.0) ** np.arange(q + 1))
    z = np.roots(p[::-1]).astype(complex)
    a = num(z) / poly.deriv()(z)
    return z, a, (-1.0) ** q


def amplification(z, scheme):
    """One-step amplification factor of the linear test problem y' = -lambda y
    at z = lambda * dtau (App. A).  'be': backward Euler; 'tr': implicit
    trapezoid rule (Eq. 4); 'fe': forward Euler and 'heun': Heun's explicit
    predictor-corrector step (the explicit counter-examples of the stability
    section);
    'gl<q>': q-stage Gauss-Legendre collocation, the (q, q) Pade approximant
    P_q(-z) / P_q(z) of e^{-z}."""
    if str(scheme).startswith("gl"):
        p = pade_denominator(gl_stages(scheme))
        zz = np.asarray(z)
        num = sum(c * (-zz) ** k for k, c in enumerate(p))
        den = sum(c * zz ** k for k, c in enumerate(p))
        return num / den
    z = np.asarray(z, dtype=float)
    if scheme == "be":
        return 1.0 / (1.0 + z)
    if scheme == "tr":
        return (1.0 - 0.5 * z) / (1.0 + 0.5 * z)
    if scheme == "fe":
        return 1.0 - z
    if scheme == "heun":
        # explicit trapezoid (predictor-corrector) step: 1 - z + z^2 / 2
        return 1.0 - z + 0.5 * z * z
    raise ValueError(scheme)


def propagate_discrete(H, psi0, dtaus, scheme, shifts=None, shift_mode="fixed",
                       normalize=True):
    """Apply prod_k R(dtau_k (H - s_k)) to psi0 through the eigendecomposition of H.

    shift_mode 'fixed': s_k = shifts[k] (scalar or array, default 0).
    shift_mode 'energy': s_k = <psi_{k-1}|H|psi_{k-1}> of the current normalised
    state (Anderson-model appendix: shift by the energy of the time-evolved state).
    Returns (list of states after each step, list of norms before normalising,
    list of shifts used)."""
    evals, evecs = np.linalg.eigh(H)
    coef = evecs.conj().T @ np.asarray(psi0, complex)
    coef = coef / np.linalg.norm(coef)
    K = len(dtaus)
    if shifts is None:
        shifts = np.zeros(K)
    shifts = np.broadcast_to(np.asarray(shifts, float), (K,))
    states, norms, used = [], [], []
    for k in range(K):
        if shift_mode == "energy":
            s = float(np.real(np.vdot(coef, evals * coef)) / np.vdot(coef, coef).real)
        else:
            s = float(shifts[k])
        coef = amplification(dtaus[k] * (evals - s), scheme) * coef
        nrm = np.linalg.norm(coef)
        norms.append(nrm)
        used.append(s)
        if normalize:
            coef = coef / nrm
        states.append(evecs @ coef)
    return states, norms, used


def propagate_exact(H, psi0, taus):
    """Normalised e^{-H tau} psi0 for each tau (Eq. 1)."""
    evals, evecs = np.linalg.eigh(H)
    coef = evecs.conj().T @ np.asarray(psi0, complex)
    out = []
    e0 = evals[0]
    for t in taus:
        v = evecs @ (np.exp(-(evals - e0) * t) * coef)
        out.append(v / np.linalg.norm(v))
    return out


def energy(H, psi):
    psi = np.asarray(psi, complex)
    return float(np.real(np.vdot(psi, H @ psi)) / np.vdot(psi, psi).real)


def infidelity(psi, phi):
    """1 - |<psi|phi>| / (|psi| |phi|): phase-free state distance."""
    return 1.0 - abs(np.vdot(psi, phi)) / (np.linalg.norm(psi) * np.linalg.norm(phi))


def trapezoid_local_error(lam, a, b):
    """Local error of the trapezoid rule on one mode e^{-lam tau} over [a, b]
    (App. A): trapezoid approximation of lam * int_a^b e^{-lam tau} minus the
    exact integral, evaluated from the definition."""
    h = b - a
    trap = 0.5 * lam * h * (np.exp(-a * lam) + np.exp(-b * lam))
    exact = np.exp(-a * lam) - np.exp(-b * lam)
    return trap - exact
