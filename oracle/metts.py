"""METTS (minimally entangled typical thermal states) on top of the implicit
steps (oracle).  Test infrastructure only.

The paper pairs its imaginary-time evolution with METTS for the
Anderson-impurity study (Anderson-impurity section): a chain of classical
product states |sigma>; each is evolved to |phi> = e^{-beta H / 2}|sigma>
(normalised) and measured, and the next product state is drawn with
probability |<sigma'|phi>|^2.  Averages of the measurements over the chain
estimate thermal averages at inverse temperature beta.

The draw is sequential in the computational basis: with the state in
right-canonical form (orthogonality centre on the first site), the
conditional probability of s at site i given the earlier choices is
|v A_i[:, s, :]|^2 / sum_s' |v A_i[:, s', :]|^2, v the normalised row
vector of the earlier choices; s is the smallest value whose cumulative
conditional probability exceeds the uniform number u_i (when rounding leaves
the total below u_i, the last value of nonzero probability).  The uniform
numbers are inputs, so that a chain is a deterministic function of them.
"""
import numpy as np

from . import ed
from . import mps as mpsmod
from . import step as stepmod


def sample(psi, u, basis=None):
    """Draw a configuration from |<sigma|psi>|^2 / <psi|psi>, sigma a product
    of the columns of `basis` (d x d unitary; None: the computational basis).
    Returns (config list, its probability)."""
    x = mpsmod.right_canonicalize(psi)
    v = np.ones(1, complex)
    config, prob = [], 1.0
    for i, A in enumerate(x):
        M = np.tensordot(v, A, axes=([0], [0]))          # (d, chi_right)
        if basis is not None:
            M = np.asarray(basis).conj().T @ M               # <b_s| components
        w = np.sum(np.abs(M) ** 2, axis=1)
        p = w / np.sum(w)
        s = _draw(p, u[i])
        config.append(s)
        prob *= p[s]
        v = M[s] / np.sqrt(w[s])
    return config, prob


def _draw(p, u):
    """Smallest s whose cumulative probability exceeds u; if rounding leaves
    the total at or below u, the last s of nonzero probability."""
    cum = 0.0
    for k in range(len(p)):
        cum += p[k]
        if cum > u:
            return k
    nz = np.nonzero(p > 0)[0]
    return int(nz[-1]) if nz.size else len(p) - 1


def product_tensors(config, d, basis=None):
    """Product state |config> as site tensors (1, d, 1), each site the column
    config[i] of `basis` (None: the computational basis)."""
    out = []
    B = np.eye(d) if basis is None else np.asarray(basis)
    for s in config:
        out.append(B[:, s].astype(complex).reshape(1, d, 1))
    return out


# collapse bases of the alternating chain (spin 1/2: z, then x); the
# alternation lets the chain leave the conserved-magnetisation sector of its
# start state
X_BASIS = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)


def metts_chain(Ws, config0, d, nodes, n_samples, uniforms, chi_max, cutoff, obs=None,
                obs_site=0, scheme="be", alt_basis=None, shift_mode="energy", shift=0.0, **kw):
    """METTS chain from config0 (computational basis): per sample, evolve the
    product state over the tau grid `nodes` (0 -> beta/2; shift as
    step.evolve, the current energy by default), record the energy and
    <obs at obs_site>, then draw the next configuration with uniforms[k] (N
    numbers) in the computational basis, or, after even samples when
    alt_basis is given, in that basis.  Returns (energies, observables,
    configurations)."""
    config, basis = list(config0), None
    energies, values, configs = [], [], []
    for k in range(n_samples):
        states, infos = stepmod.evolve(Ws, product_tensors(config, d, basis), nodes, scheme,
                                       chi_max, cutoff, shift_mode=shift_mode, shift=shift, **kw)
        phi = states[-1]
        energies.append(infos[-1].energy)
        if obs is not None:
            values.append(mpsmod.correlator(phi, obs, obs_site, np.eye(d), obs_site).real)
        basis = alt_basis if (alt_basis is not None and k % 2 == 0) else None
        config, _ = sample(phi, uniforms[k], basis)
        configs.append(list(config))
    return energies, values, configs


def dense_metts_chain(H, d, N, config0, beta, uniforms, obs_dense=None, nodes=None, scheme="be",
                      alt_basis=None):
    """The same chain on dense vectors with dense sampling (sequential
    conditional draws on the amplitude tensor).  With nodes, each sample is
    evolved by the discrete scheme on that grid with shift = the current
    energy (ed.propagate_discrete); without, by the exact e^{-beta H / 2}."""
    evals, evecs = np.linalg.eigh(H)
    prop = (evecs * np.exp(-0.5 * beta * (evals - evals[0]))) @ evecs.conj().T
    config, basis = list(config0), None
    energies, values = [], []
    for k, u in enumerate(uniforms):
        B = np.eye(d) if basis is None else np.asarray(basis)
        e = B[:, config[0]].astype(complex)
        for s in config[1:]:
            e = np.kron(e, B[:, s])
        if nodes is None:
            v = prop @ e
        else:
            states, _, _ = ed.propagate_discrete(H, e, np.diff(nodes), scheme, shift_mode="energy")
            v = states[-1]
        v = v / np.linalg.norm(v)
        energies.append(ed.energy(H, v))
        if obs_dense is not None:
            values.append(np.vdot(v, obs_dense @ v).real)
        basis = alt_basis if (alt_basis is not None and k % 2 == 0) else None
        amp = v.reshape([d] * N)
        if basis is not None:
            for i in range(N):      # <b_s| on every site
                amp = np.moveaxis(np.tensordot(np.asarray(basis).conj().T, amp, axes=([1], [i])), 0, i)
        config = []
        for i in range(N):
            w = np.abs(amp) ** 2
            if w.ndim > 1:
                w = np.sum(w, axis=tuple(range(1, w.ndim)))
            s = _draw(w / np.sum(w), u[i])
            config.append(s)
            amp = amp[s]
    return energies, values
