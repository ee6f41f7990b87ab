"""Seeded synthetic inputs shared by the CUDA library's tests/benchmarks and
the CPU oracle.

This module holds no arithmetic of the method: it only draws random numbers
and lays out the model parameters of the synthetic workloads.  Both sides
receive these arrays as data.

Workloads (random complex states; the paper's own runs use a Neel state, a
29-site sum-of-poles bath and U in {8,...,15}, which these stand in for):

* ``heisenberg_small``  -- XXX chain N=10, J=1, chi_max=32, cutoff 0,
  backward Euler on a geometric grid 1e-2 -> 1e2 with 20 steps.
* ``heisenberg_bulk``   -- XXX chain N=64, J=1, chi_max=256, cutoff 1e-10,
  geometric grid 1e-3 -> 1e3 with 40 steps, backward Euler and trapezoid.
* ``anderson_flat``     -- impurity + 99 bath sites, flat band of
  half-bandwidth 1, Gamma=0.05, U=0.3, eps_d=-U/2, chi_max=512,
  cutoff 1e-14, geometric grid 1e-2 -> 1e4 with 50 steps.
"""
import numpy as np


def random_product_state(N, d, seed):
    """Per-site normalised random complex d-vectors (g1 + i g2, ...)/norm with
    g ~ N(0,1) from numpy's default_rng(seed), drawn in site order."""
    rng = np.random.default_rng(seed)
    out = np.empty((N, d), complex)
    for i in range(N):
        g = rng.standard_normal(2 * d)
        v = g[0::2] + 1j * g[1::2]
        out[i] = v / np.linalg.norm(v)
    return out


def bond_profile(N, d, chi_max):
    """Largest bond dimensions an N-site MPS with site dimension d can use:
    chi_i = min(d^i, d^(N-i), chi_max) for the bond after site i."""
    out = []
    for i in range(1, N):
        c = chi_max
        if i * np.log(d) < np.log(chi_max) + 1e-12:
            c = min(c, d ** i)
        if (N - i) * np.log(d) < np.log(chi_max) + 1e-12:
            c = min(c, d ** (N - i))
        out.append(int(c))
    return out


def random_mps(N, d, chi_max, seed, decay=16.0):
    """A random MPS with full bond dimensions (``bond_profile``) whose tensors
    are complex Gaussian, with the right bond index b scaled by exp(-b/decay)
    so that its Schmidt spectra decay.  Used as a saturated-chi input state.
    Returns a list of arrays (chi_{i-1}, d, chi_i)."""
    rng = np.random.default_rng(seed)
    chis = [1] + bond_profile(N, d, chi_max) + [1]
    out = []
    for i in range(N):
        a, b = chis[i], chis[i + 1]
        g = rng.standard_normal((a, d, b, 2))
        T = (g[..., 0] + 1j * g[..., 1]) / np.sqrt(2 * a * d)
        T *= np.exp(-np.arange(b) / decay)[None, None, :]
        out.append(T)
    return out


def random_isometric_mps(N, d, chi_max, seed, kappa=64.0):
    """A random MPS at full bond dimension whose bond spectra decay slowly:
    site i is a Haar-like random isometry Q_i (QR of a complex Gaussian
    (chi_{i-1} d) x chi_i matrix) times weights exp(-b/kappa) on its right
    bond, so with kappa = 64 the weight ratio at b = 256 is e^-8 and a cutoff
    of 1e-10 does not bind before chi_max does.  Used as the saturated start
    state of the benchmark workload."""
    rng = np.random.default_rng(seed)
    chis = [1] + bond_profile(N, d, chi_max) + [1]
    out = []
    for i in range(N):
        a, b = chis[i], chis[i + 1]
        g = rng.standard_normal((a * d, b, 2))
        G = g[..., 0] + 1j * g[..., 1]
        if a * d >= b:
            Q, _ = np.linalg.qr(G)
        else:
            Q, _ = np.linalg.qr(G.conj().T)
            Q = Q.conj().T
        w = np.exp(-np.arange(b) / kappa)
        out.append((Q * (w / np.linalg.norm(w))[None, :]).reshape(a, d, b))
    return out


def flat_band_bath(n_bath, half_bandwidth=1.0, gamma=0.05):
    """Linear discretisation of a flat band of half-bandwidth D: symmetric
    midpoints eps_j = -D + D(2j-1)/N_b, equal couplings V_j = sqrt(2 D Gamma /
    (pi N_b)) (so that Gamma = pi rho_0 sum V^2 with rho_0 = 1/(2D))."""
    D = half_bandwidth
    j = np.arange(1, n_bath + 1)
    eps = -D + D * (2 * j - 1) / n_bath
    V = np.full(n_bath, np.sqrt(2 * D * gamma / (np.pi * n_bath)))
    return eps, V


WORKLOADS = {
    "heisenberg_small": dict(model="heisenberg", N=10, J=1.0, chi_max=32, cutoff=0.0,
                             tau0=1e-2, tau_max=1e2, K=20, schemes=("be",), seed=1000),
    "heisenberg_bulk": dict(model="heisenberg", N=64, J=1.0, chi_max=256, cutoff=1e-10,
                            tau0=1e-3, tau_max=1e3, K=40, schemes=("be", "tr"), seed=2000),
    "anderson_flat": dict(model="anderson", n_bath=99, U=0.3, gamma=0.05, half_bandwidth=1.0,
                          chi_max=512, cutoff=1e-14, tau0=1e-2, tau_max=1e4, K=50,
                          schemes=("tr",), seed=3000),
}


def serve_stream(n, rate=20.0, baths=(49, 99, 199), chis=(128, 256, 512, 1024), seed=5000):
    """Requests of the served impurity stream, drawn in this order from one
    seeded generator: Poisson inter-arrival gaps (mean 1/rate s), U ~ U[0.05,
    0.6], Gamma ~ U[0.02, 0.1], bath sizes from `baths`, bond caps from `chis`,
    tau_max from {1e2, 1e3, 1e4}.  Each request evolves on the geometric grid
    1e-2 -> tau_max in K = ceil(10 log10(tau_max / 1e-2)) steps from a random
    product state (seed + i), with eps_d = -U/2 and the flat-band bath.  Returns
    a list of dicts (model parameters and layout only)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    Us = rng.uniform(0.05, 0.6, n)
    Gs = rng.uniform(0.02, 0.1, n)
    nbs = rng.choice(list(baths), n)
    cxs = rng.choice(list(chis), n)
    tms = rng.choice([1e2, 1e3, 1e4], n)
    out = []
    for i in range(n):
        nb = int(nbs[i])
        eps, V = flat_band_bath(nb, gamma=float(Gs[i]))
        out.append({"gap_s": float(gaps[i]), "U": float(Us[i]), "eps_d": -0.5 * float(Us[i]),
                    "Gamma": float(Gs[i]), "n_bath": nb, "chi_max": int(cxs[i]),
                    "tau_max": float(tms[i]),
                    "n_steps": int(np.ceil(10 * np.log10(tms[i] / 1e-2))),
                    "eps": eps, "V": V,
                    "site_vecs": random_product_state(nb + 1, 4, seed + i)})
    return out
