"""Two-site DMRG-style MPO-MPS linear solve with GMRES local solves (oracle).
Test infrastructure only.

The paper solves each implicit step (Eq. 4) as an MPO-MPS linear system with
a two-site DMRG-like scheme: the right-hand side MPS b is projected into the
basis of the solution MPS x, each two-site block is found by GMRES, and the
block is split again by a truncated SVD (Method; App. B).
Everything below follows those steps in that order, with the readings that
the paper leaves open fixed as follows:

* A sweep is a left-to-right pass over bonds (1,2)..(N-1,N) followed by a
  right-to-left pass (N-1,N)..(1,2): 2(N-1) local solves, starting from a
  right-canonical x with its centre on site 1 (App. B: "a single DMRG-style
  sweep").
* The local system is ((1 - c s) I + c H_eff) X = B, i.e. A = I + c (H - s)
  projected, with H_eff the two-site effective Hamiltonian.
* GMRES: one cycle of at most m Arnoldi steps (m = 10: App. D fixes one
  GMRES cycle on a ten-dimensional Krylov space per local solve; more cycles,
  each restarted from the last iterate, are an option), modified
  Gram-Schmidt with one re-orthogonalisation pass, initial guess the current
  two-site block, early exit on a happy breakdown (h_{j+1,j} <= 1e-14 |A v_j|,
  |A v_j| being the norm of Hessenberg column j) or when the relative residual
  |r|/|B| <= local_tol.  The small least-squares problem is solved with LAPACK.
* Truncation: keep r = min(chi_max, smallest r >= 1 whose discarded squared
  weight sum_{k>r} s_k^2 <= max(cutoff, 1e-24) * sum_k s_k^2) (the Heisenberg
  section bounds the sum of the squared Schmidt values dropped at each bond);
  then, if
  s_{r+1} >= s_r (1 - 1e-10), lower r to just before that near-degenerate
  group, unless that would leave r = 0 (then r is left as it was).
"""
import numpy as np

from . import mps as mpsmod

TIE_REL = 1e-10
WEIGHT_FLOOR = 1e-24
BREAKDOWN_REL = 1e-14


# ------------------------------------------------------------- environments
# Left environments L[a_bra, w, a_ket] hold the block of sites left of a bond;
# right environments R[b_bra, w, b_ket] the block right of it.  Overlap
# environments drop the MPO index.

def left_env_update(L, bra, W, ket):
    """L'[b, w', b'] = sum conj(bra[a,s',b]) L[a,w,a'] W[w,s',s,w'] ket[a',s,b']."""
    T = np.tensordot(L, ket, axes=([2], [0]))                  # (a, w, s, b')
    T = np.tensordot(T, W, axes=([1, 2], [0, 2]))              # (a, b', s', w')
    T = np.tensordot(bra.conj(), T, axes=([0, 1], [0, 2]))     # (b, b', w')
    return T.transpose(0, 2, 1)


def right_env_update(R, bra, W, ket):
    """R'[a, w, a'] = sum conj(bra[a,s',b]) W[w,s',s,w'] ket[a',s,b'] R[b,w',b']."""
    T = np.tensordot(ket, R, axes=([2], [2]))                  # (a', s, b, w')
    T = np.tensordot(T, W, axes=([1, 3], [2, 3]))              # (a', b, w, s')
    T = np.tensordot(bra.conj(), T, axes=([1, 2], [3, 1]))     # (a, a', w)
    return T.transpose(0, 2, 1)


def left_overlap_update(L, bra, ket):
    """L'[b, b'] = sum conj(bra[a,s,b]) L[a,a'] ket[a',s,b']."""
    T = np.tensordot(L, ket, axes=([1], [0]))                  # (a, s, b')
    return np.tensordot(bra.conj(), T, axes=([0, 1], [0, 1]))


def right_overlap_update(R, bra, ket):
    """R'[a, a'] = sum conj(bra[a,s,b]) ket[a',s,b'] R[b,b']."""
    T = np.tensordot(ket, R, axes=([2], [1]))                  # (a', s, b)
    return np.tensordot(bra.conj(), T, axes=([1, 2], [1, 2]))


# ------------------------------------------------------------- local problem
def heff_apply(L, W1, W2, R, X):
    """Two-site effective Hamiltonian on X[a', s, t, b']:
    Y[a,s',t',b] = sum L[a,w,a'] W1[w,s',s,v] W2[v,t',t,w'] R[b,w',b'] X[a',s,t,b']."""
    T = np.tensordot(L, X, axes=([2], [0]))                    # (a, w, s, t, b')
    T = np.tensordot(T, W1, axes=([1, 2], [0, 2]))             # (a, t, b', s', v)
    T = np.tensordot(T, W2, axes=([4, 1], [0, 2]))             # (a, b', s', t', w')
    return np.tensordot(T, R, axes=([1, 4], [2, 1]))           # (a, s', t', b)


def heff_entry(L, W1, W2, R, X, a, b):
    """Y[a, :, :, b] of ``heff_apply`` for one pair (a, b), from the same sum
    restricted to that output row/column (for sampled checks at sizes where
    the whole contraction is too slow)."""
    T = np.tensordot(L[a], X, axes=([1], [0]))                 # (w, s, t, b')
    T = np.tensordot(T, W1, axes=([0, 1], [0, 2]))             # (t, b', s', v)
    T = np.tensordot(T, W2, axes=([3, 0], [0, 2]))             # (b', s', t', w')
    return np.tensordot(T, R[b], axes=([0, 3], [1, 0]))        # (s', t')


def project_two_site(Lo, A1, A2, Ro):
    """B[a,s,t,b] = sum Lo[a,a'] A1[a',s,c] A2[c,t,b'] Ro[b,b']: the two-site
    block of the MPS (A1, A2) seen in the bra basis of the environments."""
    T = np.tensordot(Lo, A1, axes=([1], [0]))                  # (a, s, c)
    T = np.tensordot(T, A2, axes=([2], [0]))                   # (a, s, t, b')
    return np.tensordot(T, Ro, axes=([3], [1]))                # (a, s, t, b)


def gmres(matvec, B, X0, m, local_tol=0.0):
    """One GMRES cycle (Saad & Schultz) of at most m Arnoldi steps.
    Returns (X, info) with info = (steps, relative residual estimate)."""
    r = B - matvec(X0)
    beta = np.linalg.norm(r)
    bnorm = np.linalg.norm(B)
    if beta == 0.0:
        return X0.copy(), (0, 0.0)
    V = [r / beta]
    H = np.zeros((m + 1, m), complex)
    k = 0
    res = beta
    for j in range(m):
        w = matvec(V[j])
        for _ in range(2):                                     # MGS + one re-orthogonalisation
            for i in range(j + 1):
                h = np.vdot(V[i], w)
                H[i, j] += h
                w = w - h * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        k = j + 1
        e1 = np.zeros(k + 1, complex)
        e1[0] = beta
        y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
        res = np.linalg.norm(e1 - H[:k + 1, :k] @ y)
        # happy breakdown: the new direction is negligible against A v_j,
        # whose norm is that of Hessenberg column j (Arnoldi relation)
        if H[j + 1, j].real <= BREAKDOWN_REL * np.linalg.norm(H[:j + 2, j]):
            break
        if local_tol > 0.0 and res <= local_tol * bnorm:
            break
        V.append(w / H[j + 1, j])
    X = X0.copy()
    for i in range(k):
        X = X + y[i] * V[i]
    return X, (k, res / bnorm if bnorm > 0 else 0.0)


def gmres_restarted(matvec, B, X0, m, cycles=1, local_tol=0.0):
    """Up to `cycles` GMRES(m) cycles, each restarted from the last iterate;
    a cycle that ends before m steps (breakdown, or the relative residual at
    local_tol) ends the solve.  Returns (X, (total steps, last residual))."""
    X, steps, res = X0, 0, 0.0
    for _ in range(max(1, cycles)):
        X, (k, res) = gmres(matvec, B, X, m, local_tol)
        steps += k
        if k < m or (local_tol > 0.0 and res <= local_tol):
            break
    return X, (steps, res)


def choose_rank(S, chi_max, cutoff):
    """Kept rank for descending singular values S (see module docstring)."""
    n = len(S)
    w = S.astype(float) ** 2
    tail = np.concatenate([np.cumsum(w[::-1])[::-1], [0.0]])  # tail[r] = sum_{k>=r} w_k
    total = tail[0]
    if total == 0.0:
        return 1, 0.0
    tol = max(cutoff, WEIGHT_FLOOR) * total
    r = n
    for cand in range(1, n + 1):
        if tail[cand] <= tol:
            r = cand
            break
    r = min(r, chi_max)
    if r < n and S[r] >= S[r - 1] * (1.0 - TIE_REL):
        g = r - 1
        while g > 0 and S[g] >= S[g - 1] * (1.0 - TIE_REL):
            g -= 1
        if g >= 1:
            r = g
    return r, float(tail[r] / total)


def split_two_site(X, chi_max, cutoff, centre_right):
    """Truncated SVD of X[a,s,t,b] as (a s) x (t b).  centre_right=True gives
    (U, S V^dag) (left-to-right move), False gives (U S, V^dag)."""
    chl, d1, d2, chr_ = X.shape
    U, S, Vh = np.linalg.svd(X.reshape(chl * d1, d2 * chr_), full_matrices=False)
    r, disc = choose_rank(S, chi_max, cutoff)
    U, S, Vh = U[:, :r], S[:r], Vh[:r]
    if centre_right:
        A1, A2 = U, S[:, None] * Vh
    else:
        A1, A2 = U * S[None, :], Vh
    return A1.reshape(chl, d1, r), A2.reshape(r, d2, chr_), disc, S


def right_canonicalize_svd(mps_in):
    """Gauge move before a sweep: from the last site to the second, split
    A_i = (U S) V^dag by an SVD that keeps every singular value above the
    weight floor, keep V^dag on site i and absorb U S into site i-1.  Dropping
    only numerically zero singular values makes the bond spaces (and hence
    the projected local problems) independent of the decomposition used."""
    out = mpsmod.copy(mps_in)
    for i in range(len(out) - 1, 0, -1):
        chl, d, chr_ = out[i].shape
        U, S, Vh = np.linalg.svd(out[i].reshape(chl, d * chr_), full_matrices=False)
        r, _ = choose_rank(S, len(S), 0.0)
        out[i] = Vh[:r].reshape(r, d, chr_)
        out[i - 1] = np.tensordot(out[i - 1], U[:, :r] * S[None, :r], axes=([2], [0]))
    return out


# ------------------------------------------------------------- sweeps
class SweepInfo:
    def __init__(self):
        self.max_discarded = 0.0
        self.max_local_residual = 0.0
        self.gmres_steps = 0
        self.max_chi = 0


def _build_right_envs(Ws, x, others):
    """Right environments of x for every site.  `others` lists
    (kind, ket_mps) pairs: kind 'op' uses the MPO, 'ov' is an overlap; a ket
    of None means x itself."""
    N = len(x)
    envs = []
    for kind, ket in others:
        E = [None] * N
        E[N - 1] = np.ones((1, 1, 1) if kind == "op" else (1, 1), complex)
        for i in range(N - 2, -1, -1):
            if kind == "op":
                E[i] = right_env_update(E[i + 1], x[i + 1], Ws[i + 1], ket[i + 1])
            else:
                E[i] = right_overlap_update(E[i + 1], x[i + 1], ket[i + 1])
        envs.append(E)
    return envs


def _sweep(Ws, x, local_block, others, chi_max, cutoff, info):
    """Generic two-site sweep.  `others` = [(kind, ket_mps)] of environments to
    keep; local_block(i, envsL, envsR, X0) returns the new two-site block."""
    N = len(x)
    others = [(kind, x if ket is None else ket) for kind, ket in others]
    Rs = _build_right_envs(Ws, x, others)
    Ls = []
    for kind, _ in others:
        E = [None] * N
        E[0] = np.ones((1, 1, 1) if kind == "op" else (1, 1), complex)
        Ls.append(E)
    order = [(i, True) for i in range(N - 1)] + [(i, False) for i in range(N - 2, -1, -1)]
    for i, lr in order:
        X0 = np.tensordot(x[i], x[i + 1], axes=([2], [0]))
        X = local_block(i, [E[i] for E in Ls], [E[i + 1] for E in Rs], X0)
        x[i], x[i + 1], disc, S = split_two_site(X, chi_max, cutoff, centre_right=lr)
        info.max_discarded = max(info.max_discarded, disc)
        for (kind, ket), EL, ER in zip(others, Ls, Rs):
            if lr:
                EL[i + 1] = (left_env_update(EL[i], x[i], Ws[i], ket[i]) if kind == "op"
                             else left_overlap_update(EL[i], x[i], ket[i]))
            else:
                ER[i] = (right_env_update(ER[i + 1], x[i + 1], Ws[i + 1], ket[i + 1])
                         if kind == "op" else right_overlap_update(ER[i + 1], x[i + 1], ket[i + 1]))
    info.max_chi = max(mpsmod.bond_dims(x) + [1])
    return x


def linsolve(Ws, x0, b, c, s, chi_max, cutoff, krylov_dim=10, local_tol=0.0,
             sweeps=1, sweep_tol=0.0, max_cycles=1):
    """Solve (I + c (H - s)) x = b for MPS x, starting from x0 (App. B).
    Returns (x, info); x has its orthogonality centre on site 1."""
    x = right_canonicalize_svd(x0)
    info = SweepInfo()
    alpha = 1.0 - c * s

    def local_block(i, EL, ER, X0):
        Lop, Lov = EL
        Rop, Rov = ER
        B = project_two_site(Lov, b[i], b[i + 1], Rov)

        def matvec(V):
            return alpha * V + c * heff_apply(Lop, Ws[i], Ws[i + 1], Rop, V)

        X, (steps, res) = gmres_restarted(matvec, B, X0, krylov_dim, max_cycles, local_tol)
        info.gmres_steps += steps
        info.max_local_residual = max(info.max_local_residual, res)
        return X

    prev = None
    for sw in range(max(1, sweeps)):
        x = _sweep(Ws, x, local_block, [("op", None), ("ov", b)], chi_max, cutoff, info)
        if sweep_tol > 0.0 and prev is not None:
            ov = abs(mpsmod.overlap(prev, x)) / (mpsmod.norm(prev) * mpsmod.norm(x))
            if 1.0 - ov < sweep_tol:
                break
        prev = mpsmod.copy(x)
    return x, info


def fit_affine(Ws, psi, alpha, beta, chi_max, cutoff, sweeps=1):
    """Two-site variational fit f ~ alpha |psi> + beta H |psi>, starting from
    f = psi.  Used to form the trapezoid right-hand side b = (I - c (H - s)) psi
    of Eq. 4 (Method, operation (i)); App. B notes b is also the initial guess
    of the solve.  Each local block is the exact projection of the target onto
    the current environments of f."""
    f = right_canonicalize_svd(psi)
    info = SweepInfo()

    def local_block(i, EL, ER, X0):
        Lop, Lov = EL
        Rop, Rov = ER
        theta = np.tensordot(psi[i], psi[i + 1], axes=([2], [0]))
        return (alpha * project_two_site(Lov, psi[i], psi[i + 1], Rov)
                + beta * heff_apply(Lop, Ws[i], Ws[i + 1], Rop, theta))

    for _ in range(max(1, sweeps)):
        f = _sweep(Ws, f, local_block, [("op", psi), ("ov", psi)], chi_max, cutoff, info)
    return f, info


def fit_combination(targets, coefs, chi_max, cutoff, sweeps=1):
    """Two-site variational fit f ~ sum_t coefs[t] |targets[t]>, starting from
    f = targets[0] (right-canonicalised).  Each local block is the exact
    projection of the combination onto the current environments of f: the
    sum of the targets' two-site blocks, each contracted with its own overlap
    environments.  Forms the Gauss-Legendre step from its partial-fraction
    solves."""
    f = right_canonicalize_svd(targets[0])
    info = SweepInfo()

    def local_block(i, EL, ER, X0):
        out = 0.0
        for c, t, Lov, Rov in zip(coefs, targets, EL, ER):
            out = out + c * project_two_site(Lov, t[i], t[i + 1], Rov)
        return out

    for _ in range(max(1, sweeps)):
        f = _sweep(None, f, local_block, [("ov", t) for t in targets], chi_max, cutoff, info)
    return f, info
