"""Matrix product state helpers (oracle).  Test infrastructure only.

An MPS is a list of complex128 arrays A_i[a, s, b] of shape
(chi_{i-1}, d, chi_i) with chi_0 = chi_N = 1 (Method: the state is
represented as an MPS).  The dense vector has site 1 as its most significant
digit.
"""
import numpy as np


def product_state(site_vecs):
    """Product MPS from per-site vectors (shape (N, d))."""
    return [np.asarray(v, complex).reshape(1, -1, 1).copy() for v in site_vecs]


def copy(mps):
    return [A.copy() for A in mps]


def to_dense(mps):
    v = mps[0].reshape(mps[0].shape[1], mps[0].shape[2])       # (s, b)
    for A in mps[1:]:
        v = np.tensordot(v, A, axes=([1], [0]))                 # (S, s, b)
        v = v.reshape(-1, A.shape[2])
    return v[:, 0]


def overlap(bra, ket):
    """<bra|ket>."""
    E = np.ones((1, 1), complex)                                # E[a_bra, a_ket]
    for B, A in zip(bra, ket):
        T = np.tensordot(E, A, axes=([1], [0]))                 # (a, s, b')
        E = np.tensordot(B.conj(), T, axes=([0, 1], [0, 1]))    # (b, b')
    return complex(E[0, 0])


def norm(mps):
    return float(np.sqrt(overlap(mps, mps).real))


def expect_mpo(mps, Ws):
    """<psi|H|psi> / <psi|psi> by a left-to-right transfer contraction."""
    L = np.ones((1, 1, 1), complex)                             # L[a_bra, w, a_ket]
    for A, W in zip(mps, Ws):
        T = np.tensordot(L, A, axes=([2], [0]))                 # (a, w, s, b')
        T = np.tensordot(T, W, axes=([1, 2], [0, 2]))           # (a, b', s', w')
        L = np.tensordot(A.conj(), T, axes=([0, 1], [0, 2]))    # (b, b', w')
        L = L.transpose(0, 2, 1)
    return float(L[0, 0, 0].real / overlap(mps, mps).real)


def apply_local(mps, ops):
    """Apply a product of one-site operators {site: matrix} (matrices act as
    O[s', s]); returns a new MPS."""
    out = copy(mps)
    for i, O in ops.items():
        out[i] = np.einsum("ps,asb->apb", O, out[i])
    return out


def correlator(mps, O, i, P, j, string=None):
    """<psi| O_i S_{i+1} ... S_{j-1} P_j |psi> / <psi|psi> for i <= j, where S
    is the optional string operator (e.g. the Jordan-Wigner parity).  For
    i == j the operator is the product O P on that site."""
    if i > j:
        raise ValueError("need i <= j")
    if i == j:
        ops = {i: np.asarray(O) @ np.asarray(P)}
    else:
        ops = {i: np.asarray(O), j: np.asarray(P)}
        if string is not None:
            for k in range(i + 1, j):
                ops[k] = np.asarray(string)
    return overlap(mps, apply_local(mps, ops)) / overlap(mps, mps).real


def right_canonicalize(mps):
    """Bring sites 2..N to right-orthonormal form by QR, sweeping right to
    left; the norm ends up on site 1."""
    out = copy(mps)
    for i in range(len(out) - 1, 0, -1):
        A = out[i]
        chl, d, chr_ = A.shape
        M = A.reshape(chl, d * chr_)
        Q, Rm = np.linalg.qr(M.conj().T)                        # M = Rm^H Q^H
        k = Q.shape[1]
        out[i] = Q.conj().T.reshape(k, d, chr_)
        out[i - 1] = np.tensordot(out[i - 1], Rm.conj().T, axes=([2], [0]))
    return out


def bond_dims(mps):
    return [A.shape[2] for A in mps[:-1]]
