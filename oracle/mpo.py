"""Matrix product operators (oracle).  Test infrastructure only.

Site tensors W_i[w, s', s, w'] have shape (D_{i-1}, d, d, D_i) with
D_0 = D_N = 1; s' is the output (bra) index and s the input (ket) index.
Channel 0 is "nothing placed yet" and channel D-1 is "all placed": the first
site keeps row 0 and the last site keeps column D-1 of the bulk tensor.  The
operator is the product W_1 W_2 ... W_N over the channel indices.

The paper builds its MPOs with ITensor's OpSum (App. B); these are the
equivalent hand-written finite-state machines, checked against the dense
Hamiltonians of ``oracle.ed`` in the tests.
"""
import numpy as np

# spin-1/2, local index 0 = up, 1 = down
SP = np.array([[0.0, 1.0], [0.0, 0.0]])
SM = SP.T.copy()
SZ = np.diag([0.5, -0.5])
I2 = np.eye(2)

# spinful fermion site, local index n_up + 2 n_down:
# 0 = |0>, 1 = |up>, 2 = |down>, 3 = |up down>, with up ordered before down.
C_UP = np.zeros((4, 4)); C_UP[0, 1] = 1.0; C_UP[2, 3] = 1.0
C_DN = np.zeros((4, 4)); C_DN[0, 2] = 1.0; C_DN[1, 3] = -1.0   # carries (-1)^{n_up}
N_UP = np.diag([0.0, 1.0, 0.0, 1.0])
N_DN = np.diag([0.0, 0.0, 1.0, 1.0])
F_PAR = np.diag([1.0, -1.0, -1.0, 1.0])                         # (-1)^{n_up + n_down}
I4 = np.eye(4)


def _boundary(Wbulk, i, N):
    if N == 1:
        return Wbulk[:1, :, :, -1:]
    if i == 0:
        return Wbulk[:1]
    if i == N - 1:
        return Wbulk[..., -1:]
    return Wbulk


def heisenberg_mpo(N, J=1.0, Jz=None):
    """Heisenberg chain J sum (SxSx + SySy) + Jz sum SzSz as a D=5 MPO
    (Heisenberg-chain section)."""
    Jz = J if Jz is None else Jz
    W = np.zeros((5, 2, 2, 5), dtype=complex)
    W[0, :, :, 0] = I2
    W[0, :, :, 1] = SP
    W[0, :, :, 2] = SM
    W[0, :, :, 3] = SZ
    W[1, :, :, 4] = 0.5 * J * SM
    W[2, :, :, 4] = 0.5 * J * SP
    W[3, :, :, 4] = Jz * SZ
    W[4, :, :, 4] = I2
    return [_boundary(W, i, N).copy() for i in range(N)]


def anderson_mpo(eps_d, U, eps, V):
    """Single-impurity Anderson model in star geometry (Anderson-impurity
    section), impurity at site 0, bath j at site j, Jordan-Wigner strings
    F = (-1)^{n_up + n_down} on the sites between impurity and bath site.
    Channels: 0 start, 1 d^dag_up F, 2 d^dag_down F, 3 F d_up, 4 F d_down,
    5 done (D = 6)."""
    eps = np.asarray(eps, float)
    V = np.asarray(V, float)
    N = 1 + len(eps)
    Ws = []
    for i in range(N):
        W = np.zeros((6, 4, 4, 6), dtype=complex)
        if i == 0:
            W[0, :, :, 0] = I4
            W[0, :, :, 1] = C_UP.T @ F_PAR
            W[0, :, :, 2] = C_DN.T @ F_PAR
            W[0, :, :, 3] = F_PAR @ C_UP
            W[0, :, :, 4] = F_PAR @ C_DN
            W[0, :, :, 5] = eps_d * (N_UP + N_DN) + U * (N_UP @ N_DN)
        else:
            e, v = eps[i - 1], V[i - 1]
            W[0, :, :, 0] = I4
            W[0, :, :, 5] = e * (N_UP + N_DN)
            for ch in range(1, 5):
                W[ch, :, :, ch] = F_PAR
            W[1, :, :, 5] = v * C_UP
            W[2, :, :, 5] = v * C_DN
            W[3, :, :, 5] = v * C_UP.T
            W[4, :, :, 5] = v * C_DN.T
            W[5, :, :, 5] = I4
        Ws.append(_boundary(W, i, N).copy())
    return Ws


def mpo_to_dense(Ws):
    """Contract an MPO into its dense matrix (site 1 most significant)."""
    M = Ws[0][0]                                  # (d, d, D)
    for W in Ws[1:]:
        # M[S', S, w] W[w, s', s, w'] -> M[(S' s'), (S s), w']
        T = np.tensordot(M, W, axes=([2], [0]))   # (S', S, s', s, w')
        ro, co = T.shape[0], T.shape[1]
        T = T.transpose(0, 2, 1, 3, 4)
        M = T.reshape(ro * T.shape[1], co * T.shape[3], T.shape[4])
    return M[:, :, 0]
