"""Helpers shared by the GPU parity tests: layout conversions between the
oracle's arrays and the library's device layouts, and random local problems.
These helpers only move data; they hold none of the method's arithmetic."""
import numpy as np


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to("cuda")


def to_host(t):
    return t.detach().cpu().numpy()


# oracle L[a_bra, w, a_ket]  <->  library L[w][a_bra][a_ket]
def L_to_lib(L):
    return np.ascontiguousarray(L.transpose(1, 0, 2))


def L_from_lib(Ld):
    return np.ascontiguousarray(Ld.transpose(1, 0, 2))


# oracle R[b_bra, w, b_ket]  <->  library R[w][b_ket][b_bra]
def R_to_lib(R):
    return np.ascontiguousarray(R.transpose(1, 2, 0))


def R_from_lib(Rd):
    return np.ascontiguousarray(Rd.transpose(2, 0, 1))


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
