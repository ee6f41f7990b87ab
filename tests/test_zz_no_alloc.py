"""The allocation-free H_eff entry point (ite_k_heff_noalloc) against the
oracle's two-site matvec.

Callers that cannot allocate device memory when they need a matvec (a
latency-critical loop that must not let cudaMalloc synchronise the device, or
a process whose device memory is all owned by another pool) use the variant
whose scratch is a fixed array inside the library.  It always computes on the
FP64 pipe, whatever kernel precision the context carries, so its output is
held to the FP64 bar against the oracle in both precision settings.  This file
is collected last so that a run stopping at its first failure has run every
other test."""
import ctypes as C

import numpy as np
import pytest

from oracle import linsolve as ls, mpo as ompo
from paper_2606_02930_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_noalloc_heff_matches_oracle(precision):
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2606_02930_gb300 import _lib, api
    from tests.gpu_util import L_to_lib, R_to_lib, crandn, rel_err, to_dev, to_host

    lib = _lib.lib
    ctx = api.ctx_create(0)
    api.set_kernel_precision(ctx, precision)
    eps, V = inputs.flat_band_bath(5)
    cases = [("heisenberg", ompo.heisenberg_mpo(12), (64, 64, 64, 64)),
             ("anderson", ompo.anderson_mpo(-0.15, 0.3, eps, V), (20, 24, 28, 16))]
    one = np.array([1.0, 0.0])
    for name, Ws, (chlB, chlK, chrK, chrB) in cases:
        H = api.mpo_create(ctx, Ws)
        i = 2
        D0, D2, d = Ws[i].shape[0], Ws[i + 1].shape[3], Ws[i].shape[1]
        rng = np.random.default_rng(len(name))
        for call in range(2):      # two calls in a row share the static scratch
            Lo, Ro = crandn(rng, chlB, D0, chlK), crandn(rng, chrB, D2, chrK)
            Xo, Zo = crandn(rng, chlK, d, d, chrK), crandn(rng, chlB, d, d, chrB)
            alpha, gamma = 0.3 - 0.2j, 1.5
            want = alpha * ls.heff_apply(Lo, Ws[i], Ws[i + 1], Ro, Xo) + gamma * Zo
            L, R, X, Z = to_dev(L_to_lib(Lo)), to_dev(R_to_lib(Ro)), to_dev(Xo), to_dev(Zo)
            Y = torch.full((chlB, d, d, chrB), float("nan"), dtype=torch.complex128, device="cuda")
            a = np.array([alpha.real, alpha.imag])
            g = np.array([gamma, 0.0])
            held = lib.ite_ctx_device_bytes(ctx.h)
            torch.cuda.synchronize()
            before = torch.cuda.memory_allocated()
            _lib.check(lib.ite_k_heff_noalloc(
                ctx.h, H.h, i, chlB, chlK, chrK, chrB, C.c_void_p(L.data_ptr()),
                C.c_void_p(R.data_ptr()), C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                a.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(Z.data_ptr()),
                g.ctypes.data_as(C.POINTER(C.c_double))), ctx.h)
            torch.cuda.synchronize()
            assert lib.ite_ctx_device_bytes(ctx.h) == held
            assert torch.cuda.memory_allocated() == before
            assert rel_err(to_host(Y), want) < 1e-12, (name, call)
            assert torch.cuda.current_device() == 0
    # sizes beyond the static scratch are rejected with a message, nothing runs
    H = api.mpo_create(ctx, ompo.heisenberg_mpo(20))
    big = torch.zeros(1, dtype=torch.complex128, device="cuda")
    p = C.c_void_p(big.data_ptr())
    st = lib.ite_k_heff_noalloc(ctx.h, H.h, 5, 256, 256, 256, 256, p, p, p, p,
                                one.ctypes.data_as(C.POINTER(C.c_double)), None, None)
    assert st == _lib.ITE_EINVAL
    assert b"static scratch" in lib.ite_last_error(ctx.h)
