"""Python binding of the library: thin wrappers with the names of the C calls
(ctx_create, mpo_create, mps_create, implicit_step, evolve_loggrid,
evolve_panels, energy, overlap, correlator, and the kernel-level k_* calls).

Argument marshalling only.  PyTorch supplies the CUDA stream and, by default,
device memory (through the caching allocator); every computation runs in
libite.so.  Host arrays are numpy complex128, device arrays torch complex128
CUDA tensors.
"""
import ctypes as C

import numpy as np

from . import _lib as L
from ._lib import lib, check

BACKWARD_EULER, TRAPEZOID = L.ITE_BACKWARD_EULER, L.ITE_TRAPEZOID
SHIFT_FIXED, SHIFT_CURRENT_ENERGY = L.ITE_SHIFT_FIXED, L.ITE_SHIFT_CURRENT_ENERGY
GAUSS_LEGENDRE_2, GAUSS_LEGENDRE_3 = L.ITE_GAUSS_LEGENDRE_2, L.ITE_GAUSS_LEGENDRE_3
FORWARD_EULER, HEUN = L.ITE_FORWARD_EULER, L.ITE_HEUN
SCHEMES = {"be": BACKWARD_EULER, "tr": TRAPEZOID, "gl2": GAUSS_LEGENDRE_2,
           "gl3": GAUSS_LEGENDRE_3, "fe": FORWARD_EULER, "heun": HEUN}


def _scheme(s):
    return SCHEMES[s] if isinstance(s, str) else int(s)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


PRECISIONS = {"fp64": L.ITE_FP64, "fp64_tc": L.ITE_FP64_TC, "mixed_bf16": L.ITE_MIXED_BF16,
              "mixed_tf32": L.ITE_MIXED_TF32}


def solver_opts(krylov_dim=10, sweeps=1, local_tol=0.0, sweep_tol=0.0, fit_sweeps=1,
                precision="fp64", max_cycles=1, refine_max=None, refine_tol=None):
    o = L.ite_solver_opts()
    lib.ite_solver_opts_default(C.byref(o))
    o.krylov_dim, o.sweeps, o.local_tol = krylov_dim, sweeps, local_tol
    o.max_cycles = max_cycles
    if refine_max is not None:
        o.refine_max = refine_max
    if refine_tol is not None:
        o.refine_tol = refine_tol
    o.sweep_tol, o.fit_sweeps = sweep_tol, fit_sweeps
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return o


class Context:
    """One device and one stream (torch's current stream by default)."""

    def __init__(self, device=0, stream=None, torch_allocator=True):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self._keep = []
        alloc_cb = L.ite_alloc_fn()
        free_cb = L.ite_free_fn()
        if torch_allocator:
            dev, st = device, stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except RuntimeError:
                    return None

            def _free(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)

            alloc_cb, free_cb = L.ite_alloc_fn(_alloc), L.ite_free_fn(_free)
            self._keep += [alloc_cb, free_cb]
        h = C.c_void_p()
        check(lib.ite_ctx_create(device, C.c_void_p(stream), alloc_cb, free_cb, None, C.byref(h)))
        self.h = h

    def error(self):
        return lib.ite_last_error(self.h).decode()

    def device_bytes(self):
        return lib.ite_ctx_device_bytes(self.h)

    def close(self):
        if self.h:
            lib.ite_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ctx_create(device=0, stream=None, torch_allocator=True):
    return Context(device, stream, torch_allocator)


class MPO:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h
        self.N = lib.ite_mpo_length(h)

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib.ite_mpo_destroy(self.h)
        except Exception:
            pass


def mpo_create(ctx, Ws):
    """MPO from site tensors W_i[w, s', s, w'] (numpy arrays)."""
    N = len(Ws)
    d = np.array([W.shape[1] for W in Ws], np.int32)
    D = np.array([Ws[0].shape[0]] + [W.shape[3] for W in Ws], np.int32)
    flat = np.concatenate([_c128(W).ravel() for W in Ws]).view(np.float64)
    h = C.c_void_p()
    check(lib.ite_mpo_create(ctx.h, N, d.ctypes.data_as(C.POINTER(C.c_int)),
                             D.ctypes.data_as(C.POINTER(C.c_int)), _dptr(flat), C.byref(h)), ctx.h)
    return MPO(ctx, h)


def mpo_create_heisenberg(ctx, N, J=1.0, Jz=None):
    h = C.c_void_p()
    check(lib.ite_mpo_create_heisenberg(ctx.h, N, J, J if Jz is None else Jz, C.byref(h)), ctx.h)
    return MPO(ctx, h)


def mpo_create_anderson(ctx, eps, V, U, eps_d):
    eps = np.ascontiguousarray(eps, np.float64)
    V = np.ascontiguousarray(V, np.float64)
    h = C.c_void_p()
    check(lib.ite_mpo_create_anderson(ctx.h, len(eps), _dptr(eps), _dptr(V), U, eps_d,
                                      C.byref(h)), ctx.h)
    return MPO(ctx, h)


class MPS:
    def __init__(self, ctx, h, N, d):
        self.ctx, self.h, self.N, self.d = ctx, h, N, d

    def save(self):
        """Checkpoint (ite_mps_save) as bytes."""
        n = C.c_size_t()
        check(lib.ite_mps_bytes(self.h, C.byref(n)), self.ctx.h)
        buf = C.create_string_buffer(n.value)
        check(lib.ite_mps_save(self.h, buf, n.value), self.ctx.h)
        return buf.raw

    def to_dense(self):
        """The state as a dense vector (ite_mps_to_dense; d^N <= 2^24)."""
        out = np.zeros(2 * self.d ** self.N)
        check(lib.ite_mps_to_dense(self.ctx.h, self.h, _dptr(out), out.size), self.ctx.h)
        return out.view(np.complex128)

    def bond_dims(self):
        chi = np.zeros(self.N + 1, np.int32)
        n = C.c_size_t()
        check(lib.ite_mps_bond_dims(self.h, chi.ctypes.data_as(C.POINTER(C.c_int)), C.byref(n)))
        return chi, n.value

    def tensors(self):
        """Site tensors as numpy complex128 arrays (chi_i, d, chi_{i+1})."""
        chi, n = self.bond_dims()
        buf = np.empty(n, np.float64)
        check(lib.ite_mps_get(self.ctx.h, self.h, _dptr(buf), n), self.ctx.h)
        z = buf.view(np.complex128)
        out, pos = [], 0
        for i in range(self.N):
            cnt = chi[i] * self.d * chi[i + 1]
            out.append(z[pos:pos + cnt].reshape(chi[i], self.d, chi[i + 1]).copy())
            pos += cnt
        return out

    def set(self, tensors):
        chi = np.array([1] + [T.shape[2] for T in tensors], np.int32)
        flat = np.concatenate([_c128(T).ravel() for T in tensors]).view(np.float64)
        check(lib.ite_mps_set(self.ctx.h, self.h, chi.ctypes.data_as(C.POINTER(C.c_int)),
                              _dptr(flat)), self.ctx.h)

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib.ite_mps_destroy(self.h)
        except Exception:
            pass


def mps_create(ctx, tensors, chi_cap):
    N, d = len(tensors), tensors[0].shape[1]
    chi = np.array([1] + [T.shape[2] for T in tensors], np.int32)
    flat = np.concatenate([_c128(T).ravel() for T in tensors]).view(np.float64)
    h = C.c_void_p()
    check(lib.ite_mps_create(ctx.h, N, d, chi.ctypes.data_as(C.POINTER(C.c_int)), _dptr(flat),
                             chi_cap, C.byref(h)), ctx.h)
    return MPS(ctx, h, N, d)


def checkpoint_info(data):
    """(N, d, chi_cap, bond dimensions, doubles of the tensors) of a
    checkpoint, read on the host (ite_mps_checkpoint_info)."""
    N, d, cap, nd = C.c_int(), C.c_int(), C.c_int(), C.c_size_t()
    check(lib.ite_mps_checkpoint_info(data, len(data), C.byref(N), C.byref(d), C.byref(cap), None,
                                      0, C.byref(nd)))
    chi = np.zeros(N.value + 1, np.int32)
    check(lib.ite_mps_checkpoint_info(data, len(data), None, None, None,
                                      chi.ctypes.data_as(C.POINTER(C.c_int)), chi.size, None))
    return N.value, d.value, cap.value, chi, nd.value


def mps_load(ctx, data):
    """A new MPS from a checkpoint made by MPS.save (ite_mps_load)."""
    N, d = checkpoint_info(data)[:2]
    h = C.c_void_p()
    check(lib.ite_mps_load(ctx.h, data, len(data), C.byref(h)), ctx.h)
    return MPS(ctx, h, N, d)


def mps_create_product(ctx, site_vecs, chi_cap):
    v = _c128(site_vecs)
    N, d = v.shape
    h = C.c_void_p()
    check(lib.ite_mps_create_product(ctx.h, N, d, _dptr(v.view(np.float64)), chi_cap,
                                     C.byref(h)), ctx.h)
    return MPS(ctx, h, N, d)


def mps_copy(ctx, src, dst):
    check(lib.ite_mps_copy(ctx.h, src.h, dst.h), ctx.h)


def implicit_step(ctx, H, psi, dtau, scheme, shift, chi_max, cutoff, opts=None):
    info = L.ite_step_info()
    o = opts if opts is not None else solver_opts()
    check(lib.ite_implicit_step(ctx.h, H.h, psi.h, dtau, _scheme(scheme), shift, chi_max, cutoff,
                                C.byref(o), C.byref(info)), ctx.h)
    return info.as_dict()


def _evolve(fn, ctx, H, psi, grid_args, n_steps, scheme, shift_mode, shift0, chi_max, cutoff,
            opts):
    infos = (L.ite_step_info * n_steps)()
    nodes = np.zeros(n_steps + 1)
    o = opts if opts is not None else solver_opts()
    st = fn(ctx.h, H.h, psi.h, *grid_args, _scheme(scheme), shift_mode, shift0, chi_max, cutoff,
            C.byref(o), infos, _dptr(nodes))
    check(st, ctx.h)
    return nodes, [i.as_dict() for i in infos]


def evolve_loggrid(ctx, H, psi, tau0, tau_max, n_steps, scheme, chi_max, cutoff,
                   shift_mode=SHIFT_FIXED, shift0=0.0, opts=None):
    return _evolve(lib.ite_evolve_loggrid, ctx, H, psi, (tau0, tau_max, n_steps), n_steps, scheme,
                   shift_mode, shift0, chi_max, cutoff, opts)


def evolve_panels(ctx, H, psi, tau_max, P, n, scheme, chi_max, cutoff, shift_mode=SHIFT_FIXED,
                  shift0=0.0, opts=None):
    return _evolve(lib.ite_evolve_panels, ctx, H, psi, (tau_max, P, n), P * n, scheme, shift_mode,
                   shift0, chi_max, cutoff, opts)


def mps_sample(ctx, psi, u, basis=None):
    """METTS collapse of psi with the uniforms u (N numbers in [0, 1)) in the
    given d x d basis (None: computational).  Returns (config, probability)."""
    u = np.ascontiguousarray(u, np.float64)
    cfg = np.zeros(psi.N, np.int32)
    p = C.c_double()
    b = None if basis is None else _c128(basis)
    check(lib.ite_mps_sample(ctx.h, psi.h, _dptr(u), None if b is None else _dptr(b.view(np.float64)),
                             cfg.ctypes.data_as(C.POINTER(C.c_int)), C.byref(p)), ctx.h)
    return cfg.tolist(), p.value


def metts(ctx, H, config0, nodes, chi_max, cutoff, uniforms, scheme="tr", opts=None,
          alt_basis=None, obs=None, obs_site=0, shift_mode=SHIFT_CURRENT_ENERGY, shift0=0.0):
    """METTS chain (ite_metts) over the tau grid `nodes` (0 -> beta/2);
    uniforms (n_samples, N).  The defaults are the paper's: trapezoid rule,
    shift = the current energy.  Returns (energies, observable values or None,
    configurations (n_samples, N))."""
    g = np.ascontiguousarray(nodes, np.float64)
    u = np.ascontiguousarray(uniforms, np.float64)
    n, N = u.shape
    c0 = np.ascontiguousarray(config0, np.int32)
    e = np.zeros(n)
    vals = np.zeros(n)
    cfgs = np.zeros((n, N), np.int32)
    o = opts if opts is not None else solver_opts()
    ab = None if alt_basis is None else _c128(alt_basis)
    ob = None if obs is None else _c128(obs)
    check(lib.ite_metts(ctx.h, H.h, c0.ctypes.data_as(C.POINTER(C.c_int)), _dptr(g), len(g) - 1,
                        _scheme(scheme), shift_mode, shift0, chi_max, cutoff, C.byref(o),
                        None if ab is None else _dptr(ab.view(np.float64)),
                        None if ob is None else _dptr(ob.view(np.float64)), obs_site, n, _dptr(u),
                        _dptr(e), _dptr(vals), cfgs.ctypes.data_as(C.POINTER(C.c_int))), ctx.h)
    return e, (vals if obs is not None else None), cfgs


def gl_partial_fractions(q):
    """(poles z_j, residues a_j, r_inf) of the q-stage Gauss-Legendre step."""
    z = np.zeros(2 * q)
    a = np.zeros(2 * q)
    r = C.c_double()
    check(lib.ite_gl_partial_fractions(q, _dptr(z), _dptr(a), C.byref(r)))
    return z.view(np.complex128), a.view(np.complex128), r.value


def grid_geometric(tau0, tau_max, n_steps):
    out = np.zeros(n_steps + 1)
    check(lib.ite_grid_geometric(tau0, tau_max, n_steps, _dptr(out)))
    return out


def grid_panels(tau_max, P, n):
    out = np.zeros(P * n + 1)
    check(lib.ite_grid_panels(tau_max, P, n, _dptr(out)))
    return out


def energy(ctx, H, psi):
    e = C.c_double()
    check(lib.ite_energy(ctx.h, H.h, psi.h, C.byref(e)), ctx.h)
    return e.value


def overlap(ctx, bra, ket):
    out = np.zeros(2)
    check(lib.ite_overlap(ctx.h, bra.h, ket.h, _dptr(out)), ctx.h)
    return complex(out[0], out[1])


def correlator(ctx, psi, O, i, P, j, string_op=None):
    o = _c128(O).view(np.float64)
    p = _c128(P).view(np.float64)
    s = _c128(string_op).view(np.float64) if string_op is not None else None
    out = np.zeros(2)
    check(lib.ite_correlator(ctx.h, psi.h, _dptr(o), i, _dptr(p), j,
                             _dptr(s) if s is not None else None, _dptr(out)), ctx.h)
    return complex(out[0], out[1])


# ------------------------------------------------------------------ kernel level
def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _cpair(z):
    a = np.array([complex(z).real, complex(z).imag])
    return a


def set_kernel_precision(ctx, precision):
    """Precision of the kernel-level contractions ("fp64" or "fp64_tc")."""
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    check(lib.ite_ctx_set_kernel_precision(ctx.h, p), ctx.h)


def k_heff(ctx, H, i, L_env, R_env, X, Y, alpha=1.0, Z=None, gamma=0.0):
    """Device tensors (torch complex128): L (D, chl_bra, chl_ket), R (D, chr_ket,
    chr_bra), X (chl_ket, d, d, chr_ket), Y/Z (chl_bra, d, d, chr_bra)."""
    a, g = _cpair(alpha), _cpair(gamma)
    check(lib.ite_k_heff(ctx.h, H.h, i, L_env.shape[1], L_env.shape[2], R_env.shape[1],
                         R_env.shape[2], _p(L_env), _p(R_env), _p(X), _p(Y), _dptr(a), _p(Z),
                         _dptr(g)), ctx.h)


def k_heff_lp_prepare(ctx, H, i, L_env, R_env, precision="mixed_bf16"):
    """Embed the environments for the low-precision H_eff (device tensors laid
    out as for k_heff)."""
    D0, chlB, chlK = L_env.shape
    D2, chrK, chrB = R_env.shape
    check(lib.ite_k_heff_lp_prepare(ctx.h, H.h, i, chlB, chlK, chrK, chrB, _p(L_env), _p(R_env),
                                    PRECISIONS[precision]), ctx.h)


def k_heff_lp_apply(ctx, H, i, X, Y, alpha=1.0, Z=None, gamma=0.0):
    """Y = alpha H_eff X + gamma Z with the operands of the last k_heff_lp_prepare."""
    chlK, chrK = X.shape[0], X.shape[3]
    chlB, chrB = Y.shape[0], Y.shape[3]
    check(lib.ite_k_heff_lp_apply(ctx.h, H.h, i, chlB, chlK, chrK, chrB, _p(X), _p(Y),
                                  _dptr(_cpair(alpha)), _p(Z) if Z is not None else None,
                                  _dptr(_cpair(gamma))), ctx.h)


def k_heff_lp_apply_n(ctx, H, i, X, Y, alpha=1.0, Z=None, gamma=0.0, reps=1):
    """k_heff_lp_apply reps times back to back, one synchronisation at the end."""
    chlK, chrK = X.shape[0], X.shape[3]
    chlB, chrB = Y.shape[0], Y.shape[3]
    check(lib.ite_k_heff_lp_apply_n(ctx.h, H.h, i, chlB, chlK, chrK, chrB, _p(X), _p(Y),
                                    _dptr(_cpair(alpha)), _p(Z) if Z is not None else None,
                                    _dptr(_cpair(gamma)), int(reps)), ctx.h)


def k_env_left(ctx, H, i, Lin, bra, ket, Lout):
    check(lib.ite_k_env_left(ctx.h, H.h, i, bra.shape[0], ket.shape[0], bra.shape[2], ket.shape[2],
                             _p(Lin), _p(bra), _p(ket), _p(Lout)), ctx.h)


def k_env_right(ctx, H, i, Rin, bra, ket, Rout):
    check(lib.ite_k_env_right(ctx.h, H.h, i, bra.shape[0], ket.shape[0], bra.shape[2],
                              ket.shape[2], _p(Rin), _p(bra), _p(ket), _p(Rout)), ctx.h)


def k_local_solve(ctx, H, i, L_env, R_env, B, X, alpha, c, krylov_dim=10, local_tol=0.0):
    steps, res = C.c_int(), C.c_double()
    check(lib.ite_k_local_solve(ctx.h, H.h, i, X.shape[0], X.shape[3], _p(L_env), _p(R_env),
                                _p(B), _p(X), alpha, c, krylov_dim, local_tol, C.byref(steps),
                                C.byref(res)), ctx.h)
    return steps.value, res.value


def k_split(ctx, X, m, n, chi_max, cutoff, centre_right, left, right, sigma=None, tc=False):
    r, disc = C.c_int(), C.c_double()
    flags = 1 if tc else 0
    check(lib.ite_k_split(ctx.h, _p(X), m, n, chi_max, cutoff, 1 if centre_right else 0, _p(left),
                          _p(right), _p(sigma), C.byref(r), C.byref(disc), flags), ctx.h)
    return r.value, disc.value


def k_barrier_selftest(ctx, blocks, absent):
    """ite_k_barrier_selftest; returns the status (ITE_OK, or ITE_ETIMEOUT
    when `absent` blocks never reach the barrier)."""
    return int(lib.ite_k_barrier_selftest(ctx.h, blocks, absent))


# ------------------------------------------------------------------ profiling
PROFILE_CATEGORIES = ("heff", "env", "solve", "svd", "gauge", "project", "step", "lq", "jacobi",
                      "heff_lp")
PROFILE_SLOTS = 16


def kernel_launches():
    return int(lib.ite_kernel_launches())


def profile_start(ctx):
    check(lib.ite_profile_start(ctx.h), ctx.h)


def profile_stop(ctx):
    ms = np.zeros(PROFILE_SLOTS)
    fl = np.zeros(PROFILE_SLOTS)
    cnt = np.zeros(PROFILE_SLOTS, np.int64)
    check(lib.ite_profile_stop(ctx.h, _dptr(ms), _dptr(fl),
                               cnt.ctypes.data_as(C.POINTER(C.c_longlong))), ctx.h)
    return {k: {"ms": float(ms[i]), "flops": float(fl[i]), "count": int(cnt[i])}
            for i, k in enumerate(PROFILE_CATEGORIES)}


def svd_stats(ctx):
    splits, total, mx = C.c_longlong(), C.c_longlong(), C.c_int()
    fl = np.zeros(3)
    check(lib.ite_svd_stats(ctx.h, C.byref(splits), C.byref(total), C.byref(mx), _dptr(fl)), ctx.h)
    return {"splits": splits.value, "sweeps_mean": total.value / max(1, splits.value),
            "sweeps_max": mx.value, "lq_fp64_flops": float(fl[0]),
            "jacobi_fp64_flops": float(fl[1]), "svd_alg_flops": float(fl[2])}


def k_gemm_bf16(ctx, A, B, Cout, k_tile=64):
    """Cout[M][N] (fp32) = A[M][K] B[N][K]^T on the tensor cores; A, B bf16
    CUDA tensors with K contiguous (row strides multiples of 8)."""
    M, K = A.shape
    N = B.shape[0]
    check(lib.ite_k_gemm_bf16(ctx.h, M, N, K, C.c_void_p(A.data_ptr()), A.stride(0),
                              C.c_void_p(B.data_ptr()), B.stride(0), C.c_void_p(Cout.data_ptr()),
                              Cout.stride(0), 1 if k_tile == 32 else 0), ctx.h)


def k_gemm_lp(ctx, A, B, Cout, bn=256, splits=1, pair=False):
    """Cout[b][s] (fp32) = A[b] B[b]^T over K split s on the tensor cores.  A
    (batch, M, K) or (M, K), B (batch, N, K) or (N, K): bf16 (kind::f16) or
    float32 (read as tf32) CUDA tensors, K contiguous; a 2-D operand is shared
    by the batch.  Cout (splits, batch, M, N) float32."""
    import torch
    tf32 = A.dtype == torch.float32
    A3 = A if A.dim() == 3 else A.unsqueeze(0)
    B3 = B if B.dim() == 3 else B.unsqueeze(0)
    batch = max(A3.shape[0], B3.shape[0])
    M, K = A3.shape[1], A3.shape[2]
    N = B3.shape[1]
    check(lib.ite_k_gemm_lp(ctx.h, M, N, K, batch, C.c_void_p(A3.data_ptr()), A3.stride(1),
                            A3.stride(0) if A.dim() == 3 else 0, C.c_void_p(B3.data_ptr()),
                            B3.stride(1), B3.stride(0) if B.dim() == 3 else 0,
                            C.c_void_p(Cout.data_ptr()), Cout.stride(2), Cout.stride(1),
                            Cout.stride(0), 1 if tf32 else 0, bn, splits, 1 if pair else 0), ctx.h)


def k_zgemm(ctx, A, B, Cout, mode=1, conjA=False, conjB=False, alpha=1.0, beta=0.0, transA=False,
            transB=False):
    """Cout = alpha op(A) op(B) + beta Cout for complex128 CUDA tensors; op is
    an optional transpose (by strides) and conjugation.  mode 0: native FP64,
    mode 1: tensor-core emulation."""
    M, K = (A.shape[1], A.shape[0]) if transA else (A.shape[0], A.shape[1])
    N = B.shape[0] if transB else B.shape[1]
    sAm, sAk = (A.stride(1), A.stride(0)) if transA else (A.stride(0), A.stride(1))
    sBk, sBn = (B.stride(1), B.stride(0)) if transB else (B.stride(0), B.stride(1))
    a, b = _cpair(alpha), _cpair(beta)
    check(lib.ite_k_zgemm(ctx.h, mode, M, N, K, C.c_void_p(A.data_ptr()), sAm, sAk,
                          1 if conjA else 0, C.c_void_p(B.data_ptr()), sBk, sBn, 1 if conjB else 0,
                          C.c_void_p(Cout.data_ptr()), Cout.stride(0), _dptr(a), _dptr(b)), ctx.h)


# ------------------------------------------------------------------ served / batched execution
MODELS = {"heisenberg": L.ITE_MODEL_HEISENBERG, "anderson": L.ITE_MODEL_ANDERSON}


def _bond_caps(N, d, chi_max):
    caps = []
    for b in range(N + 1):
        c = chi_max
        if b * np.log(d) < np.log(chi_max) + 1e-12:
            c = min(c, d ** b)
        if (N - b) * np.log(d) < np.log(chi_max) + 1e-12:
            c = min(c, d ** (N - b))
        caps.append(int(c))
    return caps


def _job_base(holder, model, n, chi_max, cutoff, tau0, tau_max, n_steps, scheme, shift_mode,
              shift0, J, Jz, U, eps_d, eps, V, opts, panels):
    j = L.ite_job()
    j.model = MODELS[model] if isinstance(model, str) else int(model)
    j.n = n
    j.J, j.Jz = J, (J if Jz is None else Jz)
    j.U, j.eps_d = U, eps_d
    if eps is not None:
        holder.eps = np.ascontiguousarray(eps, dtype=np.float64)
        holder.V = np.ascontiguousarray(V, dtype=np.float64)
        j.eps, j.V = _dptr(holder.eps), _dptr(holder.V)
    j.chi_max, j.cutoff = chi_max, cutoff
    j.scheme, j.shift_mode, j.shift0 = _scheme(scheme), shift_mode, shift0
    j.tau0, j.tau_max, j.n_steps = tau0, tau_max, n_steps
    j.grid = L.ITE_JOB_GRID_PANELS if panels else L.ITE_JOB_GRID_GEOMETRIC
    j.panels = panels
    j.opts = opts if opts is not None else solver_opts()
    return j


class Job:
    """One evolution for the server (ite_job): model, product start state
    site_vecs (N, d), truncation, and the geometric grid tau0 -> tau_max in
    n_steps steps, or with panels > 0 the panel grid (panels panels of n_steps
    steps up to tau_max; tau0 unused).  The arrays referenced by the C struct
    live as long as this object."""

    def __init__(self, model, n, site_vecs, chi_max, cutoff, tau0, tau_max, n_steps, scheme="be",
                 shift_mode=SHIFT_CURRENT_ENERGY, shift0=0.0, J=1.0, Jz=None, U=0.0, eps_d=0.0,
                 eps=None, V=None, opts=None, want_state=False, panels=0):
        j = _job_base(self, model, n, chi_max, cutoff, tau0, tau_max, n_steps, scheme, shift_mode,
                      shift0, J, Jz, U, eps_d, eps, V, opts, panels)
        self.sv = _c128(site_vecs)
        self.N, self.d = self.sv.shape
        j.site_vecs = _dptr(self.sv.view(np.float64))
        self.energies = np.zeros(n_steps * (panels if panels else 1))
        j.energies = _dptr(self.energies)
        if want_state:
            caps = _bond_caps(self.N, self.d, chi_max)
            cap = sum(2 * caps[i] * self.d * caps[i + 1] for i in range(self.N))
            self.state = np.zeros(cap)
            self.state_chi = np.zeros(self.N + 1, np.int32)
            j.state, j.state_cap = _dptr(self.state), cap
            j.state_chi = self.state_chi.ctypes.data_as(C.POINTER(C.c_int))
        else:
            self.state = None
        self.c = j

    def device_bytes(self):
        return int(lib.ite_job_device_bytes(C.byref(self.c)))

    def tensors(self):
        """Final state as site tensors (chi_i, d, chi_{i+1}) when want_state."""
        z = self.state.view(np.complex128)
        out, pos = [], 0
        for i in range(self.N):
            cnt = self.state_chi[i] * self.d * self.state_chi[i + 1]
            out.append(z[pos:pos + cnt].reshape(self.state_chi[i], self.d,
                                                self.state_chi[i + 1]).copy())
            pos += cnt
        return out


class MettsJob:
    """A METTS chain for the server (ite_job with metts_samples > 0): from
    config0 over the panel grid (panels panels of steps_per_panel steps up to
    tau_max = beta/2), one draw per row of uniforms (samples, N).  Defaults are
    the paper's: trapezoid rule, shift = the current energy.  After the job:
    energies, obs_values (with obs) and configs (samples, N)."""

    def __init__(self, model, n, config0, chi_max, cutoff, tau_max, panels, steps_per_panel,
                 uniforms, scheme="tr", shift_mode=SHIFT_CURRENT_ENERGY, shift0=0.0,
                 alt_basis=None, obs=None, obs_site=0, J=1.0, Jz=None, U=0.0, eps_d=0.0, eps=None,
                 V=None, opts=None):
        j = _job_base(self, model, n, chi_max, cutoff, 0.0, tau_max, steps_per_panel, scheme,
                      shift_mode, shift0, J, Jz, U, eps_d, eps, V, opts, panels)
        self.u = np.ascontiguousarray(uniforms, np.float64)
        samples, self.N = self.u.shape
        self.config0 = np.ascontiguousarray(config0, np.int32)
        self.energies = np.zeros(samples)
        self.obs_values = np.zeros(samples)
        self.configs = np.zeros((samples, self.N), np.int32)
        j.metts_samples = samples
        j.metts_config0 = self.config0.ctypes.data_as(C.POINTER(C.c_int))
        j.metts_uniforms = _dptr(self.u)
        if alt_basis is not None:
            self.ab = _c128(alt_basis)
            j.metts_alt_basis = _dptr(self.ab.view(np.float64))
        if obs is not None:
            self.ob = _c128(obs)
            j.metts_obs = _dptr(self.ob.view(np.float64))
            j.metts_obs_values = _dptr(self.obs_values)
        j.metts_obs_site = obs_site
        j.metts_energies = _dptr(self.energies)
        j.metts_configs = self.configs.ctypes.data_as(C.POINTER(C.c_int))
        self.c = j

    def device_bytes(self):
        return int(lib.ite_job_device_bytes(C.byref(self.c)))


class Server:
    """Independent evolutions side by side on one GPU (ite_server.h)."""

    def __init__(self, device=0, n_slots=4, mem_budget=0, grouping=0, window_ms=20.0):
        h = C.c_void_p()
        check(lib.ite_server_create(device, n_slots, mem_budget, C.byref(h)))
        self.h = h
        self.jobs = {}
        self.set_grouping(grouping, window_ms)

    def set_grouping(self, mode=0, window_ms=20.0):
        """mode 0 off, 1 continuous batching, 2 gather (ite_server_set_grouping)."""
        check(lib.ite_server_set_grouping(self.h, int(mode), float(window_ms)))

    def submit(self, job):
        t = C.c_longlong()
        check(lib.ite_server_submit(self.h, C.byref(job.c), C.byref(t)))
        self.jobs[t.value] = job
        return t.value

    def poll(self, ticket):
        r = L.ite_job_result()
        st = lib.ite_server_poll(self.h, ticket, C.byref(r))
        if st == L.ITE_PENDING:
            return None
        check(st)
        return r.as_dict()

    def wait(self, ticket):
        r = L.ite_job_result()
        check(lib.ite_server_wait(self.h, ticket, C.byref(r)))
        return r.as_dict()

    def drain(self):
        check(lib.ite_server_drain(self.h))

    def stats(self):
        s = L.ite_server_stats()
        check(lib.ite_server_stats_get(self.h, C.byref(s)))
        return s.as_dict()

    def close(self):
        if self.h:
            lib.ite_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def evolve_batch(jobs, n_slots=4, mem_budget=0, device=0, grouping=0, window_ms=20.0):
    """Run Job objects through a temporary server; returns (results, stats)."""
    n = len(jobs)
    arr = (L.ite_job * n)(*[j.c for j in jobs])
    res = (L.ite_job_result * n)()
    st = L.ite_server_stats()
    check(lib.ite_evolve_batch_grouped(device, n_slots, mem_budget, int(grouping),
                                       float(window_ms), n, arr, res, C.byref(st)))
    return [r.as_dict() for r in res], st.as_dict()
