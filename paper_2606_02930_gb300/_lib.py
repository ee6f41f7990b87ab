"""ctypes declarations of the C ABI in include/ite.h, include/ite_kernels.h and
include/ite_server.h.

Argument marshalling only: every computation happens in libite.so.  Importing
this module loads the library and fails loudly if it has not been built
(``python -m paper_2606_02930_gb300.build`` or ``__graft_entry__.build()``).
"""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libite.so")

(ITE_OK, ITE_EINVAL, ITE_ENOMEM, ITE_ESINGULAR, ITE_ENOTCONV, ITE_ETIMEOUT, ITE_ECUDA,
 ITE_PENDING) = range(8)
ITE_MODEL_HEISENBERG, ITE_MODEL_ANDERSON = 0, 1
ITE_JOB_GRID_GEOMETRIC, ITE_JOB_GRID_PANELS = 0, 1
(ITE_BACKWARD_EULER, ITE_TRAPEZOID, ITE_GAUSS_LEGENDRE_2, ITE_GAUSS_LEGENDRE_3, ITE_FORWARD_EULER,
 ITE_HEUN) = range(6)
ITE_FP64, ITE_FP64_TC, ITE_MIXED_BF16, ITE_MIXED_TF32 = 0, 1, 2, 3
ITE_SHIFT_FIXED, ITE_SHIFT_CURRENT_ENERGY = 0, 1
STATUS_NAMES = {0: "ITE_OK", 1: "ITE_EINVAL", 2: "ITE_ENOMEM", 3: "ITE_ESINGULAR",
                4: "ITE_ENOTCONV", 5: "ITE_ETIMEOUT", 6: "ITE_ECUDA", 7: "ITE_PENDING"}


class ite_solver_opts(C.Structure):
    _fields_ = [("krylov_dim", C.c_int), ("sweeps", C.c_int), ("local_tol", C.c_double),
                ("sweep_tol", C.c_double), ("fit_sweeps", C.c_int), ("precision", C.c_int),
                ("max_cycles", C.c_int), ("refine_max", C.c_int), ("refine_tol", C.c_double)]


class ite_step_info(C.Structure):
    _fields_ = [("energy", C.c_double), ("norm_before", C.c_double),
                ("max_discarded_weight", C.c_double), ("max_local_residual", C.c_double),
                ("shift", C.c_double), ("max_chi", C.c_int), ("gmres_steps", C.c_int),
                ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ite_job(C.Structure):
    _fields_ = [("model", C.c_int), ("n", C.c_int), ("J", C.c_double), ("Jz", C.c_double),
                ("U", C.c_double), ("eps_d", C.c_double), ("eps", C.POINTER(C.c_double)),
                ("V", C.POINTER(C.c_double)), ("site_vecs", C.POINTER(C.c_double)),
                ("chi_max", C.c_int), ("cutoff", C.c_double), ("scheme", C.c_int),
                ("shift_mode", C.c_int), ("shift0", C.c_double), ("tau0", C.c_double),
                ("tau_max", C.c_double), ("n_steps", C.c_int), ("opts", ite_solver_opts),
                ("energies", C.POINTER(C.c_double)), ("state", C.POINTER(C.c_double)),
                ("state_cap", C.c_size_t), ("state_chi", C.POINTER(C.c_int)),
                ("grid", C.c_int), ("panels", C.c_int), ("metts_samples", C.c_int),
                ("metts_config0", C.POINTER(C.c_int)), ("metts_uniforms", C.POINTER(C.c_double)),
                ("metts_alt_basis", C.POINTER(C.c_double)), ("metts_obs", C.POINTER(C.c_double)),
                ("metts_obs_site", C.c_int), ("metts_energies", C.POINTER(C.c_double)),
                ("metts_obs_values", C.POINTER(C.c_double)), ("metts_configs", C.POINTER(C.c_int))]


class ite_job_result(C.Structure):
    _fields_ = [("status", C.c_int), ("steps_done", C.c_int), ("energy", C.c_double),
                ("max_discarded_weight", C.c_double), ("max_chi", C.c_int),
                ("queue_ms", C.c_double), ("run_ms", C.c_double), ("latency_ms", C.c_double),
                ("device_bytes", C.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ite_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong),
                ("failed", C.c_longlong), ("peak_running", C.c_int),
                ("p50_latency_ms", C.c_double), ("p99_latency_ms", C.c_double),
                ("wall_ms", C.c_double), ("tau_steps", C.c_double),
                ("tau_steps_per_s", C.c_double), ("group_launches", C.c_longlong),
                ("group_items", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ite_alloc_fn = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
ite_free_fn = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)

_vp, _i, _d, _sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
_pi, _pd = C.POINTER(C.c_int), C.POINTER(C.c_double)

# name: (restype, argtypes)
SIGNATURES = {
    "ite_solver_opts_default": (None, [C.POINTER(ite_solver_opts)]),
    "ite_ctx_create": (_i, [_i, _vp, ite_alloc_fn, ite_free_fn, _vp, C.POINTER(_vp)]),
    "ite_ctx_set_stream": (_i, [_vp, _vp]),
    "ite_ctx_destroy": (None, [_vp]),
    "ite_last_error": (C.c_char_p, [_vp]),
    "ite_ctx_device_bytes": (_sz, [_vp]),
    "ite_kernel_launches": (C.c_ulonglong, []),
    "ite_profile_start": (_i, [_vp]),
    "ite_ctx_set_kernel_precision": (_i, [_vp, C.c_int]),
    "ite_svd_stats": (_i, [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), _pi, _pd]),
    "ite_profile_stop": (_i, [_vp, _pd, _pd, C.POINTER(C.c_longlong)]),
    "ite_mpo_create": (_i, [_vp, _i, _pi, _pi, _pd, C.POINTER(_vp)]),
    "ite_mpo_create_heisenberg": (_i, [_vp, _i, _d, _d, C.POINTER(_vp)]),
    "ite_mpo_create_anderson": (_i, [_vp, _i, _pd, _pd, _d, _d, C.POINTER(_vp)]),
    "ite_mpo_length": (_i, [_vp]),
    "ite_mpo_destroy": (None, [_vp]),
    "ite_mps_create": (_i, [_vp, _i, _i, _pi, _pd, _i, C.POINTER(_vp)]),
    "ite_mps_create_product": (_i, [_vp, _i, _i, _pd, _i, C.POINTER(_vp)]),
    "ite_mps_set": (_i, [_vp, _vp, _pi, _pd]),
    "ite_mps_copy": (_i, [_vp, _vp, _vp]),
    "ite_mps_bond_dims": (_i, [_vp, _pi, C.POINTER(_sz)]),
    "ite_mps_get": (_i, [_vp, _vp, _pd, _sz]),
    "ite_mps_destroy": (None, [_vp]),
    "ite_implicit_step": (_i, [_vp, _vp, _vp, _d, _i, _d, _i, _d, C.POINTER(ite_solver_opts),
                               C.POINTER(ite_step_info)]),
    "ite_grid_geometric": (_i, [_d, _d, _i, _pd]),
    "ite_gl_partial_fractions": (_i, [_i, _pd, _pd, _pd]),
    "ite_mps_sample": (_i, [_vp, _vp, _pd, _pd, _pi, _pd]),
    "ite_metts": (_i, [_vp, _vp, _pi, _pd, _i, _i, _i, _d, _i, _d, C.POINTER(ite_solver_opts),
                       _pd, _pd, _i, _i, _pd, _pd, _pd, _pi]),
    "ite_evolve_loggrid": (_i, [_vp, _vp, _vp, _d, _d, _i, _i, _i, _d, _i, _d,
                                C.POINTER(ite_solver_opts), C.POINTER(ite_step_info), _pd]),
    "ite_grid_panels": (_i, [_d, _i, _i, _pd]),
    "ite_evolve_panels": (_i, [_vp, _vp, _vp, _d, _i, _i, _i, _i, _d, _i, _d,
                               C.POINTER(ite_solver_opts), C.POINTER(ite_step_info), _pd]),
    "ite_energy": (_i, [_vp, _vp, _vp, _pd]),
    "ite_overlap": (_i, [_vp, _vp, _vp, _pd]),
    "ite_correlator": (_i, [_vp, _vp, _pd, _i, _pd, _i, _pd, _pd]),
    "ite_k_heff": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _pd, _vp, _pd]),
    "ite_k_env_left": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "ite_k_env_right": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "ite_k_heff_noalloc": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _pd, _vp, _pd]),
    "ite_k_heff_lp_prepare": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _i]),
    "ite_k_gemm_lp": (_i, [_vp, _i, _i, _i, _i, _vp, C.c_longlong, C.c_longlong, _vp,
                           C.c_longlong, C.c_longlong, _vp, C.c_longlong, C.c_longlong,
                           C.c_longlong, _i, _i, _i, _i]),
    "ite_k_heff_lp_apply": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _pd, _vp, _pd]),
    "ite_k_heff_lp_apply_n": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _pd, _vp, _pd, _i]),
    "ite_k_local_solve": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _d, _d, _i, _d, _pi, _pd]),
    "ite_k_gemm_bf16": (_i, [_vp, _i, _i, _i, _vp, C.c_longlong, _vp, C.c_longlong, _vp,
                             C.c_longlong, _i]),
    "ite_k_zgemm": (_i, [_vp, _i, _i, _i, _i, _vp, C.c_longlong, C.c_longlong, _i, _vp,
                         C.c_longlong, C.c_longlong, _i, _vp, C.c_longlong, _pd, _pd]),
    "ite_k_split": (_i, [_vp, _vp, _i, _i, _i, _d, _i, _vp, _vp, _vp, _pi, _pd, _i]),
    "ite_k_barrier_selftest": (_i, [_vp, _i, _i]),
    "ite_mps_bytes": (_i, [_vp, C.POINTER(C.c_size_t)]),
    "ite_mps_save": (_i, [_vp, _vp, C.c_size_t]),
    "ite_mps_load": (_i, [_vp, _vp, C.c_size_t, C.POINTER(_vp)]),
    "ite_mps_checkpoint_info": (_i, [_vp, C.c_size_t, _pi, _pi, _pi, _pi, C.c_size_t,
                                     C.POINTER(C.c_size_t)]),
    "ite_mps_to_dense": (_i, [_vp, _vp, _pd, C.c_size_t]),
    "ite_job_device_bytes": (_sz, [C.POINTER(ite_job)]),
    "ite_server_create": (_i, [_i, _i, _sz, C.POINTER(_vp)]),
    "ite_server_submit": (_i, [_vp, C.POINTER(ite_job), C.POINTER(C.c_longlong)]),
    "ite_server_poll": (_i, [_vp, C.c_longlong, C.POINTER(ite_job_result)]),
    "ite_server_wait": (_i, [_vp, C.c_longlong, C.POINTER(ite_job_result)]),
    "ite_server_drain": (_i, [_vp]),
    "ite_server_stats_get": (_i, [_vp, C.POINTER(ite_server_stats)]),
    "ite_server_destroy": (None, [_vp]),
    "ite_evolve_batch": (_i, [_i, _i, _sz, _i, C.POINTER(ite_job), C.POINTER(ite_job_result),
                              C.POINTER(ite_server_stats)]),
    "ite_evolve_batch_grouped": (_i, [_i, _i, _sz, _i, C.c_double, _i, C.POINTER(ite_job),
                                      C.POINTER(ite_job_result), C.POINTER(ite_server_stats)]),
    "ite_server_set_grouping": (_i, [_vp, _i, C.c_double]),
}


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libite.so not built at {path}: run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


class IteError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, ctx=None):
    if status != ITE_OK:
        msg = lib.ite_last_error(ctx).decode() if ctx else ""
        raise IteError(status, msg)
