"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point the public headers declare (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in ("ite.h", "ite_kernels.h", "ite_server.h"):
        with open(os.path.join(ROOT, "include", h)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ite_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_02930_gb300 import build
    return build.build()


def test_headers_declare_the_path(libpath):
    names = declared_symbols()
    for need in ("ite_ctx_create", "ite_mpo_create", "ite_mps_create", "ite_implicit_step",
                 "ite_evolve_loggrid", "ite_evolve_panels", "ite_energy", "ite_correlator",
                 "ite_overlap", "ite_k_heff", "ite_k_env_left", "ite_k_env_right",
                 "ite_k_local_solve", "ite_k_split"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(libpath):
    from paper_2606_02930_gb300 import _lib
    assert declared_symbols() <= set(_lib.SIGNATURES)


def test_host_only_calls():
    from paper_2606_02930_gb300 import api
    import numpy as np
    from oracle import grid
    g = api.grid_geometric(1e-3, 1e3, 40)
    assert np.allclose(g, grid.geometric_grid(1e-3, 1e3, 40), rtol=1e-15, atol=0)
    p = api.grid_panels(64.0, 6, 4)
    assert np.allclose(p, grid.panel_grid(64.0, 6, 4), rtol=1e-15, atol=0)
    o = api.solver_opts()
    assert o.krylov_dim == 10 and o.sweeps == 1 and o.fit_sweeps == 1


def test_invalid_arguments_fail_cleanly():
    from paper_2606_02930_gb300 import _lib
    lib = _lib.lib
    assert lib.ite_grid_geometric(0.0, 1.0, 4, None) == _lib.ITE_EINVAL
    assert lib.ite_grid_panels(1.0, 0, 4, None) == _lib.ITE_EINVAL
    out = ctypes.c_void_p()
    # a context on a missing device reports an error instead of aborting
    assert lib.ite_ctx_create(10**6, None, _lib.ite_alloc_fn(), _lib.ite_free_fn(), None,
                              ctypes.byref(out)) != _lib.ITE_OK
    assert lib.ite_last_error(None) == b"null context"
    assert lib.ite_k_barrier_selftest(None, 4, 1) == _lib.ITE_EINVAL
    n = ctypes.c_size_t()
    assert lib.ite_mps_bytes(None, ctypes.byref(n)) == _lib.ITE_EINVAL
    assert lib.ite_mps_save(None, b"x" * 64, 64) == _lib.ITE_EINVAL
    assert lib.ite_mps_load(None, b"ITEMPS01", 8, ctypes.byref(out)) == _lib.ITE_EINVAL
    assert lib.ite_mps_to_dense(None, None, None, 0) == _lib.ITE_EINVAL


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_gl_partial_fractions_match_the_oracle(q):
    # the library's Durand-Kerner poles and residues against numpy's roots of
    # the same Pade denominator (oracle)
    import numpy as np
    from oracle import ed
    from paper_2606_02930_gb300 import api
    z, a, r = api.gl_partial_fractions(q)
    zo, ao, ro = ed.pade_partial_fractions(q)
    assert r == ro
    for zj, aj in zip(zo, ao):
        k = int(np.argmin(np.abs(z - zj)))
        assert abs(z[k] - zj) < 1e-12 * abs(zj)
        assert abs(a[k] - aj) < 1e-11 * abs(aj)


def test_struct_layouts_match_the_headers():
    # offsets and sizes of the structs the binding passes by pointer, from a C
    # program compiled against the headers, against the ctypes declarations
    import ctypes as C
    import shutil
    import subprocess
    from paper_2606_02930_gb300 import _lib as L
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"ite_job": L.ite_job, "ite_job_result": L.ite_job_result,
               "ite_server_stats": L.ite_server_stats, "ite_step_info": L.ite_step_info,
               "ite_solver_opts": L.ite_solver_opts}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ite_server.h"',
             'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['  return 0;', '}']
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    work = os.path.join(root, "_build", "abi_layout")           # git-ignored scratch
    os.makedirs(work, exist_ok=True)
    src = os.path.join(work, "layout.c")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    exe = os.path.join(work, "layout")
    inc = os.path.join(root, "include")
    subprocess.run([gcc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        name, field, value = line.split()
        cls = structs[name]
        want = C.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert int(value) == want, (name, field)


def _checkpoint(N, d, cap, chi, tensors_doubles, magic=b"ITEMPS01"):
    import numpy as np
    head = np.array([N, d, cap] + list(chi), dtype=np.int64).tobytes()
    return magic + head + np.arange(tensors_doubles, dtype=np.float64).tobytes()


def test_checkpoint_header_is_read_without_a_device():
    # the byte image ite_mps_save writes (magic, N, d, chi_cap, chi[0..N],
    # tensors), built here by hand and read back on the host
    from paper_2606_02930_gb300 import api, _lib
    chi = [1, 2, 4, 2, 1]
    nd = 2 * sum(chi[i] * 2 * chi[i + 1] for i in range(4))
    img = _checkpoint(4, 2, 8, chi, nd)
    N, d, cap, got_chi, n = api.checkpoint_info(img)
    assert (N, d, cap, got_chi.tolist(), n) == (4, 2, 8, chi, nd)
    info = _lib.lib.ite_mps_checkpoint_info
    bad = [
        _checkpoint(4, 2, 8, chi, nd, magic=b"ITEMPS02"),     # wrong magic
        img[:30],                                            # truncated header
        img[:-8],                                            # truncated tensors
        _checkpoint(4, 2, 8, [1, 2, 9, 2, 1], 10 ** 4),      # bond above the capacity
        _checkpoint(4, 2, 8, [2, 2, 4, 2, 1], 10 ** 4),      # open boundary bond
        _checkpoint(0, 2, 8, [1], 0),                        # no sites
        _checkpoint(4, 17, 8, chi, 10 ** 4),                 # d out of range
    ]
    for b in bad:
        assert info(b, len(b), None, None, None, None, 0, None) == _lib.ITE_EINVAL
    # too little room for the bond dimensions
    out = (ctypes.c_int * 4)()
    assert info(img, len(img), None, None, None, out, 4, None) == _lib.ITE_EINVAL


def test_checkpoint_parser_refuses_a_header_whose_tensor_count_wraps():
    # d = 16 and N = 2^19 + 4 bonds of 2^20 (each site 2 * 2^20 * 16 * 2^20 =
    # 2^45 doubles): chi = [1, M, ..., M, M - 2, 1, 2, 1] with M = 2^20 makes
    # the total exactly 2^64 + 64 doubles, which a 64-bit sum wraps to 64.  The
    # image carries those 64 doubles; the parser must still refuse it.
    import numpy as np
    from paper_2606_02930_gb300 import _lib
    M, d = 1 << 20, 16
    N = (1 << 19) + 4
    chi = [1] + [M] * (N - 4) + [M - 2, 1, 2, 1]
    assert len(chi) == N + 1
    total = sum(2 * chi[i] * d * chi[i + 1] for i in range(N))
    assert total == 2 ** 64 + 64
    img = _checkpoint(N, d, M, chi, total % 2 ** 64)
    n = ctypes.c_size_t()
    st = _lib.lib.ite_mps_checkpoint_info(img, len(img), None, None, None, None, 0,
                                          ctypes.byref(n))
    assert st == _lib.ITE_EINVAL


def test_checkpoint_parser_survives_arbitrary_bytes():
    # random byte strings and randomly mutated valid images: the parser
    # returns ITE_OK or ITE_EINVAL and never reads past the buffer's end
    # (an accepted image's tensors fit in it)
    import numpy as np
    from paper_2606_02930_gb300 import _lib
    info = _lib.lib.ite_mps_checkpoint_info
    rng = np.random.default_rng(77)
    chi = [1, 2, 4, 4, 2, 1]
    nd = 2 * sum(chi[i] * 2 * chi[i + 1] for i in range(5))
    valid = _checkpoint(5, 2, 4, chi, nd)
    accepted = 0
    for trial in range(3000):
        if trial % 2:
            img = bytearray(valid)
            for _ in range(rng.integers(1, 6)):
                img[rng.integers(len(img))] = rng.integers(256)
            img = bytes(img[: rng.integers(1, len(img) + 1)])
        else:
            img = b"ITEMPS01" + rng.bytes(int(rng.integers(0, 200)))
        N, d, cap, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        st = info(img, len(img), ctypes.byref(N), ctypes.byref(d), ctypes.byref(cap), None, 0,
                  ctypes.byref(n))
        assert st in (_lib.ITE_OK, _lib.ITE_EINVAL)
        if st == _lib.ITE_OK:
            accepted += 1
            assert 8 + 8 * (3 + N.value + 1) + 8 * n.value <= len(img)
    assert accepted > 0
