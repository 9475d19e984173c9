"""CPU checks of the C ABI library: it builds, loads without a GPU and exports
every function declared in include/*.h; argument checks that precede any CUDA
call work without a device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(lsfft_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2001_08289_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lsfft_create_grid", "lsfft_solve", "lsfft_copy_field", "lsfft_free_result",
                     "lsfft_destroy_grid", "lsfft_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strings_without_gpu(lib):
    lib.lsfft_strerror.restype = ctypes.c_char_p
    lib.lsfft_version.restype = ctypes.c_char_p
    assert lib.lsfft_strerror(1) == b"invalid argument"
    assert b"sm_103a" in lib.lsfft_version()


def test_create_grid_rejects_bad_shapes_before_touching_cuda(lib):
    import paper_2001_08289_gb300 as L

    L.load_library()
    for d, n in [(4, (16, 16, 16)), (2, (15, 16)), (2, (16, 8)), (2, (16384, 16)), (3, (1024, 16, 16))]:
        with pytest.raises(L.LsfftError) as ei:
            L.lsfft_create_grid(d, n, np.zeros(int(np.prod(n)), np.uint8))
        assert ei.value.status == L.EINVAL


def test_tridiag_gauss_matches_dense_eigh(lib):
    """The host Gauss-quadrature helper against numpy's symmetric eigensolver."""
    import paper_2001_08289_gb300 as L

    L.load_library()
    rng = np.random.default_rng(0)
    for m in (1, 2, 5, 40, 120):
        a = rng.uniform(0.0, 1.0, m)
        b = rng.uniform(0.05, 0.5, max(m - 1, 0))
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        w, V = np.linalg.eigh(T)
        nodes, first2 = L.lsfft_tridiag_gauss(a, b)
        order = np.argsort(nodes)
        np.testing.assert_allclose(nodes[order], w, atol=1e-12)
        np.testing.assert_allclose(first2[order], V[0] ** 2, atol=1e-10)
        assert abs(first2.sum() - 1.0) < 1e-12


def test_debug_inject_rejects_null_grid_without_gpu(lib):
    lib.lsfft_debug_inject.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.lsfft_debug_inject(None, 1) == 1


def test_field_copies_reject_null_arguments_without_gpu(lib):
    lib.lsfft_copy_field.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.lsfft_copy_field_async.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    buf = ctypes.create_string_buffer(16)
    assert lib.lsfft_copy_field(None, buf, 0) == 1
    assert lib.lsfft_copy_field_async(None, buf, 0, None) == 1
    assert lib.lsfft_copy_field_async(None, None, 1, None) == 1


def test_effective_tensor_rejects_null_arguments_without_gpu(lib):
    lib.lsfft_effective_tensor.argtypes = [ctypes.c_void_p, ctypes.c_double * 2, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]
    out = ctypes.create_string_buffer(16 * 9)
    assert lib.lsfft_effective_tensor(None, (ctypes.c_double * 2)(1.0, 0.0), None, out, None) == 1


def test_fma_peak_rejects_bad_arguments_without_gpu(lib):
    import paper_2001_08289_gb300 as L

    L.load_library()
    out = ctypes.c_double()
    assert L.load_library().lsfft_fma_peak(0, 0, ctypes.byref(out)) == L.EINVAL
    assert L.load_library().lsfft_fma_peak(0, 3, None) == L.EINVAL
