"""GB300 (sm_103a) FFT Lippmann-Schwinger solver for two-phase periodic
conductors, after G. W. Milton, "Substitution of subspace collections with
nonorthogonal subspaces to accelerate Fast Fourier Transform methods applied to
conducting composites" (arXiv 2001.08289).

This package is a thin ctypes binding over the C ABI in include/lsfft.h
(liblsfft.so, built in-tree by ``build.py``).  It only marshals arguments:
every step of the iteration runs in the library's CUDA kernels.  Importing the
package does not load the library; the first call does, and raises if the
library is missing or cannot be loaded (there is no CPU fallback).

The names follow the C ABI (lsfft_create_grid, lsfft_solve, ...); `Grid` and
`solve` are convenience wrappers that manage the handles.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

__all__ = [
    "MS", "EM", "MS_SUB", "EM_SUB", "FP32", "FP64", "GREEN_TRIG", "GREEN_FD",
    "OK", "EINVAL", "ENOMEM", "ENOTCONV", "EDIVERGED", "ECUDA",
    "LsfftError", "Opts", "Result", "Grid", "load_library", "library_path",
    "lsfft_version", "lsfft_last_error", "lsfft_strerror", "lsfft_create_grid", "lsfft_create_grid_device",
    "lsfft_destroy_grid", "lsfft_default_opts", "lsfft_solve", "lsfft_copy_field", "lsfft_copy_field_async",
    "lsfft_free_result",
    "lsfft_prepare", "lsfft_launch_passes", "lsfft_fma_peak", "lsfft_field_averages_noalloc", "lsfft_lanczos_hull",
    "lsfft_tridiag_gauss", "lsfft_set_sigma_field", "lsfft_gradient", "lsfft_solve_batch", "solve_batch",
    "lsfft_solve_sweep", "solve_sweep",
    "lsfft_substitution_rates", "lsfft_debug_inject", "lsfft_effective_tensor", "lsfft_set_column_split",
    "lsfft_autotune",
    "make_opts",
    "SCHEMES", "GREENS",
]

MS, EM, MS_SUB, EM_SUB = 0, 1, 2, 3
FP32, FP64 = 0, 1
GREEN_TRIG, GREEN_FD = 0, 1
OK, EINVAL, ENOMEM, ENOTCONV, EDIVERGED, ECUDA = 0, 1, 2, 3, 4, 5
SCHEMES = {"ms": MS, "em": EM, "ms_sub": MS_SUB, "em_sub": EM_SUB}
GREENS = {"trig": GREEN_TRIG, "fd": GREEN_FD}

_PKG = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_PKG, "liblsfft.so")


class LsfftError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lsfft status {status}: {message}")
        self.status = status


class _C128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class Opts(C.Structure):
    """Mirror of lsfft_opts."""
    _fields_ = [("scheme", C.c_int), ("precision", C.c_int), ("green", C.c_int), ("max_iter", C.c_int),
                ("stop_consecutive", C.c_int), ("check_every", C.c_int), ("tol", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double)]


class _Tuning(C.Structure):
    """Mirror of lsfft_tuning."""
    _fields_ = [("check_every", C.c_int), ("column_split", C.c_int), ("ms_per_iter", C.c_double),
                ("candidates", C.c_int)]


class _Job(C.Structure):
    """Mirror of lsfft_job."""
    _fields_ = [("grid", C.c_void_p), ("sigma1", _C128), ("e", C.c_double * 3), ("opts", Opts)]


class _Result(C.Structure):
    """Mirror of lsfft_result."""
    _fields_ = [("sigma_star", _C128), ("sigma1", _C128), ("mean_E", _C128 * 3), ("mean_J", _C128 * 3),
                ("iters", C.c_int),
                ("status", C.c_int), ("hist_len", C.c_int), ("hist_sigma_re", C.POINTER(C.c_double)),
                ("hist_sigma_im", C.POINTER(C.c_double)), ("hist_rel_change", C.POINTER(C.c_double)),
                ("hist_field_norm", C.POINTER(C.c_double)), ("solve_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("packed", C.c_int), ("precision", C.c_int),
                ("d", C.c_int), ("n", C.c_int64 * 3), ("E_device", C.c_void_p)]


_lib = None


def load_library():
    """Load liblsfft.so (once).  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    lib.lsfft_version.restype = C.c_char_p
    lib.lsfft_last_error.restype = C.c_char_p
    lib.lsfft_strerror.restype = C.c_char_p
    lib.lsfft_strerror.argtypes = [C.c_int]
    lib.lsfft_create_grid.argtypes = [C.c_int, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]
    lib.lsfft_create_grid_device.argtypes = lib.lsfft_create_grid.argtypes
    lib.lsfft_destroy_grid.argtypes = [C.c_void_p]
    lib.lsfft_destroy_grid.restype = None
    lib.lsfft_default_opts.argtypes = [C.POINTER(Opts)]
    lib.lsfft_default_opts.restype = None
    lib.lsfft_solve.argtypes = [C.c_void_p, _C128, C.POINTER(C.c_double), C.POINTER(Opts),
                                C.POINTER(C.POINTER(_Result))]
    lib.lsfft_copy_field.argtypes = [C.POINTER(_Result), C.c_void_p, C.c_int]
    lib.lsfft_copy_field_async.argtypes = [C.POINTER(_Result), C.c_void_p, C.c_int, C.c_void_p]
    lib.lsfft_free_result.argtypes = [C.POINTER(_Result)]
    lib.lsfft_free_result.restype = None
    lib.lsfft_prepare.argtypes = [C.c_void_p, _C128, C.POINTER(C.c_double), C.POINTER(Opts)]
    lib.lsfft_launch_passes.argtypes = [C.c_void_p, C.c_int, C.c_int]
    lib.lsfft_fma_peak.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double)]
    lib.lsfft_field_averages_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int64), C.c_void_p, C.c_int, C.c_void_p,
                                                 _C128, C.POINTER(C.c_double), C.c_void_p, C.c_void_p]
    lib.lsfft_noalloc_last_error.restype = C.c_char_p
    lib.lsfft_lanczos_hull.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_int, C.c_int, C.c_double,
                                       C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.lsfft_tridiag_gauss.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.lsfft_set_sigma_field.argtypes = [C.c_void_p, C.c_void_p, C.c_int, _C128]
    lib.lsfft_debug_inject.argtypes = [C.c_void_p, C.c_int]
    lib.lsfft_set_column_split.argtypes = [C.c_void_p, C.c_int]
    lib.lsfft_autotune.argtypes = [C.c_void_p, _C128, C.POINTER(C.c_double), C.POINTER(Opts), C.c_int,
                                   C.POINTER(_Tuning)]
    lib.lsfft_solve_batch.argtypes = [C.c_int, C.POINTER(_Job), C.POINTER(C.POINTER(_Result)), C.POINTER(C.c_int)]
    lib.lsfft_solve_sweep.argtypes = lib.lsfft_solve_batch.argtypes
    lib.lsfft_substitution_rates.argtypes = [_C128, C.c_double, C.c_double, C.POINTER(C.c_double),
                                             C.POINTER(C.c_double)]
    lib.lsfft_effective_tensor.argtypes = [C.c_void_p, _C128, C.POINTER(Opts), C.POINTER(_C128),
                                           C.POINTER(C.POINTER(_Result))]
    lib.lsfft_gradient.argtypes = [C.c_void_p, C.POINTER(_Result), C.POINTER(C.c_double), C.c_void_p,
                                   C.POINTER(_C128), C.POINTER(_C128)]
    _lib = lib
    return lib


# --- names of the C ABI -------------------------------------------------------

def lsfft_version() -> str:
    return load_library().lsfft_version().decode()


def lsfft_last_error() -> str:
    return load_library().lsfft_last_error().decode()


def lsfft_strerror(status: int) -> str:
    return load_library().lsfft_strerror(int(status)).decode()


def _check(status: int, allowed=(OK,)):
    if status not in allowed:
        raise LsfftError(status, f"{lsfft_strerror(status)}: {lsfft_last_error()}")
    return status


def _dims(n):
    arr = (C.c_int64 * 3)(1, 1, 1)
    for i, v in enumerate(n):
        arr[i] = int(v)
    return arr


def lsfft_create_grid(d: int, n, phase_mask_host: np.ndarray, stream: int = 0) -> int:
    mask = np.ascontiguousarray(phase_mask_host, dtype=np.uint8)
    h = C.c_void_p()
    _check(load_library().lsfft_create_grid(int(d), _dims(n), mask.ctypes.data_as(C.c_void_p),
                                            C.c_void_p(stream or None), C.byref(h)))
    return h.value


def lsfft_create_grid_device(d: int, n, mask_device_ptr: int, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load_library().lsfft_create_grid_device(int(d), _dims(n), C.c_void_p(mask_device_ptr),
                                                   C.c_void_p(stream or None), C.byref(h)))
    return h.value


def lsfft_destroy_grid(grid: int) -> None:
    load_library().lsfft_destroy_grid(C.c_void_p(grid))


def lsfft_default_opts() -> Opts:
    o = Opts()
    load_library().lsfft_default_opts(C.byref(o))
    return o


def lsfft_solve(grid: int, sigma1: complex, e, opts: Opts):
    """Returns (status, result pointer); the result exists for OK, ENOTCONV, EDIVERGED."""
    s1 = complex(sigma1)
    ev = (C.c_double * 3)(*[float(x) for x in list(e) + [0.0] * (3 - len(e))])
    out = C.POINTER(_Result)()
    st = load_library().lsfft_solve(C.c_void_p(grid), _C128(s1.real, s1.imag), ev, C.byref(opts), C.byref(out))
    _check(st, (OK, ENOTCONV, EDIVERGED))
    return st, out


def lsfft_copy_field(res, dst_ptr: int, dst_on_device: bool) -> None:
    _check(load_library().lsfft_copy_field(res, C.c_void_p(dst_ptr), int(bool(dst_on_device))))


def lsfft_copy_field_async(res, dst_ptr: int, dst_on_device: bool, stream: int = 0) -> None:
    """Enqueue the copy of E on `stream` (a cudaStream_t as int) and return at once."""
    _check(load_library().lsfft_copy_field_async(res, C.c_void_p(dst_ptr), int(bool(dst_on_device)),
                                                 C.c_void_p(stream)))


def lsfft_free_result(res) -> None:
    load_library().lsfft_free_result(res)


def lsfft_prepare(grid: int, sigma1: complex, e, opts: Opts) -> None:
    s1 = complex(sigma1)
    ev = (C.c_double * 3)(*[float(x) for x in list(e) + [0.0] * (3 - len(e))])
    _check(load_library().lsfft_prepare(C.c_void_p(grid), _C128(s1.real, s1.imag), ev, C.byref(opts)))


def lsfft_field_averages_noalloc(d: int, n, E_ptr: int, precision: int, mask_ptr: int, sigma1: complex, e,
                                 out_ptr: int, stream: int = 0) -> None:
    """Volume averages of a device field into out_ptr (4 d + 3 device doubles)
    with no device allocation; asynchronous on `stream`."""
    s1 = complex(sigma1)
    ev = (C.c_double * 3)(*[float(x) for x in list(e) + [0.0] * (3 - len(e))])
    lib = load_library()
    st = lib.lsfft_field_averages_noalloc(int(d), _dims(n), C.c_void_p(E_ptr), int(precision), C.c_void_p(mask_ptr),
                                          _C128(s1.real, s1.imag), ev, C.c_void_p(out_ptr), C.c_void_p(stream or None))
    if st != OK:
        raise LsfftError(st, f"{lsfft_strerror(st)}: {lib.lsfft_noalloc_last_error().decode()}")


def lsfft_tridiag_gauss(a, b):
    """Gauss nodes and squared first eigenvector components of the Jacobi
    matrix with diagonal a and off-diagonal b (host computation)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    m = a.size
    b = np.ascontiguousarray(b if m > 1 else np.zeros(1), dtype=np.float64)
    nodes = np.empty(m)
    first2 = np.empty(m)
    p = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
    _check(load_library().lsfft_tridiag_gauss(m, p(a), p(b), p(nodes), p(first2)))
    return nodes, first2


def lsfft_lanczos_hull(grid: int, e, green="trig", precision="fp32", steps: int = 60, cutoff: float = 1e-10):
    """(alpha, beta, nodes, weights): pole interval estimate from `steps` Lanczos steps."""
    ev = (C.c_double * 3)(*[float(x) for x in list(e) + [0.0] * (3 - len(e))])
    g = GREENS[green] if isinstance(green, str) else int(green)
    pr = {"fp32": FP32, "fp64": FP64}[precision] if isinstance(precision, str) else int(precision)
    nodes = np.empty(steps)
    weights = np.empty(steps)
    al, be = C.c_double(), C.c_double()
    m = C.c_int()
    p = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
    _check(load_library().lsfft_lanczos_hull(C.c_void_p(grid), ev, g, pr, int(steps), float(cutoff), C.byref(al),
                                             C.byref(be), p(nodes), p(weights), C.byref(m)))
    return al.value, be.value, nodes[:m.value].copy(), weights[:m.value].copy()


def lsfft_substitution_rates(sigma1: complex, alpha: float, beta: float):
    """(rate, limit): EM in H'' converges at `rate` per iteration and is stable
    against rounding only if rate < limit (see include/lsfft.h)."""
    s1 = complex(sigma1)
    r, lim = C.c_double(), C.c_double()
    _check(load_library().lsfft_substitution_rates(_C128(s1.real, s1.imag), float(alpha), float(beta), C.byref(r),
                                                   C.byref(lim)))
    return r.value, lim.value


def lsfft_effective_tensor(grid: int, sigma1: complex, opts: Opts, d: int):
    """(d x d complex tensor, [Result] * d); raises on errors (status other than
    OK, ENOTCONV, EDIVERGED)."""
    lib = load_library()
    out = (_C128 * (d * d))()
    res = (C.POINTER(_Result) * d)()
    s1 = complex(sigma1)
    st = lib.lsfft_effective_tensor(C.c_void_p(grid), _C128(s1.real, s1.imag), C.byref(opts), out, res)
    _check(st, allowed=(OK, ENOTCONV, EDIVERGED))
    S = np.array([complex(v.re, v.im) for v in out]).reshape(d, d)
    return S, [Result(res[a].contents.status, res[a]) for a in range(d)]


def _job_array(jobs):
    n = len(jobs)
    arr = (_Job * max(n, 1))()
    for i, (h, s1, e, o) in enumerate(jobs):
        s1 = complex(s1)
        arr[i].grid = h
        arr[i].sigma1 = _C128(s1.real, s1.imag)
        ev = list(e) + [0.0] * (3 - len(e))
        for c in range(3):
            arr[i].e[c] = float(ev[c])
        arr[i].opts = o
    return arr


def lsfft_solve_sweep(jobs):
    """The batch in one persistent launch (lsfft_solve_sweep).  jobs: list of (grid
    handle, sigma1, e, Opts).  Returns [(status, result pointer or None)]."""
    n = len(jobs)
    arr = _job_array(jobs)
    res = (C.POINTER(_Result) * max(n, 1))()
    st = (C.c_int * max(n, 1))()
    _check(load_library().lsfft_solve_sweep(n, arr, res, st))
    return [(st[i], res[i] if res[i] else None) for i in range(n)]


def solve_sweep(jobs):
    """jobs: list of (Grid, sigma1, e, kwargs for make_opts).  Returns [Result or LsfftError]."""
    out = []
    for st, ptr in lsfft_solve_sweep([(g.handle, s1, e, make_opts(**kw)) for g, s1, e, kw in jobs]):
        out.append(Result(st, ptr) if ptr else LsfftError(st, lsfft_strerror(st)))
    return out


def lsfft_solve_batch(jobs):
    """jobs: list of (grid handle, sigma1, e, Opts).  Returns [(status, result pointer or None)]."""
    n = len(jobs)
    arr = (_Job * max(n, 1))()
    for i, (h, s1, e, o) in enumerate(jobs):
        s1 = complex(s1)
        arr[i].grid = h
        arr[i].sigma1 = _C128(s1.real, s1.imag)
        ev = list(e) + [0.0] * (3 - len(e))
        for c in range(3):
            arr[i].e[c] = float(ev[c])
        arr[i].opts = o
    res = (C.POINTER(_Result) * max(n, 1))()
    st = (C.c_int * max(n, 1))()
    _check(load_library().lsfft_solve_batch(n, arr, res, st))
    return [(st[i], res[i] if res[i] else None) for i in range(n)]


def solve_batch(jobs):
    """jobs: list of (Grid, sigma1, e, kwargs for make_opts).  Returns [Result or LsfftError]."""
    out = []
    for st, ptr in lsfft_solve_batch([(g.handle, s1, e, make_opts(**kw)) for g, s1, e, kw in jobs]):
        out.append(Result(st, ptr) if ptr else LsfftError(st, lsfft_strerror(st)))
    return out


def lsfft_set_sigma_field(grid: int, sigma_ptr, on_device: bool, sigma0: complex = 0.0) -> None:
    """Per-voxel complex conductivity (N lsfft_c128 values at sigma_ptr), or None
    to return to the two-phase medium."""
    s0 = complex(sigma0)
    _check(load_library().lsfft_set_sigma_field(C.c_void_p(grid), C.c_void_p(sigma_ptr) if sigma_ptr else None,
                                                int(bool(on_device)), _C128(s0.real, s0.imag)))


def lsfft_set_column_split(grid: int, split: bool) -> None:
    _check(load_library().lsfft_set_column_split(C.c_void_p(grid), int(bool(split))))


def lsfft_autotune(grid: int, sigma1: complex, e, opts: Opts, iters: int = 32) -> dict:
    ev = (C.c_double * 3)(*[float(x) for x in list(e) + [0.0] * (3 - len(e))])
    s1 = complex(sigma1)
    out = _Tuning()
    _check(load_library().lsfft_autotune(C.c_void_p(grid), _C128(s1.real, s1.imag), ev, C.byref(opts), int(iters),
                                         C.byref(out)))
    return {"check_every": out.check_every, "column_split": out.column_split, "ms_per_iter": out.ms_per_iter,
            "candidates": out.candidates}


def lsfft_debug_inject(grid: int, kind: int) -> None:
    _check(load_library().lsfft_debug_inject(C.c_void_p(grid), int(kind)))


def lsfft_gradient(grid: int, res, e, grad_ptr=None):
    """(d sigma_*/d sigma_1, <sigma E.E>/|e|^2); d sigma_*/d sigma(x) into grad_ptr if given."""
    ev = (C.c_double * 3)(*[float(x) for x in list(e) + [0.0] * (3 - len(e))])
    d1, en = _C128(), _C128()
    _check(load_library().lsfft_gradient(C.c_void_p(grid), res, ev, C.c_void_p(grad_ptr) if grad_ptr else None,
                                         C.byref(d1), C.byref(en)))
    return complex(d1.re, d1.im), complex(en.re, en.im)


def lsfft_launch_passes(grid: int, kind: int, count: int) -> None:
    _check(load_library().lsfft_launch_passes(C.c_void_p(grid), int(kind), int(count)))


def lsfft_fma_peak(paired: bool = False, reps: int = 3) -> float:
    """FP32 FMA throughput of the current device in TFLOP/s (benchmark ceiling)."""
    out = C.c_double()
    _check(load_library().lsfft_fma_peak(int(bool(paired)), int(reps), C.byref(out)))
    return out.value


# --- convenience wrappers ----------------------------------------------------

class Result:
    """Host copy of a solve: sigma_*, averages, history; E on request."""

    def __init__(self, status, ptr):
        r = ptr.contents
        self.status = int(status)
        self.sigma_star = complex(r.sigma_star.re, r.sigma_star.im)
        self.d = r.d
        self.n = tuple(int(r.n[a]) for a in range(r.d))
        self.mean_E = np.array([complex(r.mean_E[c].re, r.mean_E[c].im) for c in range(r.d)])
        self.mean_J = np.array([complex(r.mean_J[c].re, r.mean_J[c].im) for c in range(r.d)])
        self.iterations = int(r.iters)
        L = int(r.hist_len)
        self.hist_sigma = np.array([complex(r.hist_sigma_re[k], r.hist_sigma_im[k]) for k in range(L)])
        self.hist_rel_change = np.array([r.hist_rel_change[k] for k in range(L)])
        self.hist_field_norm = np.array([r.hist_field_norm[k] for k in range(L)])
        self.solve_ms = float(r.solve_ms)
        self.kernel_launches = int(r.kernel_launches)
        self.packed = int(r.packed)    # 0 complex, 1 packed real, 2 packed real with the split layout
        self.precision = int(r.precision)
        self._ptr = ptr

    def field_numpy(self) -> np.ndarray:
        """E as a host complex array of shape (d, *reversed(n)) ([c][z][y][x])."""
        dt = np.complex64 if self.precision == FP32 else np.complex128
        out = np.empty((self.d,) + tuple(reversed(self.n)), dtype=dt)
        lsfft_copy_field(self._ptr, out.ctypes.data, False)
        return out

    def field_into(self, dst_ptr: int) -> None:
        """Copy E into device memory at dst_ptr (e.g. a torch tensor's data_ptr())."""
        lsfft_copy_field(self._ptr, dst_ptr, True)

    def field_into_async(self, dst_ptr: int, on_device: bool, stream: int) -> None:
        """Enqueue the copy of E to dst_ptr (pinned host or device memory) on
        `stream` and return; keep this Result and the destination alive until
        the stream has run the copy."""
        if self._ptr is None:
            raise ValueError("the result has been freed")
        lsfft_copy_field_async(self._ptr, dst_ptr, on_device, stream)

    def field_tensor(self):
        """E as a CUDA torch tensor of shape (d, *reversed(n)) that shares the
        result's device memory (no copy).  The tensor keeps this Result alive;
        the memory is released when both are gone."""
        import torch

        if self._ptr is None:
            raise ValueError("the result has been freed")
        dt = "<c8" if self.precision == FP32 else "<c16"
        shape = (self.d,) + tuple(reversed(self.n))
        holder = _DeviceArray(self, int(self._ptr.contents.E_device), shape, dt)
        return torch.as_tensor(holder, device="cuda")

    def free(self):
        if self._ptr is not None:
            lsfft_free_result(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _DeviceArray:
    """__cuda_array_interface__ view of a result's device field; holds the Result."""

    def __init__(self, owner, ptr: int, shape, typestr: str):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None, "stream": None}


def make_opts(scheme="ms", precision="fp32", green="trig", tol=1e-6, max_iter=1000, stop_consecutive=3,
              check_every=8, alpha=0.0, beta=0.0) -> Opts:
    o = lsfft_default_opts()
    o.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    o.precision = {"fp32": FP32, "fp64": FP64}[precision] if isinstance(precision, str) else int(precision)
    o.green = GREENS[green] if isinstance(green, str) else int(green)
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.stop_consecutive = int(stop_consecutive)
    o.check_every = int(check_every)
    o.alpha = float(alpha)
    o.beta = float(beta)
    return o


class Grid:
    """A phase mask resident on the GPU (lsfft_create_grid / lsfft_destroy_grid).

    mask: uint8 array of shape (n_y, n_x) or (n_z, n_y, n_x) (x fastest), on the
    host (numpy) or on the device (a CUDA torch tensor).
    """

    def __init__(self, mask, stream: int = 0):
        self.handle = None
        shape = tuple(int(s) for s in mask.shape)
        self.d = len(shape)
        self.n = tuple(reversed(shape))
        if hasattr(mask, "is_cuda") and mask.is_cuda:
            import torch

            self._mask_ref = mask.contiguous()
            torch.cuda.current_stream().synchronize()
            self.handle = lsfft_create_grid_device(self.d, self.n, self._mask_ref.data_ptr(), stream)
        else:
            m = np.asarray(mask)
            if hasattr(mask, "numpy"):
                m = mask.numpy()
            self.handle = lsfft_create_grid(self.d, self.n, m, stream)
        self.shape = shape
        self.N = int(math.prod(shape))

    def solve(self, sigma1, e, **kw) -> Result:
        st, ptr = lsfft_solve(self.handle, sigma1, e, make_opts(**kw))
        return Result(st, ptr)

    def prepare(self, sigma1, e, **kw) -> None:
        lsfft_prepare(self.handle, sigma1, e, make_opts(**kw))

    def set_sigma_field(self, sigma, sigma0: complex = 0.0) -> None:
        """Per-voxel conductivity: array of shape `shape` (numpy, or a CUDA torch
        tensor), any real or complex dtype; None returns to the two-phase medium."""
        if sigma is None:
            lsfft_set_sigma_field(self.handle, None, False)
            return
        if hasattr(sigma, "is_cuda") and sigma.is_cuda:
            import torch

            t = sigma.to(torch.complex128).contiguous()
            torch.cuda.current_stream().synchronize()
            lsfft_set_sigma_field(self.handle, t.data_ptr(), True, sigma0)
        else:
            a = np.ascontiguousarray(np.asarray(sigma), dtype=np.complex128)
            lsfft_set_sigma_field(self.handle, a.ctypes.data, False, sigma0)

    def effective_tensor(self, sigma1, **kw):
        """The full d x d effective tensor (lsfft_effective_tensor): d solves with
        applied fields e_a, sigma_* = [<J>] [<E>]^-1 formed in the library.
        Returns (tensor, results)."""
        return lsfft_effective_tensor(self.handle, sigma1, make_opts(**kw), self.d)

    def gradient(self, result, e, grad_ptr=None):
        """(d sigma_*/d sigma_1, energy estimate); d sigma_*/d sigma(x) into grad_ptr."""
        return lsfft_gradient(self.handle, result._ptr, e, grad_ptr)

    def lanczos_hull(self, e, **kw):
        """(alpha, beta, nodes, weights) of the pole measure seen from chi e."""
        return lsfft_lanczos_hull(self.handle, e, **kw)

    def set_column_split(self, split: bool) -> None:
        """Strided-pass layout of 4096/8192-point 2-D columns (lsfft_set_column_split)."""
        lsfft_set_column_split(self.handle, split)

    def launch_passes(self, kind: int, count: int) -> None:
        lsfft_launch_passes(self.handle, kind, count)

    def close(self):
        if self.handle:
            lsfft_destroy_grid(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
