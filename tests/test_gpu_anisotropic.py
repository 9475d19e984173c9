"""Full effective tensor (lsfft_effective_tensor: d solves, one per applied field
e_a, and [<J>][<E>]^-1 in the library) on masks without square symmetry,
against the FP64 oracle's direct solve and a closed form."""
import numpy as np
import pytest

from oracle import exact as X
from synth import random_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_08289_gb300 as lib
    from paper_2001_08289_gb300 import build

    build.build()
    lib.load_library()
    return lib


def _rect_mask(ny, nx):
    m = np.zeros((ny, nx), np.uint8)
    m[ny // 4: ny // 4 + ny // 8, nx // 8: nx // 8 + 3 * nx // 4] = 1
    return m


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
@pytest.mark.parametrize("scheme", ["ms", "em", "em_sub"])
@pytest.mark.parametrize("s1", [10.0, 2.0 + 3.0j])
def test_effective_tensor_matches_direct_solve(L, prec, tol, scheme, s1):
    for mask in (_rect_mask(32, 64), random_mask((32, 32), 0.3, seed=11)):
        ref = X.effective_tensor(mask, s1, "fd")
        with L.Grid(mask) as g:
            a, b, _, _ = g.lanczos_hull([1.0, 0.0], green="fd", precision="fp64", steps=120, cutoff=1e-10)
            a2, b2, _, _ = g.lanczos_hull([0.0, 1.0], green="fd", precision="fp64", steps=120, cutoff=1e-10)
            lo, hi = min(a, a2) * 0.9, max(b, b2) * 1.1
            S, res = g.effective_tensor(s1, scheme=scheme, precision=prec, green="fd",
                                        tol=1e-13 if prec == "fp64" else 1e-6, max_iter=6000, alpha=lo, beta=hi)
            assert all(r.status == L.OK for r in res)
        assert np.abs(S - ref).max() < tol * np.abs(ref).max(), (S, ref)


def test_effective_tensor_diagonal_laminate_and_3d(L):
    n, w = 64, 8
    s = (np.arange(n)[:, None] + np.arange(n)[None, :]) % (2 * w)
    mask = (s < w).astype(np.uint8)
    s1 = 10.0
    sa, sh = 0.5 * s1 + 0.5, 1.0 / (0.5 / s1 + 0.5)
    nn = np.full((2, 2), 0.5)
    expect = sh * nn + sa * (np.eye(2) - nn)
    with L.Grid(mask) as g:
        S, _ = g.effective_tensor(s1, scheme="em", precision="fp64", green="fd", tol=1e-14, max_iter=4000)
    np.testing.assert_allclose(S, expect, rtol=1e-10, atol=1e-10)

    m3 = random_mask((16, 16, 16), 0.25, seed=12)
    ref = X.effective_tensor(m3, 5.0, "fd")
    with L.Grid(m3) as g:
        S3, _ = g.effective_tensor(5.0, scheme="em", precision="fp64", green="fd", tol=1e-14, max_iter=4000)
    assert np.abs(S3 - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(S3 - S3.T).max() < 1e-10  # reciprocity for real sigma_1


def test_effective_tensor_without_results_and_with_cap(L):
    """results = NULL frees the d solves inside the call; a solve that hits max_iter
    makes the call return ENOTCONV with the tensor of the last iterates."""
    import ctypes as C

    mask = _rect_mask(32, 32)
    lib = L.load_library()
    ref = X.effective_tensor(mask, 4.0, "fd")
    with L.Grid(mask) as g:
        out = (L._C128 * 4)()
        st = lib.lsfft_effective_tensor(C.c_void_p(g.handle), L._C128(4.0, 0.0),
                                        C.byref(L.make_opts(scheme="ms", precision="fp64", green="fd", tol=1e-14,
                                                            max_iter=4000)), out, None)
        assert st == L.OK
        S = np.array([complex(v.re, v.im) for v in out]).reshape(2, 2)
        assert np.abs(S - ref).max() < 1e-10 * np.abs(ref).max()
        st = lib.lsfft_effective_tensor(C.c_void_p(g.handle), L._C128(4.0, 0.0),
                                        C.byref(L.make_opts(scheme="ms", precision="fp64", green="fd", tol=1e-14,
                                                            max_iter=3)), out, None)
        assert st == L.ENOTCONV
