"""GPU Lanczos estimate of [alpha, beta] against the oracle's exact pole measure
(dense eigen-decomposition of chi Gamma chi, section "Estimating the
parameters alpha and beta")."""
import numpy as np
import pytest

from oracle import exact as X
from oracle import lanczos as OL
from synth import random_mask, square_array_mask

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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 2e-5)])
@pytest.mark.parametrize("green", ["fd", "trig"])
def test_lanczos_moments_match_exact_measure(L, prec, tol, green):
    """Gauss quadrature from s Lanczos steps reproduces the first moments of the measure."""
    mask = square_array_mask(32)
    e = [1.0, 0.0]
    m, w = X.poles(mask, e, green)
    with L.Grid(mask) as g:
        a, b, th, wt = g.lanczos_hull(e, green=green, precision=prec, steps=12, cutoff=1e-10)
    for p in range(5):
        exact = np.sum(w * m ** p)
        assert abs(np.sum(wt * th ** p) - exact) <= tol * np.sum(w), p


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_lanczos_hull_matches_exact_fd_hull(L, prec):
    """For the forward-difference symbol the weighted poles fill a clean interval and
    the extreme Gauss nodes converge to its ends."""
    for mask in (square_array_mask(32), random_mask((32, 64), 0.3, seed=2)):
        e = [1.0, 0.0]
        m, w = X.poles(mask, e, "fd")
        a_ex, b_ex, _, _ = X.pole_hull(m, w, 1e-10)
        with L.Grid(mask) as g:
            a, b, th, wt = g.lanczos_hull(e, green="fd", precision=prec, steps=80, cutoff=1e-10)
        assert abs(a - a_ex) < 1e-3 * a_ex and abs(b - b_ex) < 1e-3 * b_ex, (a, a_ex, b, b_ex)


def test_lanczos_matches_oracle_lanczos_3d(L):
    mask = square_array_mask(16, d=3)
    e = [1.0, 0.0, 0.0]
    th_o, wt_o, a_o, b_o = OL.lanczos_nodes(mask, e, "fd", steps=10)
    with L.Grid(mask) as g:
        a, b, th, wt = g.lanczos_hull(e, green="fd", precision="fp64", steps=10, cutoff=1e-10)
    np.testing.assert_allclose(np.sort(th), np.sort(th_o), atol=1e-9)
    np.testing.assert_allclose(np.sum(wt), np.sum(wt_o), rtol=1e-12)
