"""Pins for the exact discrete solution, the poles of sigma_*(sigma_1), the
energy/gradient identities and the Lanczos estimate of [alpha, beta]."""
import numpy as np
import pytest

from oracle import exact as X
from oracle import fourier as F
from oracle import lanczos as L
from synth import random_mask, square_array_mask

E2 = np.array([1.0, 0.0])


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("s1", [10.0, 0.05, 2 - 3j])
def test_reduced_direct_solve_equals_full_brute_force(green, s1):
    m = random_mask((6, 8), 0.35, seed=3)
    sr, Er = X.direct_solve(m, s1, E2, green)
    sf, Ef = X.direct_solve_full(1 + (s1 - 1) * m, E2, green)
    assert abs(sr - sf) < 1e-12 * abs(sf)
    np.testing.assert_allclose(Er, Ef, atol=1e-11)


@pytest.mark.parametrize("green", F.GREENS)
def test_direct_solution_satisfies_field_equations(green):
    """E curl-free with mean e; J = sigma E divergence-free (Eq. J12)."""
    m = square_array_mask(16)
    s1 = 10.0
    _, E = X.direct_solve(m, s1, E2, green)
    sigma = 1 + (s1 - 1) * m
    Eh = F.fft(E)
    Jh = F.fft(sigma[None] * E)
    np.testing.assert_allclose(E.reshape(2, -1).mean(1), E2, atol=1e-13)
    # Gamma_1 E~ = E~  and  Gamma_1 J = 0
    Et = Eh.copy()
    Et[:, 0, 0] = 0
    assert np.abs(F.apply_gamma(Et, green) - Et).max() < 1e-9
    assert np.abs(F.apply_gamma(Jh, green)).max() < 1e-9


@pytest.mark.parametrize("green", F.GREENS)
def test_pole_expansion_equals_direct_solve(green):
    m = square_array_mask(16)
    mm, w = X.poles(m, E2, green)
    assert mm.min() > -1e-12 and mm.max() < 1 + 1e-12                   # 0 <= A <= I
    assert abs(w.sum() - m.sum()) < 1e-9                                  # sum of weights = |chi e|^2
    for s1 in (10.0, 0.01, 1e4, 3 + 4j, -0.2 + 0.01j):
        sd, _ = X.direct_solve(m, s1, E2, green)
        sp = X.sigma_star_from_poles(mm, w, s1, m.size, E2)
        assert abs(sd - sp) < 1e-10 * abs(sd)


def test_fd_hull_is_clean_and_trig_hull_has_outliers():
    """The forward-difference symbol keeps the weighted poles inside a fixed interval;
    the trigonometric one spreads tiny-weight poles over (-inf, 0)."""
    m = square_array_mask(32)
    mm, w = X.poles(m, E2, "fd")
    a10, b10, _, _ = X.pole_hull(mm, w, 1e-10)
    a3, b3, _, _ = X.pole_hull(mm, w, 1e-3)
    assert 0.1 < a10 < 0.25 and 4.0 < b10 < 7.0
    assert a10 <= a3 < 0.5 and 3.0 < b3 <= b10          # the cutoff only trims the ends
    mm, w = X.poles(m, E2, "trig")
    a10, b10, _, _ = X.pole_hull(mm, w, 1e-10)
    assert a10 < 1e-2 and b10 > 1e2


def test_energy_identity_and_euler_relation():
    """sigma_* |e|^2 = <sigma E.E>, i.e. sum_x sigma(x) d sigma_*/d sigma(x) = sigma_*."""
    for s1 in (10.0, 2 + 1j):
        m = square_array_mask(16)
        sd, E = X.direct_solve(m, s1, E2, "trig")
        sigma = 1 + (s1 - 1) * m
        assert abs(X.energy(sigma, E) - sd) < 1e-12 * abs(sd)
        g = X.gradient_sigma_field(E, E2)
        assert abs(np.sum(sigma * g) - sd) < 1e-12 * abs(sd)


def test_gradient_wrt_sigma1_central_difference():
    m = square_array_mask(16)
    for s1 in (20.0, 2 + 1j):
        _, E = X.direct_solve(m, s1, E2, "fd")
        g = np.sum(m * X.gradient_sigma_field(E, E2))
        h = 1e-4
        fd = (X.direct_solve(m, s1 + h, E2, "fd")[0] - X.direct_solve(m, s1 - h, E2, "fd")[0]) / (2 * h)
        assert abs(g - fd) < 1e-7 * abs(fd)


def test_gradient_wrt_voxel_sigma_central_difference():
    rng = np.random.default_rng(4)
    sig = 1.0 + 19.0 * (rng.random((6, 6)) < 0.3)
    _, E = X.direct_solve_full(sig, E2, "trig")
    g = X.gradient_sigma_field(E, E2)
    for (y, x) in [(0, 0), (2, 3), (5, 1)]:
        h = 1e-4
        sp, sm = sig.copy(), sig.copy()
        sp[y, x] += h
        sm[y, x] -= h
        fd = (X.direct_solve_full(sp, E2, "trig")[0] - X.direct_solve_full(sm, E2, "trig")[0]) / (2 * h)
        assert abs(g[y, x] - fd) < 1e-7 * abs(fd) + 1e-12


@pytest.mark.parametrize("green", F.GREENS)
def test_lanczos_nodes_reproduce_measure_and_hull(green):
    m = square_array_mask(16)
    mm, w = X.poles(m, E2, green)
    th, wt, _, _ = L.lanczos_nodes(m, E2, green, steps=80)
    # Gauss quadrature reproduces the low moments of the spectral measure
    for p in range(6):
        assert abs(np.sum(wt * th ** p) - np.sum(w * mm ** p)) < 1e-9 * np.sum(w)
    if green == "fd":
        a, b, _, _ = X.pole_hull(mm, w, 1e-10)
        la, lb = L.lanczos_hull(th, wt, 1e-10)
        assert abs(la - a) < 1e-6 * a and abs(lb - b) < 1e-6 * b


def test_effective_tensor_diagonal_laminate_closed_form():
    """Layers normal to n = (1,1)/sqrt 2 (mask a function of x + y), volume fraction
    1/2, forward-difference symbol: the discrete fields are exactly one-dimensional,
    so sigma_* = s_h n n^T + s_a (I - n n^T) with the harmonic and arithmetic means
    (a non-diagonal tensor; the anisotropic case of Eq. J13)."""
    n, w = 32, 4
    s = (np.arange(n)[:, None] + np.arange(n)[None, :]) % (2 * w)
    mask = (s < w).astype(np.uint8)
    nn = np.full((2, 2), 0.5)
    for s1 in (10.0, 0.2 + 0.7j):
        sa = 0.5 * s1 + 0.5
        sh = 1.0 / (0.5 / s1 + 0.5)
        expect = sh * nn + sa * (np.eye(2) - nn)
        got = X.effective_tensor(mask, s1, "fd")
        np.testing.assert_allclose(got, expect, rtol=1e-11, atol=1e-12)
