"""Pins for the four oracle schemes: fixed points against the exact discrete
solution, laminate closed forms, Keller's phase interchange, Wiener and
Hashin-Shtrikman bounds, Obnosov's continuum value, the H'' invariants of
Eq. J39-J41, and the convergence rates of Eq. J1, J2, J4/J46."""
import json
import os

import numpy as np
import pytest

from oracle import exact as X
from oracle import fourier as F
from oracle import schemes as S
from synth import laminate_mask, random_mask, square_array_mask

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))
E2 = np.array([1.0, 0.0])


def _solve(mask, s1, scheme, green="trig", e=E2, tol=1e-13, max_iter=3000, ab=(0.25, 4.0), **kw):
    return S.solve(S.Problem(mask, s1, e, green), scheme, alpha=ab[0], beta=ab[1], tol=tol,
                   max_iter=max_iter, **kw)


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("scheme", S.SCHEMES)
@pytest.mark.parametrize("s1", [10.0, 0.1, 3 + 4j])
def test_fixed_point_is_exact_discrete_solution(green, scheme, s1):
    m = square_array_mask(16)
    sd, Ed = X.direct_solve(m, s1, E2, green)
    r = _solve(m, s1, scheme, green, ab=(0.17, 6.0))
    assert r.status == S.STATUS_OK
    assert abs(r.sigma_star - sd) < 1e-11 * abs(sd)
    assert np.abs(r.E - Ed).max() < 1e-8


@pytest.mark.parametrize("scheme", S.SCHEMES)
def test_fixed_point_3d(scheme):
    m = square_array_mask(8, d=3)
    e = np.array([1.0, 0.0, 0.0])
    for green in F.GREENS:
        sd, Ed = X.direct_solve(m, 5.0, e, green)
        r = S.solve(S.Problem(m, 5.0, e, green), scheme, alpha=0.1, beta=10.0, tol=1e-13, max_iter=3000)
        assert abs(r.sigma_star - sd) < 1e-11 * abs(sd)
        assert np.abs(r.E - Ed).max() < 1e-8


def test_ms_step_equals_dense_real_space_definition():
    """One MS update written with the dense real-space Gamma kernel instead of FFTs."""
    m = random_mask((6, 4), 0.5, seed=7)
    pb = S.Problem(m, 4.0, E2, "trig")
    sch = S.make_scheme(pb, "ms")
    rng = np.random.default_rng(8)
    E = rng.standard_normal((2, 6, 4)) + 1j * rng.standard_normal((2, 6, 4))
    new = sch.update({"Q": E})["Q"]
    g = F.gamma_real_space_kernel((6, 4), "trig")
    tau = (pb.sigma / sch.sigma0 - 1.0) * E
    ref = np.zeros_like(E)
    for y in range(6):
        for x in range(4):
            ref[:, y, x] = pb.e
            for yy in range(6):
                for xx in range(4):
                    ref[:, y, x] -= g[:, :, (y - yy) % 6, (x - xx) % 4] @ tau[:, yy, xx]
    np.testing.assert_allclose(new, ref, atol=1e-12)


@pytest.mark.parametrize("scheme", S.SCHEMES)
@pytest.mark.parametrize("green", F.GREENS)
def test_laminate_closed_forms(scheme, green):
    """Layers stacked along y (width 2, even): field along x gives the arithmetic
    mean, field along y the harmonic mean, exactly on the grid."""
    n, w, s1 = 16, 2, 7.0
    m = laminate_mask((n, n), w, axis=0)
    f = m.mean()
    arith = f * s1 + (1 - f)
    harm = 1.0 / (f / s1 + (1 - f))
    rx = _solve(m, s1, scheme, green, e=np.array([1.0, 0.0]), ab=(0.05, 20.0))
    ry = _solve(m, s1, scheme, green, e=np.array([0.0, 1.0]), ab=(0.05, 20.0))
    assert abs(rx.sigma_star - arith) < 1e-11
    assert abs(ry.sigma_star - harm) < 1e-11


@pytest.mark.parametrize("s1", [7.0, 0.2, 2 + 1j])
def test_keller_phase_interchange_odd_grid(s1):
    """2-D duality (matrix 1): rotating J and E by 90 degrees maps the medium with
    inclusion conductivity sigma_1 to the one with 1/sigma_1, so that
    sigma_*(1/sigma_1) = sigma_*(sigma_1)^T / det sigma_*(sigma_1) for any mask, exactly on
    odd grids with the trigonometric symbol (no Nyquist index).  For a square-
    symmetric mask this is sigma_*(sigma_1) sigma_*(1/sigma_1) = 1."""
    m = random_mask((15, 15), 0.4, seed=11)
    A = X.effective_tensor(m, s1, "trig")
    B = X.effective_tensor(m, 1.0 / s1, "trig")
    assert abs(A[0, 1]) > 1e-4                       # the random mask is anisotropic
    np.testing.assert_allclose(B, A.T / np.linalg.det(A), atol=1e-11)
    sq = np.zeros((15, 15), np.uint8)
    sq[4:11, 4:11] = 1
    sxx, _ = X.direct_solve(sq, s1, np.array([1.0, 0.0]), "trig")
    syy, _ = X.direct_solve(sq, 1.0 / s1, np.array([0.0, 1.0]), "trig")
    assert abs(sxx * syy - 1.0) < 1e-11
    r1 = _solve(sq, s1, "em_sub", e=np.array([1.0, 0.0]), ab=(1e-3, 1e3))
    r2 = _solve(sq, 1.0 / s1, "em_sub", e=np.array([0.0, 1.0]), ab=(1e-3, 1e3))
    assert abs(r1.sigma_star * r2.sigma_star - 1.0) < 1e-10


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("s1", [10.0, 0.1, 100.0])
def test_wiener_and_hashin_shtrikman_bounds(green, s1):
    m = square_array_mask(32)
    f = m.mean()
    sd, _ = X.direct_solve(m, s1, E2, green)
    sd = sd.real
    harm = 1 / (f / s1 + (1 - f))
    arith = f * s1 + 1 - f
    assert harm - 1e-12 <= sd <= arith + 1e-12
    # 2-D Hashin-Shtrikman bounds for an isotropic (square-symmetric) two-phase medium
    lo_m, hi_m = (1.0, s1) if s1 > 1 else (s1, 1.0)
    f_lo = f if s1 > 1 else 1 - f     # fraction of the high phase
    hs_lo = lo_m + f_lo / (1 / (hi_m - lo_m) + (1 - f_lo) / (2 * lo_m))
    hs_hi = hi_m + (1 - f_lo) / (1 / (lo_m - hi_m) + f_lo / (2 * hi_m))
    assert hs_lo - 1e-3 <= sd <= hs_hi + 1e-3


@pytest.mark.parametrize("s1", [10.0, 0.1, 100.0])
def test_obnosov_continuum_limit(s1):
    """The discrete sigma_* approaches Eq. J47a as the grid is refined."""
    exact = np.sqrt((1 + 3 * s1) / (3 + s1))
    assert GOLDEN["obnosov_closed_form"]["cite"] == "Eq. J47a"
    errs = []
    for n in (8, 16, 32):
        sd, _ = X.direct_solve(square_array_mask(n), s1, E2, "fd")
        errs.append(abs(sd - exact))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 2e-2 * exact


def test_obnosov_64_within_grid_error():
    sd, _ = X.direct_solve(square_array_mask(64), 10.0, E2, "trig")
    assert abs(sd - np.sqrt(31 / 13)) < 1e-3


@pytest.mark.parametrize("scheme", ["ms_sub", "em_sub"])
@pytest.mark.parametrize("s1", [10.0, 3 + 4j])
def test_substituted_space_invariants(scheme, s1):
    """At convergence E'' = (E, E2' E chi, 0) and J'' = (J, 0, J3' E chi) (Eq. J39-J41)."""
    m = square_array_mask(16)
    r = _solve(m, s1, scheme, "fd", ab=(0.17, 6.0))
    sch = S.make_scheme(S.Problem(m, s1, E2, "fd"), scheme, 0.17, 6.0)
    (EQ, ES, ET), (JQ, JS, JT) = sch.full_fields(r.state)
    chi = m[None].astype(float)
    k = sch.k
    sd, Ed = X.direct_solve(m, s1, E2, "fd")
    assert np.abs(EQ - Ed).max() < 1e-8
    assert np.abs(ES - k.E2p * EQ * chi).max() < 1e-8
    assert np.abs(ET).max() < 1e-8
    assert np.abs(JS).max() < 1e-8
    assert np.abs(JT - k.J3p * EQ * chi).max() < 1e-8
    sigma = 1 + (s1 - 1) * m
    assert np.abs(JQ - sigma[None] * EQ).max() < 1e-8


@pytest.mark.parametrize("scheme", ["ms_sub", "em_sub"])
def test_sign_of_p_flips_S_and_T_only(scheme):
    m = square_array_mask(8)
    pb = S.Problem(m, 5.0, E2, "trig")
    a = S.solve(pb, scheme, alpha=0.2, beta=5.0, tol=0, max_iter=6, record_states=True)
    b = S.solve(pb, scheme, alpha=0.2, beta=5.0, tol=0, max_iter=6, record_states=True, sign2=-1, sign3=-1)
    for sa, sb in zip(a.states, b.states):
        np.testing.assert_allclose(sa["Q"], sb["Q"], atol=1e-13)
        np.testing.assert_allclose(sa["S"], -sb["S"], atol=1e-13)
        if "T" in sa:
            np.testing.assert_allclose(sa["T"], -sb["T"], atol=1e-13)


def test_real_sigma1_gives_real_Q_and_imaginary_S_T():
    m = square_array_mask(8)
    r = S.solve(S.Problem(m, 20.0, E2, "fd"), "em_sub", alpha=0.2, beta=5.0, tol=0, max_iter=5,
                record_states=True)
    for st in r.states:
        assert np.abs(st["Q"].imag).max() < 1e-13
        assert np.abs(st["S"].real).max() < 1e-13
        assert np.abs(st["T"].real).max() < 1e-13


def _observed_ratio(r, s_exact, window=4, floor=1e-12):
    """Mean per-iteration decay of the error envelope (max over `window` iterates),
    which averages out the oscillation of complex iteration eigenvalues."""
    err = np.abs(r.hist_sigma[:-1] - s_exact)
    last = int(np.nonzero(err > floor)[0].max()) - window
    k1 = 4
    env = lambda k: err[k:k + window].max()
    return (env(last) / env(k1)) ** (1.0 / (last - k1))


def test_convergence_rates_match_predictions():
    """Observed asymptotic sigma_* error ratios against Eq. J1, J2 and J46."""
    m = square_array_mask(16)
    mm, w = X.poles(m, E2, "fd")
    a, b, mmin, mmax = X.pole_hull(mm, w, 1e-10)
    s1 = 10.0
    sd, _ = X.direct_solve(m, s1, E2, "fd")
    for scheme in ("em", "em_sub", "ms"):
        r = _solve(m, s1, scheme, "fd", tol=0, max_iter=120, ab=(a, b))
        pred = S.predicted_rate(scheme, s1, a, b, (mmin, mmax))
        obs = _observed_ratio(r, sd)
        assert obs <= pred * 1.1, (scheme, obs, pred)
        assert obs >= pred * 0.5, (scheme, obs, pred)


def test_accelerated_scheme_beats_basic_ones_on_fd_hull():
    """With [alpha, beta] covering the weighted poles, EM in H'' needs fewer iterations."""
    m = square_array_mask(16)
    mm, w = X.poles(m, E2, "fd")
    a, b, _, _ = X.pole_hull(mm, w, 1e-10)
    for s1 in (100.0, 1e4):
        sd, _ = X.direct_solve(m, s1, E2, "fd")
        its = {}
        for scheme in ("ms", "em", "em_sub"):
            r = _solve(m, s1, scheme, "fd", tol=0, max_iter=400, ab=(a, b))
            err = np.abs(r.hist_sigma - sd) / abs(sd)
            above = np.nonzero(err >= 1e-8)[0]
            its[scheme] = np.inf if above.size and above[-1] == len(err) - 1 else (
                int(above[-1]) + 1 if above.size else 0)
        assert its["em_sub"] < its["ms"] and its["em_sub"] < its["em"], its


def test_stop_rule_and_status_codes():
    m = square_array_mask(8)
    r = _solve(m, 10.0, "ms", tol=0, max_iter=5)
    assert r.status == S.STATUS_NOTCONV and r.iterations == 5 and len(r.hist_sigma) == 6
    r = _solve(m, 10.0, "ms", tol=1e-8, max_iter=500)
    assert r.status == S.STATUS_OK
    assert np.all(r.hist_rel_change[r.iterations - 3:r.iterations] < 1e-8)
    assert len(r.hist_sigma) == r.iterations + 1
    r = _solve(m, -2.0, "ms", tol=1e-8, max_iter=5000)    # |z| = 3: diverges
    assert r.status == S.STATUS_DIVERGED


def test_em_undefined_at_sigma1_zero_but_em_sub_defined():
    m = square_array_mask(8)
    with pytest.raises(ValueError):
        S.make_scheme(S.Problem(m, 0.0, E2), "em")
    r = _solve(m, 0.0, "em_sub", "fd", ab=(0.17, 6.0))
    sd, _ = X.direct_solve(m, 0.0, E2, "fd")
    assert abs(r.sigma_star - sd) < 1e-10


def test_per_voxel_sigma_mode_matches_full_direct_solve():
    rng = np.random.default_rng(12)
    sig = 1.0 + 9.0 * rng.random((6, 8))
    pb = S.Problem(np.zeros((6, 8), np.uint8), 1.0, E2, "trig", sigma_field=sig)
    sf, Ef = X.direct_solve_full(sig, E2, "trig")
    for scheme in ("ms", "em"):
        r = S.solve(pb, scheme, tol=1e-14, max_iter=2000)
        assert abs(r.sigma_star - sf) < 1e-11
        assert np.abs(r.E - Ef).max() < 1e-9


def test_substituted_em_rounding_stability_limit():
    """chi Gamma chi has eigenvalues 1 and 0 on modes with no weight for sigma_*; in
    H'' they sit at t(0) and t(inf).  Where |z(t(sigma_1))| exceeds
    min(|z(t(0))|, |z(t(inf))|) the iteration amplifies rounding noise and the field
    diverges although sigma_* converges; below it the field converges."""
    import cmath

    from oracle import constants as C
    from synth import rsa_disk_mask

    m, _ = rsa_disk_mask(64, seed=3)
    mm, w = X.poles(m, E2, "fd")
    a, b, _, _ = X.pole_hull(mm, w, 1e-10)
    a, b = 0.9 * a, 1.1 * b
    zabs = lambda t: abs((cmath.sqrt(t) - 1) / (cmath.sqrt(t) + 1))
    limit = min(zabs(C.t_of_sigma1(0.0, a, b)), zabs((1 + b) / (1 + a)))
    unstable, stable = -0.33 + 0.065j, 3.0 + 4.0j
    assert zabs(C.t_of_sigma1(unstable, a, b)) > limit > zabs(C.t_of_sigma1(stable, a, b))
    ru = S.solve(S.Problem(m, unstable, E2, "fd"), "em_sub", alpha=a, beta=b, tol=1e-6, max_iter=300)
    re_ = S.solve(S.Problem(m, unstable, E2, "fd"), "em", tol=1e-6, max_iter=600)
    rs = S.solve(S.Problem(m, stable, E2, "fd"), "em_sub", alpha=a, beta=b, tol=1e-8, max_iter=300)
    assert re_.status == S.STATUS_OK and rs.status == S.STATUS_OK
    # sigma_* settles to the right value while the field norm runs away: the stop
    # rule, which watches both, never reports convergence
    assert ru.status in (S.STATUS_DIVERGED, S.STATUS_NOTCONV)
    k = int(np.argmax(ru.hist_field_norm > 1e3 * ru.hist_field_norm[0]))
    assert k > 0 and abs(ru.hist_sigma[k] - re_.sigma_star) < 1e-4 * abs(re_.sigma_star)
    assert rs.hist_field_norm.max() < 10 * rs.hist_field_norm[0]


def test_insulating_squares_experiment():
    """The sigma_1 = 0 experiment with [alpha, beta] = [1/4, 4]: MS (reference 1/2) and MS
    in H'' share the bound 0.6 (Eq. J1 with the weighted eigenvalues in [1/5, 4/5];
    Eq. J42a with t(0) = 1/4), EM in H'' has 1/3 (Eq. J46); all reach the same discrete
    sigma_*, which lies within discretisation error of Eq. J47a."""
    from oracle import constants as C

    mask = square_array_mask(64)
    e = np.array([1.0, 0.0])
    assert abs(C.t_of_sigma1(0.0, 0.25, 4.0) - 0.25) < 1e-15
    assert abs(S.predicted_rate("ms_sub", 0.0, 0.25, 4.0) - 0.6) < 1e-15
    assert abs(S.predicted_rate("ms", 0.0, m_hull=(0.2, 0.8)) - 0.6) < 1e-15
    assert abs(S.predicted_rate("em_sub", 0.0, 0.25, 4.0) - 1.0 / 3.0) < 1e-15
    out = {}
    for sch in ("ms", "ms_sub", "em_sub"):
        r = S.solve(S.Problem(mask, 0.0, e, "fd"), sch, alpha=0.25, beta=4.0, tol=1e-10, max_iter=500)
        assert r.status == S.STATUS_OK
        out[sch] = r
    s = out["ms"].sigma_star.real
    for r in out.values():
        assert abs(r.sigma_star - s) < 1e-9
    assert out["em_sub"].iterations < out["ms"].iterations
    assert abs(s - np.sqrt(1.0 / 3.0)) < 1e-3


def test_estimate_sensitivity_of_the_slit():
    """Section "Estimating the parameters alpha and beta": a slit estimate wider
    than the exact weighted-pole interval still converges, at the slower rate its
    own t predicts (Eq. J46); one that leaves poles outside still converges, but
    the poles outside set a factor above the nominal |z| of the estimate."""
    mask = square_array_mask(32)
    e = np.array([1.0, 0.0])
    m, w = X.poles(mask, e, "fd")
    a, b, _, _ = X.pole_hull(m, w, cutoff=1e-10)
    s1 = 100.0
    ref = None
    runs = {}
    for name, (aa, bb) in {"exact": (a, b), "wide": (a * 0.8, b * 1.25), "narrow": (a * 1.4, b * 0.7)}.items():
        r = S.solve(S.Problem(mask, s1, e, "fd"), "em_sub", alpha=aa, beta=bb, tol=1e-12, max_iter=3000)
        assert r.status == S.STATUS_OK
        ref = r.sigma_star if ref is None else ref
        assert abs(r.sigma_star - ref) < 1e-9
        err = np.abs(r.hist_sigma - r.sigma_star)
        # observed asymptotic factor over a window where the error is well above rounding
        ok = np.nonzero(err > 1e-11)[0]
        k1 = ok[-1]
        k0 = max(1, k1 - 8)
        observed = (err[k1] / err[k0]) ** (1.0 / (k1 - k0))
        runs[name] = (r.iterations, observed, S.predicted_rate("em_sub", s1, aa, bb))
    assert runs["wide"][0] >= runs["exact"][0] and runs["narrow"][0] >= runs["exact"][0]
    assert runs["wide"][2] > runs["exact"][2]
    assert runs["exact"][1] <= runs["exact"][2] * 1.05
    assert runs["wide"][1] <= runs["wide"][2] * 1.05
    assert runs["narrow"][1] > runs["narrow"][2] * 1.05
