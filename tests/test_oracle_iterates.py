"""Pins on the iterate paths of the four oracle schemes (not only their fixed
points): starting states, one update against dense real-space definitions
built from the paper's operators, and the exact error recurrences of a medium
whose sigma_*(sigma_1) has a single pole.

Single-pole medium.  A laminate whose layers are normal to the applied field
has sigma_* = 1/(f/sigma_1 + 1 - f) (the harmonic mean), one pole at
s_p = -f/(1 - f), i.e. one weighted eigenvalue m = 1/(1 - s_p) = 1 - f of
chi Gamma_1 chi.  Every field of every scheme is then piecewise constant across
the layers, and the errors obey closed forms:

* MS (Eq. J0-0, J1): the error operator is z Gamma_1 (1 - 2 chi) with
  z = (sigma_1 - 1)/(sigma_1 + 1); on the weighted mode it multiplies the
  sigma_k error by z (1 - 2 m) per iteration, exactly.
* MS in H'' (Eq. J42a, reference (t + 1)/2): the same with z'' = (t - 1)/(t + 1)
  and the pole of sigma_*''(t) at t_p = t(s_p) (Eq. J3), m'' = 1/(1 - t_p).
* EM (Eq. J2) and EM in H'' (Eq. J43): the error operator is w (I - 2 Gamma_1)(1 - 2 chi),
  w = (1 - sqrt s)/(1 + sqrt s) with s = sigma_1 or t; a product of two reflections
  whose restriction to the weighted mode has trace 2 w (2 m - 1) and
  determinant w^2.  Any linear functional x_k of the iterate error (here
  <E_k>.e - |e|^2 and <J_k>.e - sigma_* |e|^2) satisfies
  x_{k+2} = 2 w (2 m - 1) x_{k+1} - w^2 x_k.
A wrong reference medium, a wrong w or a wrong reflection changes these
ratios; the tests at the end plant such mistakes in the oracle and check that
a pin fails.
"""
import cmath

import numpy as np
import pytest

from oracle import fourier as F
from oracle import schemes as S
from synth import random_mask

AB = (0.2, 4.0)


def _layered_mask(n=16, period=8, width=2):
    """Layers normal to y: rows y with y mod period < width are phase 1."""
    m = np.zeros((n, n), np.uint8)
    m[(np.arange(n) % period) < width, :] = 1
    return m


def _slit_map(s, alpha, beta):
    """t(sigma_1) from Eq. J22 solved for t, with p_1^2, p_2^2 from Eq. J24."""
    p1sq, p2sq, _ = _p_squares(alpha, beta)
    return 1.0 + 1.0 / (p1sq / (s - 1.0) - p2sq)


def _p_squares(alpha, beta):
    """Eq. J24 (alpha = -1 - p1^2/(p2^2 - 1), beta = -1 - p1^2/p2^2) as a linear
    system in (p1^2, p2^2), and p3^2 = 1 - p1^2 - p2^2 (p . p = 1)."""
    # (1 + beta) p2^2 + p1^2 = 0;  (1 + alpha)(p2^2 - 1) + p1^2 = 0
    A = np.array([[1.0, 1.0 + beta], [1.0, 1.0 + alpha]])
    rhs = np.array([0.0, 1.0 + alpha])
    p1sq, p2sq = np.linalg.solve(A, rhs)
    return p1sq, p2sq, 1.0 - p1sq - p2sq


def _p_vector(alpha, beta):
    p1sq, p2sq, p3sq = _p_squares(alpha, beta)
    return np.array([np.sqrt(p1sq), 1j * np.sqrt(-p2sq), 1j * np.sqrt(-p3sq)])


# ---------------------------------------------------------------------------
# starting states
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", S.SCHEMES)
@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("s1", [10.0, 0.1, 3 + 4j])
def test_initial_state_is_the_applied_field(scheme, green, s1):
    """E^0 = e for MS and EM; E''^0 = (e, 0, 0) and J''^0 = L'' E''^0 for the
    substituted schemes (start of Eq. J42a / J43; J''_Q equals sigma E only at
    convergence, Eq. J39-J41)."""
    m = random_mask((8, 6), 0.4, seed=3)
    e = np.array([0.6, -0.8])
    pb = S.Problem(m, s1, e, green)
    sch = S.make_scheme(pb, scheme, *AB)
    st = sch.init_state()
    E, J = sch.fields(st)
    ef = pb.e_field()
    np.testing.assert_allclose(E, ef, atol=1e-14)
    if scheme in ("ms", "em"):           # J = sigma E at every iterate of MS and EM
        np.testing.assert_allclose(J, pb.sigma[None] * ef, atol=1e-13)
    if scheme in ("ms_sub", "em_sub"):
        (EQ, ES, ET), (JQ, JS, JT) = sch.full_fields(st)
        np.testing.assert_allclose(EQ, ef, atol=1e-14)
        assert np.abs(ES).max() < 1e-14 and np.abs(ET).max() < 1e-14
        # J'' = L'' E'' = E'' + (t - 1) p (p . E'') chi: on phase 1 (p1 e, p2 e, p3 e)(t - 1) p1
        t = _slit_map(s1, *AB)
        p = _p_vector(*AB)
        chi = m[None].astype(float)
        for comp, Jc in zip(range(3), (JQ, JS, JT)):
            ref = (comp == 0) * ef + (t - 1.0) * p[comp] * p[0] * chi * ef
            np.testing.assert_allclose(Jc, ref, atol=1e-12)


# ---------------------------------------------------------------------------
# one update against dense real-space definitions
# ---------------------------------------------------------------------------
def _dense_gamma(shape, green):
    """Gamma_1 as a dense (d N) x (d N) matrix from its real-space kernel."""
    g = F.gamma_real_space_kernel(shape, green)
    d = len(shape)
    N = int(np.prod(shape))
    idx = np.array(np.unravel_index(np.arange(N), shape))             # (d, N) spatial coords
    diff = tuple((idx[ax][:, None] - idx[ax][None, :]) % shape[ax] for ax in range(d))
    G = np.zeros((d * N, d * N), dtype=np.complex128)
    for a in range(d):
        for b in range(d):
            G[a * N:(a + 1) * N, b * N:(b + 1) * N] = g[a, b][diff]
    return G


def _flat(f):
    return f.reshape(-1)


def _setup(green, s1, seed):
    m = random_mask((6, 4), 0.5, seed=seed)
    e = np.array([1.0, 0.5])
    pb = S.Problem(m, s1, e, green)
    G = _dense_gamma(m.shape, green)
    rng = np.random.default_rng(seed + 100)
    rnd = lambda: rng.standard_normal((2,) + m.shape) + 1j * rng.standard_normal((2,) + m.shape)
    return m, e, pb, G, rnd


def _L_matrix(t, p, inc):
    """L'' of Eq. J36 at one voxel, acting on (Q, S, T): I + (t - 1) p p^T on phase 1."""
    return np.eye(3) + (t - 1.0) * np.outer(p, p) * inc


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("s1", [4.0, 3 + 2j])
def test_em_step_equals_dense_definition(green, s1):
    """P <- (I - 2 Gamma_1)(W P) + 2 sigma_0 e with W = (sigma - sigma_0)/(sigma + sigma_0),
    sigma_0 = sqrt(sigma_1) (Eq. J2)."""
    m, e, pb, G, rnd = _setup(green, s1, 21)
    sch = S.make_scheme(pb, "em")
    P = rnd()
    new = sch.update({"Q": P})["Q"]
    s0 = cmath.sqrt(s1)
    sig = 1.0 + (s1 - 1.0) * m.astype(float)
    WP = ((sig - s0) / (sig + s0))[None] * P
    ref = _flat(WP) - 2.0 * G @ _flat(WP) + 2.0 * s0 * _flat(pb.e_field())
    np.testing.assert_allclose(_flat(new), ref, atol=1e-12)


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("s1", [4.0, 3 + 2j])
def test_ms_sub_step_equals_dense_definition(green, s1):
    """E'' <- e'' - Gamma_1''[(L''/sigma_0'' - I) E''] with sigma_0'' = (t + 1)/2
    (Eq. J42a), Gamma_1''(Q, S, T) = (Gamma_1 Q, S, 0) (Eq. J44)."""
    m, e, pb, G, rnd = _setup(green, s1, 22)
    sch = S.make_scheme(pb, "ms_sub", *AB)
    chi = m[None].astype(float)
    Q, Sf = rnd(), rnd() * chi
    new = sch.update({"Q": Q, "S": Sf})
    t = _slit_map(s1, *AB)
    p = _p_vector(*AB)
    s0 = (t + 1.0) / 2.0
    tau = np.zeros((3,) + Q.shape, dtype=np.complex128)
    for c in range(2):
        for iy in range(m.shape[0]):
            for ix in range(m.shape[1]):
                L = _L_matrix(t, p, m[iy, ix])
                x = np.array([Q[c, iy, ix], Sf[c, iy, ix], 0.0])
                tau[:, c, iy, ix] = (L / s0 - np.eye(3)) @ x
    refQ = _flat(pb.e_field()) - G @ _flat(tau[0])
    np.testing.assert_allclose(_flat(new["Q"]), refQ, atol=1e-12)
    np.testing.assert_allclose(new["S"], -tau[1] * chi, atol=1e-12)


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("s1", [4.0, 3 + 2j])
def test_em_sub_step_equals_dense_definition(green, s1):
    """P'' <- (I - 2 Gamma_1'')(W'' P'') + 2 sqrt(t) e'' with W'' = (L'' - sqrt t)(L'' + sqrt t)^-1
    voxel by voxel (Eq. J36, J43) and I - 2 Gamma_1'' = ((I - 2 Gamma_1) Q, -S, T) (Eq. J44)."""
    m, e, pb, G, rnd = _setup(green, s1, 23)
    sch = S.make_scheme(pb, "em_sub", *AB)
    chi = m[None].astype(float)
    Q, Sf, Tf = rnd(), rnd() * chi, rnd() * chi
    new = sch.update({"Q": Q, "S": Sf, "T": Tf})
    E_, J_ = sch.full_fields({"Q": Q, "S": Sf, "T": Tf})
    t = _slit_map(s1, *AB)
    p = _p_vector(*AB)
    rt = cmath.sqrt(t)
    WP = np.zeros((3,) + Q.shape, dtype=np.complex128)
    Ed = np.zeros_like(WP)
    for c in range(2):
        for iy in range(m.shape[0]):
            for ix in range(m.shape[1]):
                inc = m[iy, ix]
                L = _L_matrix(t, p, inc)
                W = (L - rt * np.eye(3)) @ np.linalg.inv(L + rt * np.eye(3))
                x = np.array([Q[c, iy, ix], Sf[c, iy, ix], Tf[c, iy, ix]])
                if not inc:          # S and T vanish on phase 2
                    W = np.diag([W[0, 0], 0.0, 0.0])
                WP[:, c, iy, ix] = W @ x
                Ed[:, c, iy, ix] = np.linalg.solve(L + rt * np.eye(3), x) if inc else \
                    np.array([x[0] / (1.0 + rt), 0.0, 0.0])
    refQ = _flat(WP[0]) - 2.0 * G @ _flat(WP[0]) + 2.0 * rt * _flat(pb.e_field())
    np.testing.assert_allclose(_flat(new["Q"]), refQ, atol=1e-12)
    np.testing.assert_allclose(new["S"], -WP[1], atol=1e-12)
    np.testing.assert_allclose(new["T"], WP[2], atol=1e-12)
    # fields of the iterate: P'' = (L'' + sqrt t) E''
    for comp in range(3):
        np.testing.assert_allclose(E_[comp], Ed[comp], atol=1e-12)


# ---------------------------------------------------------------------------
# exact error recurrences on a single-pole medium
# ---------------------------------------------------------------------------
def _single_pole_case(green, s1, scheme, max_iter=14, oracle=S):
    m = _layered_mask()
    f = m.mean()
    e = np.array([0.0, 1.0])
    sp = -f / (1.0 - f)
    sd = 1.0 / (f / s1 + 1.0 - f)
    pb = oracle.Problem(m, s1, e, green)
    r = oracle.solve(pb, scheme, alpha=AB[0], beta=AB[1], tol=0, max_iter=max_iter, record_states=True)
    sch = oracle.make_scheme(pb, scheme, *AB)
    return m, f, sp, sd, r, sch


def _ms_residual(green, s1, scheme):
    m, f, sp, sd, r, _ = _single_pole_case(green, s1, scheme)
    err = r.hist_sigma - sd
    if scheme == "ms":
        q = (s1 - 1.0) / (s1 + 1.0) * (1.0 - 2.0 / (1.0 - sp))
    else:
        t, tp = _slit_map(s1, *AB), _slit_map(sp, *AB)
        q = (t - 1.0) / (t + 1.0) * (1.0 - 2.0 / (1.0 - tp))
    res = err[1:10] - q * err[:9]
    return np.abs(res).max() / np.abs(err[0])


def _em_residual(green, s1, scheme):
    m, f, sp, sd, r, sch = _single_pole_case(green, s1, scheme)
    xE, xJ = [], []
    for st in r.states:
        E, J = sch.fields(st)
        xE.append(E[1].mean() - 1.0)
        xJ.append(J[1].mean() - sd)
    if scheme == "em":
        w, mm = (1 - cmath.sqrt(s1)) / (1 + cmath.sqrt(s1)), 1.0 / (1.0 - sp)
    else:
        t, tp = _slit_map(s1, *AB), _slit_map(sp, *AB)
        w, mm = (1 - cmath.sqrt(t)) / (1 + cmath.sqrt(t)), 1.0 / (1.0 - tp)
    worst = 0.0
    for x in (np.array(xE), np.array(xJ)):
        res = x[2:12] - 2.0 * w * (2.0 * mm - 1.0) * x[1:11] + w * w * x[:10]
        worst = max(worst, np.abs(res).max() / np.abs(x[:3]).max())
    return worst


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("s1", [10.0, 0.1, 100.0, 3 + 4j])
@pytest.mark.parametrize("scheme", ["ms", "ms_sub"])
def test_ms_type_error_ratio_on_single_pole_medium(green, s1, scheme):
    assert _ms_residual(green, s1, scheme) < 1e-12


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("s1", [10.0, 0.1, 100.0, 3 + 4j])
@pytest.mark.parametrize("scheme", ["em", "em_sub"])
def test_em_type_error_recurrence_on_single_pole_medium(green, s1, scheme):
    assert _em_residual(green, s1, scheme) < 1e-12


def test_single_pole_medium_is_single_pole():
    """The layered mask has one weighted pole at -f/(1 - f) (harmonic mean)."""
    from oracle import exact as X

    m = _layered_mask()
    f = m.mean()
    for green in F.GREENS:
        mm, w = X.poles(m, np.array([0.0, 1.0]), green)
        keep = w > 1e-10 * w.sum()
        np.testing.assert_allclose(mm[keep], 1.0 - f, atol=1e-12)


# ---------------------------------------------------------------------------
# planted mistakes: each pin above must notice a wrong constant in the oracle
# ---------------------------------------------------------------------------
def test_pins_notice_a_wrong_ms_sub_reference(monkeypatch):
    orig = S.MSSub.__init__

    def wrong(self, *a, **k):
        orig(self, *a, **k)
        self.s0 = (self.k.t + 1.5) / 2.0          # not Eq. J42a

    monkeypatch.setattr(S.MSSub, "__init__", wrong)
    assert _ms_residual("fd", 10.0, "ms_sub") > 1e-3
    with pytest.raises(AssertionError):
        test_ms_sub_step_equals_dense_definition("fd", 4.0)


def test_pins_notice_a_wrong_em_sub_w(monkeypatch):
    orig = S.EMSub.__init__

    def wrong(self, *a, **k):
        orig(self, *a, **k)
        self.w = self.w * 1.01

    monkeypatch.setattr(S.EMSub, "__init__", wrong)
    assert _em_residual("fd", 10.0, "em_sub") > 1e-4
    with pytest.raises(AssertionError):
        test_em_sub_step_equals_dense_definition("fd", 4.0)


def test_pins_notice_a_wrong_em_reference(monkeypatch):
    orig = S.EM.__init__

    def wrong(self, pb):
        orig(self, pb)
        self.sigma0 = self.sigma0 * 1.1           # not sqrt(sigma_1)
        s = self.pb.sigma
        self.W = (s - self.sigma0) / (s + self.sigma0)

    monkeypatch.setattr(S.EM, "__init__", wrong)
    assert _em_residual("trig", 10.0, "em") > 1e-4
    with pytest.raises(AssertionError):
        test_em_step_equals_dense_definition("trig", 4.0)


def test_pins_notice_a_wrong_starting_state(monkeypatch):
    def zero_start(self):
        z = np.zeros((self.pb.d,) + self.pb.shape, dtype=np.complex128)
        return {"Q": z, "S": z.copy(), "T": z.copy()}

    monkeypatch.setattr(S.EMSub, "init_state", zero_start)
    with pytest.raises(AssertionError):
        test_initial_state_is_the_applied_field("em_sub", "trig", 10.0)
