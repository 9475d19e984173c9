"""Pins for the substitution constants against the paper's scalar identities
(Eq. J3, J19-J26) and the monotonicity argument of section "Proof of acceleration"."""
import cmath
import json
import os

import numpy as np
import pytest

from oracle import constants as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")
HULLS = [(1 / 3, 3.0), (0.25, 4.0), (0.17, 5.8), (1e-3, 1e3)]
SIGMAS = [10.0, 0.01, 1e4, 0.0, 3 + 4j, -0.5 + 0.2j, 2.5e-3 - 1j]


@pytest.mark.parametrize("alpha,beta", HULLS)
def test_p_is_unit_in_bilinear_sense_and_reproduces_alpha_beta(alpha, beta):
    k = C.sub_constants(2.0, alpha, beta)
    assert abs(k.p1 ** 2 + k.p2 ** 2 + k.p3 ** 2 - 1.0) < 1e-13           # p.p = 1
    a, b = C.alpha_beta_of_p(k.p1 ** 2, k.p2 ** 2)                         # Eq. J24
    assert abs(a - alpha) < 1e-12 * max(1, alpha) and abs(b - beta) < 1e-12 * max(1, beta)
    assert k.p1.imag == 0 and k.p2.real == 0 and k.p3.real == 0            # p1 real, p2, p3 imaginary
    # Hermitian norm of p (p p^T is a non-orthogonal projection).
    assert abs(abs(k.p1) ** 2 + abs(k.p2) ** 2 + abs(k.p3) ** 2 - 1.0) > 1e-3


@pytest.mark.parametrize("alpha,beta", HULLS)
@pytest.mark.parametrize("s1", SIGMAS)
def test_t_forms_agree_and_invert(alpha, beta, s1):
    k = C.sub_constants(s1, alpha, beta)
    t_j23 = 1.0 + (s1 - 1.0) / (k.p1sq - k.p2sq * (s1 - 1.0))              # Eq. J23, first form
    t_j3 = 1.0 + (s1 - 1.0) * (beta - alpha) / ((s1 + beta) * (1.0 + alpha))  # Eq. J3, second form
    assert abs(k.t - t_j23) < 1e-12 * max(1, abs(k.t))
    assert abs(k.t - t_j3) < 1e-12 * max(1, abs(k.t))
    if abs(k.t - 1) > 1e-12:
        assert abs(C.sigma1_of_t(k.t, k.p1sq, k.p2sq) - s1) < 1e-9 * max(1, abs(s1))   # Eq. J22


@pytest.mark.parametrize("alpha,beta", HULLS)
def test_t_maps_slit_endpoints(alpha, beta):
    assert abs(C.t_of_sigma1(1.0, alpha, beta) - 1.0) < 1e-15
    assert abs(C.t_of_sigma1(-alpha, alpha, beta)) < 1e-15
    assert abs(1.0 / C.t_of_sigma1(-beta * (1 + 1e-13), alpha, beta)) < 1e-9
    # the slit interior goes to the negative t axis
    for s in np.linspace(-beta, -alpha, 7)[1:-1]:
        t = C.t_of_sigma1(s, alpha, beta)
        assert t.real < 0 and abs(t.imag) < 1e-12


@pytest.mark.parametrize("alpha,beta", HULLS)
@pytest.mark.parametrize("s1", SIGMAS)
def test_three_component_field_equations(alpha, beta, s1):
    """(t - 1) p p^T (1, E2', 0) + (1, E2', 0) = (sigma_1, 0, J3')  (Eq. J19-J26)."""
    k = C.sub_constants(s1, alpha, beta)
    if abs((k.t - 1.0) * k.p2sq + 1.0) < 1e-12:
        pytest.skip("sigma_1 at the pole of E2'")
    p = np.array([k.p1, k.p2, k.p3])
    E = np.array([1.0, k.E2p, 0.0])
    J = (k.t - 1.0) * p * np.dot(p, E) + E
    np.testing.assert_allclose(J, [s1, 0.0, k.J3p], atol=1e-10 * max(1, abs(s1)))
    assert abs(k.J3p - k.p3 * (k.t - 1.0) * (k.p1 + k.p2 * k.E2p)) < 1e-10 * max(1, abs(k.J3p))  # Eq. J25


def test_sign_choice_of_p_only_flips_E2p_and_J3p():
    a = C.sub_constants(5.0, 0.3, 3.0, 1, 1)
    b = C.sub_constants(5.0, 0.3, 3.0, -1, -1)
    assert abs(a.E2p + b.E2p) < 1e-14 and abs(a.J3p + b.J3p) < 1e-14 and a.t == b.t


def test_acceleration_monotonicity():
    """For real sigma_1 > 1, t (hence |z| of Eq. J46) decreases as alpha grows and as beta shrinks."""
    s1 = 10.0
    ts = [C.t_of_sigma1(s1, a, 4.0).real for a in np.linspace(0.0, 3.9, 30)]
    assert all(x > y for x, y in zip(ts, ts[1:]))
    ts = [C.t_of_sigma1(s1, 0.25, b).real for b in np.linspace(40.0, 0.3, 30)]
    assert all(x > y for x, y in zip(ts, ts[1:]))
    assert abs(C.t_of_sigma1(s1, 0.0, 4.0) - (1 + (s1 - 1) * 4.0 / (s1 + 4.0))) < 1e-14
    zs = [abs((cmath.sqrt(t) - 1) / (cmath.sqrt(t) + 1)) for t in ts]
    assert all(x > y for x, y in zip(zs, zs[1:]))


def test_obnosov_cut_is_the_papers():
    facts = json.load(open(GOLDEN))
    a, b = facts["obnosov_branch_cut"]["alpha"], facts["obnosov_branch_cut"]["beta"]
    # sigma_* = sqrt((1 + 3 s)/(3 + s)) has its branch points at s = -1/3 and s = -3.
    assert abs(1 + 3 * (-a)) < 1e-15 and abs(3 + (-b)) < 1e-15
    # the slit map with the paper's cut sends both branch points to t = 0 and t = inf
    assert abs(C.t_of_sigma1(-a, a, b)) < 1e-15


@pytest.mark.parametrize("s1", [10.0, 3 + 4j, 0.01])
def test_expansion_variables_in_unit_disk(s1):
    assert abs(C.em_z(s1)) < 1
    t = C.t_of_sigma1(s1, 0.25, 4.0)
    assert abs((cmath.sqrt(t) - 1) / (cmath.sqrt(t) + 1)) < abs(C.em_z(s1)) + 1e-15
