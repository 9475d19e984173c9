"""Scheme constants, in complex FP64.  Test infrastructure only.

Reference media
    Moulinec-Suquet:  sigma_0 = (sigma_1 + 1)/2                       (Eq. J1)
    Eyre-Milton:      sigma_0 = sqrt(sigma_1), principal branch       (Eq. J2)
    MS in H'':        sigma_0'' = (t + 1)/2                           (Eq. J42a)
    EM in H'':        sigma_0'' = sqrt(t)                             (Eq. J43)

Substitution constants (matrix conductivity sigma_2 = 1, 0 < alpha < beta)
    t = (sigma_1 + alpha)(1 + beta) / ((sigma_1 + beta)(1 + alpha))  (Eq. J3, J6, J23)
    p is obtained by solving Eq. J24 for p_1^2, p_2^2 with p_1^2 + p_2^2 + p_3^2 = 1:
        p_1^2 = (1 + alpha)(1 + beta)/(beta - alpha)   (> 0, p_1 real)
        p_2^2 = -(1 + alpha)/(beta - alpha)            (< 0, p_2 imaginary)
        p_3^2 = -alpha(1 + beta)/(beta - alpha)        (< 0, p_3 imaginary)
    E_2' = (1 - t) p_1 p_2 / ((t - 1) p_2^2 + 1)       (Eq. J21 with sigma_2 = 1)
    J_3' = p_1 p_3 (t - 1) / ((t - 1) p_2^2 + 1)       (Eq. J26 with sigma_2 = 1)
The signs of p_2 and p_3 are a free choice (only p_2^2, p_3^2 are fixed); the
oracle takes p_2 = +i sqrt(-p_2^2), p_3 = +i sqrt(-p_3^2).
"""
from __future__ import annotations

import cmath
from dataclasses import dataclass


def ms_sigma0(sigma1: complex) -> complex:
    return (complex(sigma1) + 1.0) / 2.0


def em_sigma0(sigma1: complex) -> complex:
    return cmath.sqrt(complex(sigma1))


def ms_z(sigma1: complex) -> complex:
    """Expansion variable of the Moulinec-Suquet series, Eq. J1."""
    s = complex(sigma1)
    return (s - 1.0) / (s + 1.0)


def em_z(sigma1: complex) -> complex:
    """Expansion variable of the Eyre-Milton series, Eq. J2."""
    w = cmath.sqrt(complex(sigma1))
    return (w - 1.0) / (w + 1.0)


def t_of_sigma1(sigma1: complex, alpha: float, beta: float) -> complex:
    """Slit map of Eq. J3: sends [-beta, -alpha] to (-inf, 0] and sigma_1 = 1 to t = 1."""
    s = complex(sigma1)
    return (s + alpha) * (1.0 + beta) / ((s + beta) * (1.0 + alpha))


def sigma1_of_t(t: complex, p1sq: complex, p2sq: complex) -> complex:
    """Effective modulus of the three-dimensional collection H' (Eq. J22, sigma_2 = 1)."""
    return 1.0 + p1sq / (p2sq + 1.0 / (t - 1.0))


def alpha_beta_of_p(p1sq: complex, p2sq: complex):
    """Eq. J24."""
    return -1.0 - p1sq / (p2sq - 1.0), -1.0 - p1sq / p2sq


@dataclass(frozen=True)
class SubConstants:
    alpha: float
    beta: float
    p1sq: float
    p2sq: float
    p3sq: float
    p1: complex
    p2: complex
    p3: complex
    t: complex
    sqrt_t: complex
    E2p: complex
    J3p: complex


def sub_constants(sigma1: complex, alpha: float, beta: float,
                  sign2: int = 1, sign3: int = 1) -> SubConstants:
    """Constants of the substituted space H'' for inclusion conductivity sigma_1."""
    alpha = float(alpha)
    beta = float(beta)
    if not (0.0 < alpha < beta):
        raise ValueError("need 0 < alpha < beta")
    d = beta - alpha
    p1sq = (1.0 + alpha) * (1.0 + beta) / d
    p2sq = -(1.0 + alpha) / d
    p3sq = -alpha * (1.0 + beta) / d
    p1 = complex(cmath.sqrt(p1sq).real, 0.0)
    p2 = sign2 * 1j * cmath.sqrt(-p2sq).real
    p3 = sign3 * 1j * cmath.sqrt(-p3sq).real
    t = t_of_sigma1(sigma1, alpha, beta)
    den = (t - 1.0) * p2sq + 1.0
    E2p = (1.0 - t) * p1 * p2 / den
    J3p = p1 * p3 * (t - 1.0) / den
    return SubConstants(alpha, beta, p1sq, p2sq, p3sq, p1, p2, p3, t, cmath.sqrt(t), E2p, J3p)
