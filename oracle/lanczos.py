"""Lanczos estimate of the pole interval [alpha, beta].  Test infrastructure only.

The paper needs only estimates of alpha and beta (section "Estimating the
parameters alpha and beta").  The poles of sigma_*(sigma_1) are 1 - 1/m_n with m_n
the eigenvalues of A = chi Gamma_1 chi weighted by |u_n^H chi e|^2, i.e. the
spectral measure of A seen from the vector chi e.  Lanczos from v_1 = chi e/|chi e|
builds the Jacobi matrix of that measure; its eigenvalues theta_i (Gauss nodes)
with weights |chi e|^2 y_i[0]^2 approximate the measure, and the extreme nodes
converge to the extreme weighted eigenvalues.  Then alpha ~ 1/theta_max - 1 and
beta ~ 1/theta_min - 1 over nodes whose weight exceeds `cutoff` times the total.

The oracle applies A with FFTs (Eq. J11) on full-grid fields masked by chi and
keeps full re-orthogonalisation, which is slow but leaves no spurious copies.
"""
from __future__ import annotations

import numpy as np

from .fourier import apply_gamma, fft, ifft


def apply_A(v, mask, green):
    chi = np.asarray(mask, dtype=np.float64)[None]
    return chi * ifft(apply_gamma(fft(chi * v), green))


def lanczos_nodes(mask, e, green: str = "trig", steps: int = 60):
    """Gauss nodes and weights of the spectral measure of chi Gamma chi from chi e.

    Returns (theta, weight, a, b) with a, b the Jacobi matrix diagonals.
    """
    mask = np.asarray(mask)
    d = mask.ndim
    e = np.asarray(e, dtype=np.float64)
    chi = mask.astype(np.float64)[None]
    v = chi * e.reshape((-1,) + (1,) * d) * np.ones((d,) + mask.shape)
    v = v.astype(np.complex128)
    nrm0 = np.sqrt(np.vdot(v, v).real)
    V = [v / nrm0]
    a, b = [], []
    for j in range(steps):
        w = apply_A(V[-1], mask, green)
        aj = np.vdot(V[-1], w).real
        a.append(aj)
        w = w - aj * V[-1] - (b[-1] * V[-2] if b else 0.0)
        for q in V:                       # full re-orthogonalisation
            w = w - np.vdot(q, w) * q
        bj = np.sqrt(np.vdot(w, w).real)
        if bj < 1e-12 * nrm0 or j == steps - 1:
            break
        b.append(bj)
        V.append(w / bj)
    T = np.diag(a) + np.diag(b[:len(a) - 1], 1) + np.diag(b[:len(a) - 1], -1)
    theta, Y = np.linalg.eigh(T)
    weight = nrm0 ** 2 * np.abs(Y[0, :]) ** 2
    return theta, weight, np.array(a), np.array(b[:len(a) - 1])


def lanczos_hull(theta, weight, cutoff: float = 1e-10, m_floor: float = 1e-14):
    keep = (weight > cutoff * weight.sum()) & (theta > m_floor)
    tmin, tmax = float(theta[keep].min()), float(theta[keep].max())
    return 1.0 / tmax - 1.0, 1.0 / tmin - 1.0
