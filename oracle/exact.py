"""Exact discrete solution, poles of sigma_*(sigma_1), and the identities used
to pin the oracle.  Complex FP64, dense linear algebra.  Test infrastructure only.

Discrete problem (Eq. J12, J13): E = e + E~ with E~ = Gamma_1 E~ and
Gamma_1 (sigma E) = 0.  Since sigma - 1 = (sigma_1 - 1) chi, the unknowns reduce to
the field on the inclusion voxels, u = chi E:
    (I + (sigma_1 - 1) A) u = chi e,      A = chi Gamma_1 chi,
and then E = e - (sigma_1 - 1) Gamma_1 (chi E), sigma_* = <J>.e / <E>.e.
A is Hermitian with spectrum in [0, 1]; with eigenpairs (m_n, u_n) and weights
w_n = |u_n^H (chi e)|^2,
    sigma_*(sigma_1) |e|^2 = |e|^2 + (sigma_1 - 1)/N sum_n w_n / (1 + (sigma_1 - 1) m_n),
so the singularities are simple poles at sigma_1 = 1 - 1/m_n on the negative
real axis (the picture of the introduction and Fig. Jfig1), and the interval
[-beta, -alpha] holding every weighted pole has alpha = 1/m_max - 1,
beta = 1/m_min - 1.  Which poles count as "weighted" needs a cutoff the paper
does not give; the reading here keeps poles whose weight exceeds
`cutoff * sum(w)`.
"""
from __future__ import annotations

import numpy as np

from .fourier import apply_gamma, fft, gamma_real_space_kernel, ifft


def _inclusion_coords(mask):
    return np.argwhere(np.asarray(mask) != 0)


def inclusion_operator(mask, green: str):
    """Dense A = chi Gamma_1 chi on the inclusion voxels, index (a, i) -> a*N1 + i."""
    mask = np.asarray(mask)
    shape = mask.shape
    d = mask.ndim
    g = gamma_real_space_kernel(shape, green)
    coords = _inclusion_coords(mask)
    N1 = coords.shape[0]
    diff = [(coords[:, None, ax] - coords[None, :, ax]) % shape[ax] for ax in range(d)]
    A = np.zeros((d * N1, d * N1), dtype=np.complex128)
    for a in range(d):
        for b in range(d):
            A[a * N1:(a + 1) * N1, b * N1:(b + 1) * N1] = g[a, b][tuple(diff)]
    return A, coords


def _stack_e(e, N1):
    return np.concatenate([np.full(N1, float(ea)) for ea in e]).astype(np.complex128)


def direct_solve(mask, sigma1: complex, e, green: str = "trig"):
    """Exact discrete solution via the reduced dense system on the inclusion voxels.

    Returns (sigma_star, E) with E of shape (d, *shape).
    """
    mask = np.asarray(mask)
    d = mask.ndim
    e = np.asarray(e, dtype=np.float64)
    A, coords = inclusion_operator(mask, green)
    N1 = coords.shape[0]
    s1 = complex(sigma1)
    v = _stack_e(e, N1)
    u = np.linalg.solve(np.eye(d * N1) + (s1 - 1.0) * A, v)
    chiE = np.zeros((d,) + mask.shape, dtype=np.complex128)
    idx = tuple(coords.T)
    for a in range(d):
        chiE[a][idx] = u[a * N1:(a + 1) * N1]
    E = e.reshape((-1,) + (1,) * d) - (s1 - 1.0) * ifft(apply_gamma(fft(chiE), green))
    sigma = 1.0 + (s1 - 1.0) * mask.astype(np.float64)
    J = sigma[None] * E
    mJ = J.reshape(d, -1).mean(axis=1)
    mE = E.reshape(d, -1).mean(axis=1)
    return complex(np.dot(mJ, e) / np.dot(mE, e)), E


def effective_tensor(mask, sigma1: complex, green: str = "trig"):
    """Full effective tensor: column a is <J> for the applied field e_a (<E> = e_a)."""
    mask = np.asarray(mask)
    d = mask.ndim
    sigma = 1.0 + (complex(sigma1) - 1.0) * mask.astype(np.float64)
    out = np.zeros((d, d), dtype=np.complex128)
    for a in range(d):
        e = np.zeros(d)
        e[a] = 1.0
        _, E = direct_solve(mask, sigma1, e, green)
        out[:, a] = (sigma[None] * E).reshape(d, -1).mean(axis=1)
    return out


def direct_solve_full(sigma_field, e, green: str = "trig"):
    """Brute-force solve over all voxels (tiny grids): (I + G diag(sigma - 1)) E~ =
    -G((sigma - 1) e), with G the dense matrix of Gamma_1.  Any per-voxel sigma(x)."""
    sig = np.asarray(sigma_field, dtype=np.complex128)
    shape = sig.shape
    d = sig.ndim
    N = sig.size
    e = np.asarray(e, dtype=np.float64)
    g = gamma_real_space_kernel(shape, green)
    coords = np.argwhere(np.ones(shape, dtype=bool))
    diff = [(coords[:, None, ax] - coords[None, :, ax]) % shape[ax] for ax in range(d)]
    G = np.zeros((d * N, d * N), dtype=np.complex128)
    for a in range(d):
        for b in range(d):
            G[a * N:(a + 1) * N, b * N:(b + 1) * N] = g[a, b][tuple(diff)]
    sm1 = np.tile((sig - 1.0).ravel(), d)
    rhs = -G @ (sm1 * np.repeat(e, N))
    Et = np.linalg.solve(np.eye(d * N) + G * sm1[None, :], rhs)
    E = (Et + np.repeat(e, N)).reshape((d,) + shape)
    J = sig[None] * E
    mJ = J.reshape(d, -1).mean(axis=1)
    mE = E.reshape(d, -1).mean(axis=1)
    return complex(np.dot(mJ, e) / np.dot(mE, e)), E


def poles(mask, e, green: str = "trig", merge_tol: float = 1e-9):
    """Eigenvalues m_n of A = chi Gamma chi and their weights w_n = |u_n^H chi e|^2
    (degenerate eigenvalues within merge_tol are merged, weights summed)."""
    mask = np.asarray(mask)
    A, coords = inclusion_operator(mask, green)
    N1 = coords.shape[0]
    A = (A + A.conj().T) / 2.0
    m, U = np.linalg.eigh(A)
    v = _stack_e(np.asarray(e, dtype=np.float64), N1)
    w = np.abs(U.conj().T @ v) ** 2
    ms, ws = [], []
    for mi, wi in zip(m, w):
        if ms and abs(mi - ms[-1]) < merge_tol:
            ws[-1] += wi
        else:
            ms.append(mi)
            ws.append(wi)
    return np.array(ms), np.array(ws)


def sigma_star_from_poles(m, w, sigma1: complex, N: int, e) -> complex:
    e = np.asarray(e, dtype=np.float64)
    e2 = float(np.dot(e, e))
    s1 = complex(sigma1)
    return (e2 + (s1 - 1.0) / N * np.sum(w / (1.0 + (s1 - 1.0) * m))) / e2


def pole_hull(m, w, cutoff: float = 1e-10, m_floor: float = 1e-14):
    """[alpha, beta] from the weighted poles: alpha = 1/m_max - 1, beta = 1/m_min - 1.

    Returns (alpha, beta, m_min, m_max).
    """
    keep = (w > cutoff * np.sum(w)) & (m > m_floor)
    mk = m[keep]
    mmin, mmax = float(mk.min()), float(mk.max())
    alpha = 1.0 / mmax - 1.0
    beta = 1.0 / mmin - 1.0 if mmin > 0 else np.inf
    return alpha, beta, mmin, mmax


def energy(sigma, E):
    """<sigma E . E> with the bilinear (unconjugated) dot product."""
    d = E.shape[0]
    return complex(np.mean(np.sum(sigma[None] * E * E, axis=0))) if d else 0j


def gradient_sigma_field(E, e):
    """d sigma_* / d sigma(x) = E(x).E(x) / (N |e|^2) (first variation of the
    stationary energy <sigma E . E> = sigma_* |e|^2 of Eq. J12/J13)."""
    e = np.asarray(e, dtype=np.float64)
    N = int(np.prod(E.shape[1:]))
    return np.sum(E * E, axis=0) / (N * float(np.dot(e, e)))
