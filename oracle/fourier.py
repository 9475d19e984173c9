"""Fourier-side pieces of the oracle: frequencies, a brute-force DFT and the
projection Gamma_1 onto periodic gradient fields (Eq. J11, reused as Eq. J45).

Test infrastructure only (see the package docstring).

Conventions
-----------
A field with d components on a grid of shape `shape` is an array of shape
(d, *shape).  `shape` is (n_y, n_x) in 2-D and (n_z, n_y, n_x) in 3-D; component
a = 0 is the x component, a = 1 the y component, a = 2 the z component, so the
frequency k_a lives on spatial axis d-1-a.  The forward DFT is unnormalised,
F(k) = sum_x f(x) exp(-2 pi i k.x/n); the inverse carries 1/N.  Integer
frequencies follow the order 0, 1, ..., n/2-1, -n/2, ..., -1.

Green symbols
-------------
"trig": Gamma(k) = k (x) k / |k|^2 for k != 0 (Eq. J11), and 0 at k = 0.  For even n
        the paper is silent about the Nyquist index k_a = -n/2; the reading used
        here sets Gamma(k) = 0 whenever any component sits at the Nyquist index,
        which keeps Gamma an orthogonal projection that maps real fields to real
        fields.
"fd":   the projection onto forward-difference gradients of the resistor network
        picture (section "Substitution at the level of the Hilbert space"):
        k~_a = exp(2 pi i k_a / n_a) - 1 and Gamma(k) = k~ (x) conj(k~) / |k~|^2,
        0 at k = 0, with no Nyquist special case.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as _sfft

GREENS = ("trig", "fd")

# Threads of the FFT library: every host core (the transforms are the plain
# library routine; only their threading changes, not the arithmetic).
WORKERS = os.cpu_count() or 1


def integer_freqs(n: int) -> np.ndarray:
    """Integer frequencies 0..n/2-1, -n/2..-1 (odd n: 0..(n-1)/2, -(n-1)/2..-1)."""
    return np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)


def freq_components(shape):
    """List [k_x, k_y(, k_z)] of integer frequency arrays broadcastable to `shape`."""
    d = len(shape)
    ks = []
    for a in range(d):
        ax = d - 1 - a
        bshape = [1] * d
        bshape[ax] = shape[ax]
        ks.append(integer_freqs(shape[ax]).reshape(bshape))
    return ks


def spatial_axes(d: int):
    return tuple(range(1, d + 1))


def fft(field: np.ndarray) -> np.ndarray:
    """Unnormalised forward DFT of every component over the spatial axes."""
    d = field.ndim - 1
    return _sfft.fftn(field, axes=spatial_axes(d), workers=WORKERS)


def ifft(field_hat: np.ndarray) -> np.ndarray:
    """Inverse DFT (with the 1/N factor) of every component."""
    d = field_hat.ndim - 1
    return _sfft.ifftn(field_hat, axes=spatial_axes(d), workers=WORKERS)


def brute_force_dft(f: np.ndarray, inverse: bool = False) -> np.ndarray:
    """O(N^2) DFT of a scalar array over all its axes, straight from the definition."""
    shape = f.shape
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    pts = np.stack([g.ravel() for g in grids], axis=1)             # (N, ndim)
    phase = np.zeros((pts.shape[0], pts.shape[0]))
    for ax, n in enumerate(shape):
        phase += np.outer(pts[:, ax], pts[:, ax]) / n
    sign = 1.0 if inverse else -1.0
    M = np.exp(sign * 2j * np.pi * phase)
    out = M @ f.ravel().astype(np.complex128)
    if inverse:
        out /= pts.shape[0]
    return out.reshape(shape)


def symbol_vectors(shape, green: str):
    """Per-frequency vector u(k) with Gamma(k) = u conj(u)^T / |u|^2, and the set
    of frequencies where Gamma(k) is non-zero.

    Returns (u, active): u has shape (d, *shape), complex; active is boolean of
    shape `shape`.
    """
    if green not in GREENS:
        raise ValueError(f"unknown green symbol {green!r}")
    d = len(shape)
    ks = freq_components(shape)
    u = np.zeros((d,) + tuple(shape), dtype=np.complex128)
    active = np.ones(tuple(shape), dtype=bool)
    for a in range(d):
        n_a = shape[d - 1 - a]
        k = np.broadcast_to(ks[a], shape)
        if green == "trig":
            u[a] = k
            if n_a % 2 == 0:
                active &= k != -(n_a // 2)
        else:
            u[a] = np.exp(2j * np.pi * k / n_a) - 1.0
    norm2 = np.sum(np.abs(u) ** 2, axis=0)
    active &= norm2 > 0
    return u, active


def apply_gamma(vhat: np.ndarray, green: str) -> np.ndarray:
    """Gamma_1 applied per frequency to a field given in Fourier space (Eq. J11).

    (Gamma v)(k) = u(k) [conj(u(k)) . v(k)] / |u(k)|^2 on active frequencies, 0 elsewhere.
    """
    shape = vhat.shape[1:]
    u, active = symbol_vectors(shape, green)
    norm2 = np.where(active, np.sum(np.abs(u) ** 2, axis=0), 1.0)
    proj = np.sum(np.conj(u) * vhat, axis=0) / norm2
    out = u * proj[None]
    out[:, ~active] = 0.0
    return out


def gamma_symbol_matrices(shape, green: str) -> np.ndarray:
    """Gamma(k) as explicit d x d matrices, array of shape (*shape, d, d)."""
    u, active = symbol_vectors(shape, green)
    d = len(shape)
    norm2 = np.where(active, np.sum(np.abs(u) ** 2, axis=0), 1.0)
    G = np.zeros(tuple(shape) + (d, d), dtype=np.complex128)
    for a in range(d):
        for b in range(d):
            G[..., a, b] = np.where(active, u[a] * np.conj(u[b]) / norm2, 0.0)
    return G


def gamma_real_space_kernel(shape, green: str) -> np.ndarray:
    """Convolution kernel g_ab(x) of Gamma_1 in real space: (Gamma v)_a(x) =
    sum_y sum_b g_ab(x - y) v_b(y).  Shape (d, d, *shape)."""
    G = gamma_symbol_matrices(shape, green)
    d = len(shape)
    g = np.zeros((d, d) + tuple(shape), dtype=np.complex128)
    for a in range(d):
        for b in range(d):
            g[a, b] = np.fft.ifftn(G[..., a, b])
    return g
