"""Pins for the oracle's Fourier pieces: numpy FFT against a brute-force DFT,
and the Green projection Gamma_1 (Eq. J11) against its defining properties."""
import numpy as np
import pytest

from oracle import fourier as F


@pytest.mark.parametrize("shape", [(4, 6), (5, 3), (2, 3, 4), (3, 3, 2)])
def test_fft_matches_brute_force_dft(shape):
    rng = np.random.default_rng(1)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    field = f[None]
    np.testing.assert_allclose(F.fft(field)[0], F.brute_force_dft(f), atol=1e-12)
    np.testing.assert_allclose(F.ifft(field)[0], F.brute_force_dft(f, inverse=True), atol=1e-12)


def test_integer_freqs_order():
    assert list(F.integer_freqs(8)) == [0, 1, 2, 3, -4, -3, -2, -1]
    assert list(F.integer_freqs(5)) == [0, 1, 2, -2, -1]


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (7, 5), (4, 6, 8), (5, 5, 5)])
def test_gamma_is_orthogonal_projection(green, shape):
    G = F.gamma_symbol_matrices(shape, green)
    GG = G @ G
    np.testing.assert_allclose(GG, G, atol=1e-13)                          # idempotent
    np.testing.assert_allclose(G, np.conj(np.swapaxes(G, -1, -2)), atol=1e-14)  # Hermitian
    zero = (0,) * len(shape)
    assert np.all(G[zero] == 0)                                          # Gamma(0) = 0
    _, active = F.symbol_vectors(shape, green)
    tr = np.trace(G, axis1=-2, axis2=-1)
    np.testing.assert_allclose(tr[active], 1.0, atol=1e-13)               # rank one where active
    np.testing.assert_allclose(tr[~active], 0.0, atol=0)


@pytest.mark.parametrize("green", F.GREENS)
@pytest.mark.parametrize("shape", [(8, 8), (4, 6, 8)])
def test_gamma_range_is_gradients_and_complement_is_divergence_free(green, shape):
    """Gamma v lies along u(k) (a gradient: curl-free) and (I - Gamma) v is
    orthogonal to u(k) (divergence-free), for the symbol's own difference operator."""
    d = len(shape)
    rng = np.random.default_rng(2)
    v = rng.standard_normal((d,) + shape) + 1j * rng.standard_normal((d,) + shape)
    gv = F.apply_gamma(v, green)
    u, active = F.symbol_vectors(shape, green)
    for a in range(d):
        for b in range(d):
            curl = u[a] * gv[b] - u[b] * gv[a]
            assert np.abs(curl).max() < 1e-12
    div = np.sum(np.conj(u) * (v - gv), axis=0)
    assert np.abs(div[active]).max() < 1e-12


def test_trig_symbol_is_kk_over_k2_and_zero_on_nyquist():
    shape = (8, 6)
    G = F.gamma_symbol_matrices(shape, "trig")
    ky, kx = 3, 2                                  # array index (y, x)
    k = np.array([kx, ky], dtype=float)
    np.testing.assert_allclose(G[ky, kx], np.outer(k, k) / k.dot(k), atol=1e-15)
    assert np.all(G[4, :] == 0)                    # k_y = -4 is the Nyquist index of n_y = 8
    assert np.all(G[:, 3] == 0)                    # k_x = -3 is the Nyquist index of n_x = 6


def test_fd_symbol_matches_forward_difference_gradient():
    """Gamma_fd of a forward-difference gradient field returns it unchanged."""
    shape = (6, 8)
    rng = np.random.default_rng(3)
    phi = rng.standard_normal(shape)
    gx = np.roll(phi, -1, axis=1) - phi
    gy = np.roll(phi, -1, axis=0) - phi
    g = np.stack([gx, gy]).astype(np.complex128)
    out = F.ifft(F.apply_gamma(F.fft(g), "fd"))
    np.testing.assert_allclose(out, g, atol=1e-12)


@pytest.mark.parametrize("green", F.GREENS)
def test_gamma_keeps_real_fields_real(green):
    shape = (8, 8)
    rng = np.random.default_rng(4)
    v = rng.standard_normal((2,) + shape)
    out = F.ifft(F.apply_gamma(F.fft(v), green))
    assert np.abs(out.imag).max() < 1e-13


@pytest.mark.parametrize("green", F.GREENS)
def test_real_space_kernel_is_a_convolution_by_gamma(green):
    shape = (4, 6)
    d = 2
    rng = np.random.default_rng(5)
    v = rng.standard_normal((d,) + shape) + 1j * rng.standard_normal((d,) + shape)
    g = F.gamma_real_space_kernel(shape, green)
    out = np.zeros_like(v)
    for y in range(shape[0]):
        for x in range(shape[1]):
            for yy in range(shape[0]):
                for xx in range(shape[1]):
                    out[:, y, x] += g[:, :, (y - yy) % shape[0], (x - xx) % shape[1]] @ v[:, yy, xx]
    np.testing.assert_allclose(out, F.ifft(F.apply_gamma(F.fft(v), green)), atol=1e-12)
