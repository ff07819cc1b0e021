"""Pins of the oracle's frequency-domain Wiener filter (``oracle.wiener_deconv``):
a plain DFT written out with explicit complex exponentials on tiny images,
the identity PSF, a pure shift (fixes the PSF's centring and the sign of the
exponent), blur-then-deconvolve recovery, and transposition."""
import cmath

import numpy as np
import pytest

import oracle


def _dft2(x, sign):
    H, W = x.shape
    out = np.zeros((H, W), dtype=complex)
    for u in range(H):
        for v in range(W):
            acc = 0j
            for y in range(H):
                for xx in range(W):
                    acc += x[y, xx] * cmath.exp(sign * 2j * cmath.pi * (u * y / H + v * xx / W))
            out[u, v] = acc
    return out


def _circ_conv(g, psf):
    """g blurred by the PSF with wrap-around (the tap at the PSF's centre
    weighs the pixel itself)."""
    H, W = g.shape
    kh, kw = psf.shape
    out = np.zeros((H, W))
    for i in range(kh):
        for j in range(kw):
            out += psf[i, j] * np.roll(np.roll(g.astype(np.float64), i - kh // 2, axis=0), j - kw // 2, axis=1)
    return out


@pytest.mark.parametrize("H,W", [(3, 5), (4, 4), (2, 7), (5, 1)])
def test_deconv_against_explicit_dft(H, W):
    rng = np.random.default_rng(H * 10 + W)
    g = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    psf = rng.random((3, 3))
    psf /= psf.sum()
    nsr = 0.05
    Pm = np.zeros((H, W))
    for i in range(3):
        for j in range(3):
            Pm[(i - 1) % H, (j - 1) % W] += psf[i, j]
    P = _dft2(Pm, -1)
    G = _dft2(g.astype(float), -1)
    y = np.real(_dft2(np.conj(P) / (np.abs(P) ** 2 + nsr) * G, +1)) / (H * W)
    out, y_or = oracle.wiener_deconv(g, psf, nsr)
    np.testing.assert_allclose(y_or, y, rtol=1e-10, atol=1e-9)
    np.testing.assert_array_equal(out, np.clip(np.floor(y + 0.5), 0, 255).astype(np.uint8))


@pytest.mark.parametrize("nsr", [0.0, 0.25, 3.0])
def test_deconv_identity_psf(nsr):
    rng = np.random.default_rng(1)
    g = rng.integers(0, 4096, size=(12, 17)).astype(np.uint16)
    _, y = oracle.wiener_deconv(g, np.ones((1, 1)), nsr, bits=12)
    np.testing.assert_allclose(y, g / (1.0 + nsr), rtol=1e-12, atol=1e-9)


def test_deconv_shift_fixes_centre_and_sign():
    # a PSF whose only tap sits one column right of the centre shifts the image
    # one column right (circularly); deconvolving undoes it
    rng = np.random.default_rng(2)
    g = rng.integers(0, 256, size=(9, 11)).astype(np.uint8)
    psf = np.zeros((3, 3))
    psf[1, 2] = 1.0
    blurred = _circ_conv(g, psf)
    np.testing.assert_array_equal(blurred, np.roll(g.astype(float), 1, axis=1))   # blurred[x] = g[x - 1]
    out, y = oracle.wiener_deconv(np.rint(blurred).astype(np.uint8), psf, 0.0)
    np.testing.assert_allclose(y, g, atol=1e-9)
    np.testing.assert_array_equal(out, g)


def test_deconv_recovers_a_blur():
    rng = np.random.default_rng(3)
    g = rng.integers(0, 4096, size=(16, 21)).astype(np.uint16)
    psf = np.array([[0.05, 0.05, 0.0], [0.1, 0.6, 0.05], [0.05, 0.1, 0.0]])   # |P| >= 0.2: no zeros
    blurred = _circ_conv(g, psf)
    P = oracle.psf_transfer(psf, 16, 21)
    assert np.min(np.abs(P)) >= 0.2 - 1e-12
    y = np.real(np.fft.ifft2(np.conj(P) / np.abs(P) ** 2 * np.fft.fft2(blurred)))
    np.testing.assert_allclose(y, g, atol=1e-8)
    # the oracle on an integer blur: within the rounding of the blur, amplified by 1/min|P|
    out, y2 = oracle.wiener_deconv(np.rint(blurred).astype(np.uint16), psf, 0.0, bits=12)
    assert np.max(np.abs(y2 - g)) <= 0.5 / 0.2 + 1e-9


def test_deconv_transpose_symmetry():
    rng = np.random.default_rng(4)
    g = rng.integers(0, 256, size=(10, 13)).astype(np.uint8)
    psf = rng.random((3, 5))
    a = oracle.wiener_deconv(g, psf, 0.1)[1]
    b = oracle.wiener_deconv(np.ascontiguousarray(g.T), np.ascontiguousarray(psf.T), 0.1)[1]
    np.testing.assert_allclose(a, b.T, rtol=1e-12, atol=1e-9)
