"""The Wiener filter in the Fourier domain (wiener_deconvolve) against the
oracle's binary64 deconvolution.

Tolerance, from the arithmetic: the GPU runs binary32 transforms (unit
roundoff u = 2^-24) with twiddles rounded from binary64.  A radix-2 transform
of length M has log2 M butterfly stages; Bluestein's method runs two of them
plus two chirp products.  Each stage adds a relative error of about 2u to
the transform's 2-norm, so the rounding error of the output y is about
L * 2u * rms(g) * A in root-mean-square, where L counts the stages of the
forward and inverse row and column passes and A = max |P| / (|P|^2 + nsr)
is the filter's largest gain.  The test allows 6 times that at any pixel
(the largest of ~10^7 Gaussian-like errors stays within 6 sigma), plus
maxv 2^-20 for the final product.  The integer output must equal
round-half-up of y64 except where y64 lies within the tolerance of a tie.
"""
import math

import numpy as np
import pytest

from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ensure_built()
import oracle  # noqa: E402
import paper_2005_05371_gb300 as hd  # noqa: E402
import synth  # noqa: E402

DEV = "cuda:0"


def _stages(N):
    if N & (N - 1) == 0:
        return max(1, int(math.log2(N)))
    M = 1
    while M < 2 * N - 1:
        M <<= 1
    return 2 * int(math.log2(M)) + 2


def gaussian_psf(k, sigma):
    r = np.arange(k) - k // 2
    g = np.exp(-(r[:, None] ** 2 + r[None, :] ** 2) / (2 * sigma * sigma))
    return (g / g.sum()).astype(np.float32)


def _run(g, psf, nsr, bits):
    src = torch.from_numpy(g.view(np.int16) if g.dtype == np.uint16 else g).to(DEV)
    dst = torch.full_like(src, 3)
    y = torch.empty(g.shape, dtype=torch.float32, device=DEV)
    hd.wiener_deconvolve(src, dst, torch.from_numpy(psf).to(DEV), nsr, bits=bits, y_out=y)
    assert hd.hd_get_device_error() == hd.HD_OK
    out = dst.cpu().numpy()
    return (out.view(np.uint16) if g.dtype == np.uint16 else out), y.cpu().numpy()


def _check(g, psf, nsr, bits):
    out, y = _run(g, psf, nsr, bits)
    ref_out, y64 = oracle.wiener_deconv(g, psf.astype(np.float64), nsr, bits=bits)
    H, W = g.shape
    P = oracle.psf_transfer(psf.astype(np.float64), H, W)
    A = float(np.max(np.abs(P) / (np.abs(P) ** 2 + nsr)))
    L = 2 * (_stages(W) + _stages(H))
    rms = float(np.sqrt(np.mean(g.astype(np.float64) ** 2)))
    maxv = (1 << bits) - 1
    tol = 6 * L * 2 * 2.0 ** -24 * rms * A + maxv * 2.0 ** -20
    err = np.abs(y.astype(np.float64) - y64)
    assert err.max() <= tol, (err.max(), tol)
    diff = out != ref_out
    frac = y64 - np.floor(y64)
    inside = (y64 > -0.5 + tol) & (y64 < maxv + 0.5 - tol)
    assert np.all(np.abs(frac[diff & inside] - 0.5) <= tol)
    return err.max(), tol, int(diff.sum())


@pytest.mark.parametrize("H,W", [(64, 64), (100, 75), (1, 17), (17, 1), (512, 768), (37, 4096), (8192, 16)])
def test_fourier_wiener_shapes(H, W):
    rng = np.random.default_rng(H * 7 + W)
    g = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    _check(g, gaussian_psf(5, 1.2), 0.02, 8)


@pytest.mark.parametrize("name", ["paper1620", "stress4096"])
def test_fourier_wiener_workload_images(name):
    spec, _, g = synth.config_image(name)
    psf = gaussian_psf(7, 1.5)
    e, tol, nd = _check(g, psf, 0.01, spec.bits)
    print(f"{name}: max |y - y64| = {e:.3e} (bound {tol:.3e}), {nd} pixels off round(y64)")


def test_fourier_wiener_identity_motion_and_shift():
    rng = np.random.default_rng(5)
    g = rng.integers(0, 4096, size=(120, 90)).astype(np.uint16)
    _check(g, np.ones((1, 1), np.float32), 0.0, 12)                          # identity: y = g
    _check(g, np.full((1, 9), 1 / 9, np.float32), 0.05, 12)                  # motion blur along rows
    shift = np.zeros((3, 3), np.float32)
    shift[1, 2] = 1.0
    _check(g, shift, 0.0, 12)                                                # a circular shift, undone
    _check(g, np.ones((1, 1), np.float32), 1.0, 12)                          # y = g / 2


def test_fourier_wiener_psf_wider_than_the_image():
    rng = np.random.default_rng(6)
    g = rng.integers(0, 256, size=(6, 10)).astype(np.uint8)
    psf = rng.random((9, 13)).astype(np.float32)
    psf /= psf.sum()
    _check(g, psf, 0.1, 8)
