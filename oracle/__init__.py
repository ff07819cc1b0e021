"""CPU oracle of the hybrid denoiser (adaptive median -> local-statistics Wiener).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg are the only callers.  The CUDA
library never imports this package and shares no code with it.

The arithmetic lives in ``hd_oracle.c`` (plain C, compiled with gcc, binary64
unless stated); this module compiles it on first use and wraps it with numpy.
What each function follows in the paper:

* ``amf``          - Algorithm 1, step 6 (adaptive median, level A / level B,
                     window growth k = 3..Smax over the noisy image).
* ``wiener``       - Algorithm 1, step 4d, in the spatial local-statistics
                     form (local mean / variance over a wh x w window, square
                     by default; noise variance = mean local variance unless
                     supplied).
* ``hybrid``       - Algorithm 1, step 4: Wiener(AMF(g)).  The contrast
                     stretch of step 4e is the separate ``contrast``.
* ``amf_strips`` / ``hybrid_strips`` - Algorithm 1, step 6 as the listing
                     partitions it: the image is cut into ``parts`` row strips
                     (rows floor(i H / parts) .. floor((i+1) H / parts) - 1)
                     and each strip is median-filtered alone, its borders
                     reflected at the strip's own edges; the Wiener filter then
                     runs on the whole reassembled image.
* ``reference_noise_variance`` - Algorithm 1, step 4d with the original
                     image passed to the Wiener stage: nu2 = mean (f - ref)^2.
* ``wiener_deconv`` - the Wiener filter as Section IV places it, in the
                     Fourier domain: deconvolution by a point-spread function
                     with a noise-to-signal ratio (both the caller's; the
                     paper gives neither), circular boundary, binary64.
* ``contrast``     - Algorithm 1, step 4e (the paper gives no rule): linear
                     stretch between the k-th smallest and k-th largest
                     values, k = floor(tol * N), exact integer rounding.

Pins: every function here is checked, in ``tests/test_oracle_pins.py``,
against brute force on tiny images, library order-statistic filters,
closed forms and exact rational arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORACLE_OK = 0
ORACLE_ERR_ARG = 1
ORACLE_ERR_SMAX = 2
ORACLE_ERR_WINDOW = 3
ORACLE_ERR_OOM = 5


def build(force: bool = False) -> str:
    """Compile hd_oracle.c into liboracle.so next to it (gcc, -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["cc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            L = ctypes.c_long
            I = ctypes.c_int
            lib.oracle_amf.argtypes = [P, P, L, L, I, I, P]
            lib.oracle_amf.restype = I
            lib.oracle_wiener.argtypes = [P, L, L, I, I, ctypes.c_double, I, P, P, P, P, P, P]
            lib.oracle_wiener.restype = I
            lib.oracle_wiener_rect.argtypes = [P, L, L, I, I, I, ctypes.c_double, I, P, P, P, P, P, P]
            lib.oracle_wiener_rect.restype = I
            lib.oracle_wiener_stats.argtypes = [P, L, L, I, I, I, P, P]
            lib.oracle_wiener_stats.restype = I
            lib.oracle_amf_pixel.argtypes = [P, L, L, I, I, L, L]
            lib.oracle_amf_pixel.restype = I
            lib.oracle_reference_noise_var.argtypes = [P, P, L, P, P]
            lib.oracle_reference_noise_var.restype = I
            lib.oracle_contrast.argtypes = [P, L, I, ctypes.c_double, P, P]
            lib.oracle_contrast.restype = I
            lib.oracle_check_smax.argtypes = [I]
            lib.oracle_check_smax.restype = I
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def _as_u16(img: np.ndarray) -> np.ndarray:
    if img.ndim != 2:
        raise ValueError("image must be 2-D")
    if img.dtype not in (np.uint8, np.uint16):
        raise TypeError("image must be uint8 or uint16")
    return np.ascontiguousarray(img, dtype=np.uint16)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def check_smax(smax: int) -> int:
    """Algorithm 1, step 6a: status 0 if Smax is an odd integer > 1, else 2."""
    return _load().oracle_check_smax(int(smax))


def amf(g: np.ndarray, smax: int, keep_unresolved: bool = False, return_k: bool = False):
    """Adaptive median filter of the noisy image ``g`` (Algorithm 1, step 6).

    Returns the filtered image with ``g``'s dtype (and, with ``return_k``, the
    window size at which each pixel passed level A, 0 where none did).
    """
    lib = _load()
    g16 = _as_u16(g)
    H, W = g16.shape
    f = np.empty_like(g16)
    kk = np.empty((H, W), dtype=np.uint8) if return_k else None
    rc = lib.oracle_amf(_ptr(g16), _ptr(f), H, W, int(smax), int(bool(keep_unresolved)), _ptr(kk))
    if rc != ORACLE_OK:
        raise OracleError(rc, "oracle_amf")
    out = f.astype(g.dtype)
    return (out, kk) if return_k else out


def amf_pixel(g: np.ndarray, smax: int, y: int, x: int, keep_unresolved: bool = False) -> int:
    """Adaptive median of one pixel (for sampled checks of large images)."""
    lib = _load()
    g16 = g if (g.dtype == np.uint16 and g.flags.c_contiguous) else _as_u16(g)
    H, W = g16.shape
    v = lib.oracle_amf_pixel(_ptr(g16), H, W, int(smax), int(bool(keep_unresolved)), int(y), int(x))
    if v < 0:
        raise OracleError(ORACLE_ERR_ARG, "oracle_amf_pixel")
    return v


@dataclass
class WienerResult:
    out64: np.ndarray      # round-half-up of y64, input dtype
    y64: np.ndarray        # binary64 value (the paper's precision)
    out32: np.ndarray      # rounding of the binary32 twin, input dtype
    y32: np.ndarray        # binary32 twin in the kernel's evaluation order
    nu2: float             # noise variance used
    sumD: int              # exact sum over pixels of D = n*S2 - S1^2


def wiener(f: np.ndarray, w: int, noise_var: float = -1.0, bits: int | None = None,
           border_zero: bool = False, wh: int | None = None) -> WienerResult:
    """Local-statistics Wiener filter of the integer image ``f`` over a window
    of ``wh`` rows (default ``w``: square) by ``w`` columns.

    ``noise_var < 0`` estimates the noise variance as the mean local variance.
    ``bits`` sets the output clamp 2^bits - 1 (default: 8 for uint8, 16 for uint16).
    """
    lib = _load()
    f16 = _as_u16(f)
    H, W = f16.shape
    if bits is None:
        bits = 8 if f.dtype == np.uint8 else 16
    maxv = (1 << int(bits)) - 1
    out64 = np.empty_like(f16)
    out32 = np.empty_like(f16)
    y64 = np.empty((H, W), dtype=np.float64)
    y32 = np.empty((H, W), dtype=np.float32)
    nu2 = ctypes.c_double()
    sumD = np.zeros(2, dtype=np.uint64)
    rc = lib.oracle_wiener_rect(_ptr(f16), H, W, int(w if wh is None else wh), int(w), int(bool(border_zero)),
                                float(noise_var), maxv, _ptr(out64), _ptr(y64), _ptr(out32), _ptr(y32),
                                ctypes.byref(nu2), _ptr(sumD))
    if rc != ORACLE_OK:
        raise OracleError(rc, "oracle_wiener")
    total = int(sumD[0]) + (int(sumD[1]) << 64)
    return WienerResult(out64.astype(f.dtype), y64, out32.astype(f.dtype), y32, nu2.value, total)


def wiener_stats(f: np.ndarray, w: int, border_zero: bool = False, wh: int | None = None):
    """(S1, D) per pixel as uint64 arrays, D = n*S2 - S1^2, over ``wh`` rows
    (default ``w``) by ``w`` columns, n = wh * w."""
    lib = _load()
    f16 = _as_u16(f)
    H, W = f16.shape
    S1 = np.empty((H, W), dtype=np.uint64)
    D = np.empty((H, W), dtype=np.uint64)
    rc = lib.oracle_wiener_stats(_ptr(f16), H, W, int(w if wh is None else wh), int(w), int(bool(border_zero)),
                                 _ptr(S1), _ptr(D))
    if rc != ORACLE_OK:
        raise OracleError(rc, "oracle_wiener_stats")
    return S1, D


def hybrid(g: np.ndarray, smax: int, w: int, noise_var: float = -1.0, bits: int | None = None,
           keep_unresolved: bool = False, border_zero: bool = False, wh: int | None = None):
    """Algorithm 1, step 4 without the contrast stretch: Wiener(AMF(g)), the
    Wiener window ``wh`` rows (default ``w``) by ``w`` columns.

    Returns (f, WienerResult) where f is the adaptive-median output.
    """
    f = amf(g, smax, keep_unresolved=keep_unresolved)
    return f, wiener(f, w, noise_var=noise_var, bits=bits, border_zero=border_zero, wh=wh)


def strip_bounds(H: int, parts: int) -> list[int]:
    """Row boundaries of the listing's image partition: strip i covers rows
    [b[i], b[i+1]), b[i] = floor(i * H / parts)."""
    if not (1 <= parts <= H):
        raise ValueError("parts must be in [1, H]")
    return [(i * H) // parts for i in range(parts + 1)]


def amf_strips(g: np.ndarray, smax: int, parts: int, keep_unresolved: bool = False) -> np.ndarray:
    """Adaptive median of each row strip alone (Algorithm 1, step 6, with the
    listing's ``parts`` partitions): windows reflect at each strip's edges."""
    b = strip_bounds(g.shape[0], parts)
    f = np.empty_like(g)
    for i in range(parts):
        f[b[i]:b[i + 1]] = amf(g[b[i]:b[i + 1]], smax, keep_unresolved=keep_unresolved)
    return f


def hybrid_strips(g: np.ndarray, smax: int, w: int, parts: int, noise_var: float = -1.0,
                  bits: int | None = None, keep_unresolved: bool = False, border_zero: bool = False):
    """Algorithm 1, step 4 with a partitioned median: Wiener of the whole image
    assembled from the strips' medians.  Returns (f, WienerResult)."""
    f = amf_strips(g, smax, parts, keep_unresolved=keep_unresolved)
    return f, wiener(f, w, noise_var=noise_var, bits=bits, border_zero=border_zero)


def contrast(x: np.ndarray, tol: float = 0.01, bits: int | None = None):
    """Contrast stretch of an integer image (Algorithm 1, step 4e, read as a
    linear stretch between saturation limits; see ``oracle_contrast``).

    Returns ``(out, lo, hi)``: the stretched image with ``x``'s dtype and the
    two limits.  ``bits`` sets maxv = 2^bits - 1 (default 8 for uint8, 16 for
    uint16)."""
    lib = _load()
    x16 = _as_u16(x)
    if bits is None:
        bits = 8 if x.dtype == np.uint8 else 16
    out = np.empty_like(x16)
    lohi = np.zeros(2, dtype=np.int64)
    rc = lib.oracle_contrast(_ptr(x16), x16.size, int(bits), float(tol), _ptr(out), _ptr(lohi))
    if rc != ORACLE_OK:
        raise OracleError(rc, "oracle_contrast")
    return out.astype(x.dtype), int(lohi[0]), int(lohi[1])


def reference_noise_variance(f: np.ndarray, ref: np.ndarray):
    """Noise variance of ``f`` against a clean reference image (Algorithm 1,
    step 4d, where the original image reaches the Wiener stage): the mean of
    (f - ref)^2 over all pixels, summed exactly, one binary64 division.
    Returns (nu2, exact sum)."""
    lib = _load()
    f16, r16 = _as_u16(f), _as_u16(ref)
    if f16.shape != r16.shape:
        raise ValueError("f and ref must have the same shape")
    nu2 = ctypes.c_double()
    tot = np.zeros(1, dtype=np.uint64)
    rc = lib.oracle_reference_noise_var(_ptr(f16), _ptr(r16), f16.size, ctypes.byref(nu2), _ptr(tot))
    if rc != ORACLE_OK:
        raise OracleError(rc, "oracle_reference_noise_var")
    return nu2.value, int(tot[0])


def psf_transfer(psf: np.ndarray, H: int, W: int) -> np.ndarray:
    """The PSF's transfer function on the H x W frequency grid: the PSF placed
    on an H x W grid with its centre tap (row kh // 2, column kw // 2) at the
    origin and the other taps wrapped around, then its 2-D DFT (binary64)."""
    psf = np.asarray(psf, dtype=np.float64)
    kh, kw = psf.shape
    P = np.zeros((H, W), dtype=np.float64)
    for i in range(kh):
        for j in range(kw):
            P[(i - kh // 2) % H, (j - kw // 2) % W] += psf[i, j]
    return np.fft.fft2(P)


def wiener_deconv(g: np.ndarray, psf: np.ndarray, nsr: float, bits: int | None = None):
    """Frequency-domain Wiener filter (Section IV): with G the 2-D DFT of the
    image and P the PSF's transfer function, the estimate's spectrum is
    F = conj(P) / (|P|^2 + nsr) * G, and the estimate y the real part of the
    inverse DFT of F (the DFT's periodic extension is the border rule).
    out = min(maxv, max(0, floor(y + 1/2))).  Returns (out, y) with y in
    binary64."""
    g = np.asarray(g)
    if bits is None:
        bits = 8 if g.dtype == np.uint8 else 16
    maxv = (1 << int(bits)) - 1
    H, W = g.shape
    P = psf_transfer(psf, H, W)
    G = np.fft.fft2(g.astype(np.float64))
    F = np.conj(P) / (np.abs(P) ** 2 + float(nsr)) * G
    y = np.real(np.fft.ifft2(F))
    out = np.clip(np.floor(y + 0.5), 0, maxv).astype(g.dtype)
    return out, y
