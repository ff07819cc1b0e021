"""Brute-force restatements used to pin the oracle on tiny inputs.

These are written differently from the C oracle on purpose: borders come from
``numpy.pad(mode="symmetric")`` (a library routine), windows are numpy
slices, order statistics come from ``sorted``, and the Wiener statistics are
exact ``fractions.Fraction`` values from the two-pass variance formula.
"""
from fractions import Fraction

import numpy as np


def amf_brute(g, smax, keep_unresolved=False):
    """Per-pixel adaptive median; returns (f, k_resolved)."""
    g = np.asarray(g)
    H, W = g.shape
    R = smax // 2
    ext = np.pad(g.astype(np.int64), R, mode="symmetric")
    f = np.empty((H, W), dtype=np.int64)
    kk = np.zeros((H, W), dtype=np.int64)
    for y in range(H):
        for x in range(W):
            zxy = int(g[y, x])
            out = None
            for k in range(3, smax + 1, 2):
                r = k // 2
                win = sorted(ext[y + R - r:y + R + r + 1, x + R - r:x + R + r + 1].ravel().tolist())
                zmin, zmax, zmed = win[0], win[-1], win[len(win) // 2]
                if zmin < zmed < zmax:
                    out = zxy if zmin < zxy < zmax else zmed
                    kk[y, x] = k
                    break
                last_med = zmed
            if out is None:
                out = zxy if keep_unresolved else last_med
            f[y, x] = out
    return f, kk


def window_values(f, y, x, w, border_zero=False, wh=None):
    """All samples of the wh x w window (wh rows, default w) around (y, x)
    with the symmetric (or zero) border."""
    f = np.asarray(f).astype(np.int64)
    wh = w if wh is None else wh
    pad = ((wh // 2, wh // 2), (w // 2, w // 2))
    if border_zero:
        ext = np.pad(f, pad, mode="constant", constant_values=0)
    else:
        ext = np.pad(f, pad, mode="symmetric")
    return ext[y:y + wh, x:x + w].ravel().tolist()


def local_stats_exact(f, w, border_zero=False, wh=None):
    """Exact (mean, variance) per pixel as Fractions, two-pass formula, over a
    wh x w window (wh rows, default w)."""
    f = np.asarray(f)
    H, W = f.shape
    n = w * (w if wh is None else wh)
    mu = [[None] * W for _ in range(H)]
    var = [[None] * W for _ in range(H)]
    for y in range(H):
        for x in range(W):
            v = window_values(f, y, x, w, border_zero, wh)
            m = Fraction(sum(v), n)
            mu[y][x] = m
            var[y][x] = sum((Fraction(a) - m) ** 2 for a in v) / n
    return mu, var


def wiener_exact(f, w, noise_var=None, border_zero=False, wh=None):
    """Exact rational Wiener output y and the exact noise variance (window wh
    rows, default w, by w columns)."""
    f = np.asarray(f)
    H, W = f.shape
    mu, var = local_stats_exact(f, w, border_zero, wh)
    if noise_var is None:
        nu2 = sum(var[y][x] for y in range(H) for x in range(W)) / (H * W)
    else:
        nu2 = Fraction(noise_var)
    y_out = np.empty((H, W), dtype=object)
    for y in range(H):
        for x in range(W):
            s2 = var[y][x]
            den = max(s2, nu2)
            if den == 0:
                y_out[y, x] = mu[y][x]
            else:
                y_out[y, x] = mu[y][x] + max(s2 - nu2, 0) / den * (int(f[y, x]) - mu[y][x])
    return y_out, nu2, var


def contrast_brute(x, bits, tol):
    """Contrast stretch from the sorted pixel list: lo and hi are the k-th
    smallest and k-th largest values, k = floor(tol * N); the map is rounded
    half up with exact fractions.  Returns (out, lo, hi)."""
    import math
    x = np.asarray(x)
    vals = sorted(int(v) for v in x.ravel())
    n = len(vals)
    k = math.floor(tol * n)
    lo, hi = vals[k], vals[n - 1 - k]
    if lo == hi:
        return x.astype(np.int64), lo, hi
    maxv = (1 << bits) - 1
    out = np.empty(x.shape, dtype=np.int64)
    for idx, v in np.ndenumerate(x):
        c = min(max(int(v), lo), hi)
        out[idx] = math.floor(Fraction((c - lo) * maxv, hi - lo) + Fraction(1, 2))
    return out, lo, hi
