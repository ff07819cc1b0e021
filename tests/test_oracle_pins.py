"""Pins of the CPU oracle against things other than itself (CPU only).

Adaptive median (Algorithm 1, step 6):
  * hand-derived worked examples (tests/golden/amf_worked_examples.json),
  * exhaustive brute force on every binary 3x3 image and random tiny images,
  * reduction to library order-statistic filters (scipy.ndimage, mode
    "reflect" = half-sample symmetric) for every window size,
  * invariants: constant image, isolated impulses, output range.
Wiener (Algorithm 1, step 4d, local-statistics form):
  * exact rational arithmetic (two-pass variance) on small images,
  * closed forms: constant, checkerboard c +- d, linear ramp,
  * limits: nu2 = 0 gives the identity, huge nu2 gives the box mean,
  * library routine scipy.signal.wiener with zero borders,
  * the binary32 twin within maxv * 2^-20 of binary64.
Partitioned median (Algorithm 1, step 6 with `parts` strips):
  * a hand-derived seam example (tests/golden/strips_worked_examples.json),
  * every strip equals the brute-force median of that strip alone,
  * one part is the whole-image median; rows whose Smax window stays inside
    their strip equal the whole-image median rows.
Noise variance from a clean reference (Algorithm 1, step 4d):
  * closed forms: a constant offset c gives c^2, a +-d checkerboard d^2,
  * the exact sum against numpy's int64 sum, and the division's rounding,
  * the largest sum that can occur (every pixel 65535 apart) stays exact.
Contrast stretch (Algorithm 1, step 4e; the rule is a reading, the paper
gives none):
  * hand-derived worked examples (tests/golden/contrast_worked_examples.json),
  * the limits as order statistics of the sorted pixel list, and the map in
    exact fractions, on random tiny images,
  * closed forms: full-range ramp, affine ramps, two levels, constants,
  * invariants: order preserved, at most k pixels beyond each limit, the
    stretched range reaches 0 and maxv.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests._brute import amf_brute, contrast_brute, local_stats_exact, wiener_exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "amf_worked_examples.json")
GOLDEN_CONTRAST = os.path.join(os.path.dirname(__file__), "golden", "contrast_worked_examples.json")
GOLDEN_STRIPS = os.path.join(os.path.dirname(__file__), "golden", "strips_worked_examples.json")


# --------------------------------------------------------------------------- AMF
def test_smax_validation():
    # Algorithm 1, step 6a: Smax must be an odd integer > 1.
    for bad in (-3, 0, 1, 2, 4, 10, 12):
        assert oracle.check_smax(bad) == oracle.ORACLE_ERR_SMAX
        with pytest.raises(oracle.OracleError):
            oracle.amf(np.zeros((4, 4), np.uint8), bad)
    for good in (3, 5, 7, 9, 11, 15):
        assert oracle.check_smax(good) == oracle.ORACLE_OK


def test_amf_golden_worked_examples():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        g = np.array(c["image"], dtype=np.uint8)
        f = oracle.amf(g, c["smax"])
        if "expected" in c:
            np.testing.assert_array_equal(f, np.array(c["expected"]), err_msg=c["name"])
        if "expected_keep_unresolved" in c:
            fk = oracle.amf(g, c["smax"], keep_unresolved=True)
            np.testing.assert_array_equal(fk, np.array(c["expected_keep_unresolved"]))
        if "pixel" in c:
            y, x = c["pixel"]
            assert f[y, x] == c["expected_pixel"], c["name"]
            assert oracle.amf_pixel(g, c["smax"], y, x) == c["expected_pixel"]


@pytest.mark.parametrize("smax", [3, 5])
def test_amf_exhaustive_binary_3x3(smax):
    for code in range(512):
        bits = [(code >> i) & 1 for i in range(9)]
        g = (np.array(bits, dtype=np.uint8).reshape(3, 3) * 200 + 20)
        for keep in (False, True):
            ref, _ = amf_brute(g, smax, keep)
            np.testing.assert_array_equal(oracle.amf(g, smax, keep_unresolved=keep), ref)


def test_amf_exhaustive_ternary_2x3():
    for code in range(3 ** 6):
        vals, c = [], code
        for _ in range(6):
            vals.append(c % 3)
            c //= 3
        g = np.array(vals, dtype=np.uint16).reshape(2, 3) * 1000 + 7
        for smax in (3, 5, 7):
            ref, _ = amf_brute(g, smax)
            np.testing.assert_array_equal(oracle.amf(g, smax), ref)


def test_amf_random_tiny_vs_brute():
    rng = np.random.default_rng(7)
    for trial in range(120):
        H, W = int(rng.integers(1, 10)), int(rng.integers(1, 10))
        levels = int(rng.integers(2, 6))
        smax = int(rng.choice([3, 5, 7, 9, 11]))
        g = rng.integers(0, levels, size=(H, W)).astype(np.uint8) * (250 // (levels - 1))
        if trial % 3 == 0:  # continuous values with impulses
            g = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
            g[rng.random((H, W)) < 0.3] = 255
        keep = bool(trial % 2)
        ref, kref = amf_brute(g, smax, keep)
        f, kk = oracle.amf(g, smax, keep_unresolved=keep, return_k=True)
        np.testing.assert_array_equal(f, ref)
        np.testing.assert_array_equal(kk, kref)


def _amf_by_scipy(g, smax, keep=False):
    """Algorithm 1 step 6 in its whole-image mask form, order statistics from scipy."""
    import scipy.ndimage as ndi
    g = g.astype(np.int64)
    f = g.copy()
    t = np.zeros(g.shape, dtype=bool)
    zmed = None
    for k in range(3, smax + 1, 2):
        zmin = ndi.minimum_filter(g, size=k, mode="reflect")
        zmax = ndi.maximum_filter(g, size=k, mode="reflect")
        zmed = ndi.median_filter(g, size=k, mode="reflect")
        lvl_a = (zmed > zmin) & (zmax > zmed) & ~t
        z_b = (g > zmin) & (zmax > g)
        f[lvl_a & z_b] = g[lvl_a & z_b]
        f[lvl_a & ~z_b] = zmed[lvl_a & ~z_b]
        t |= lvl_a
    if not keep:
        f[~t] = zmed[~t]
    return f


@pytest.mark.parametrize("smax,dtype,density", [(3, np.uint8, 0.3), (5, np.uint8, 0.5),
                                                 (7, np.uint16, 0.6), (11, np.uint16, 0.7)])
def test_amf_matches_library_order_statistics(smax, dtype, density):
    rng = np.random.default_rng(smax)
    maxv = 255 if dtype == np.uint8 else 4095
    g = rng.integers(0, maxv + 1, size=(37, 53)).astype(dtype)
    u = rng.random(g.shape)
    g[u < density / 2] = 0
    g[(u >= density / 2) & (u < density)] = maxv
    # a flat patch forces growth all the way to Smax
    g[5:20, 10:30] = maxv // 3
    for keep in (False, True):
        np.testing.assert_array_equal(oracle.amf(g, smax, keep_unresolved=keep),
                                      _amf_by_scipy(g, smax, keep))


def test_amf_invariants():
    rng = np.random.default_rng(11)
    # constant image passes through unchanged
    for v in (0, 17, 255):
        g = np.full((9, 14), v, np.uint8)
        np.testing.assert_array_equal(oracle.amf(g, 7), g)
    # isolated impulses on a flat background are replaced by the window median
    g = np.full((21, 21), 90, np.uint8)
    g[5, 5], g[15, 9], g[10, 17] = 255, 0, 255
    np.testing.assert_array_equal(oracle.amf(g, 5), np.full_like(g, 90))
    # isolated impulse on a varied background: output equals its 3x3 median
    g = rng.integers(60, 200, size=(15, 15)).astype(np.uint8)
    g[7, 7] = 255
    win = np.sort(g[6:9, 6:9].ravel())
    assert win[4] > win[0]
    assert oracle.amf(g, 3)[7, 7] == win[4]
    # output within [min g, max g]; a pixel strictly inside its 3x3 range with level A
    # holding is unchanged
    g = rng.integers(0, 4096, size=(40, 31)).astype(np.uint16)
    g[rng.random(g.shape) < 0.4] = 4095
    f, kk = oracle.amf(g, 9, return_k=True)
    assert f.min() >= g.min() and f.max() <= g.max()
    import scipy.ndimage as ndi
    lo = ndi.minimum_filter(g, 3, mode="reflect")
    hi = ndi.maximum_filter(g, 3, mode="reflect")
    keep = (kk == 3) & (g > lo) & (g < hi)
    np.testing.assert_array_equal(f[keep], g[keep])


def test_amf_pixel_matches_full():
    rng = np.random.default_rng(3)
    g = rng.integers(0, 4096, size=(33, 29)).astype(np.uint16)
    g[rng.random(g.shape) < 0.45] = 0
    f = oracle.amf(g, 11)
    for _ in range(60):
        y, x = int(rng.integers(0, 33)), int(rng.integers(0, 29))
        assert oracle.amf_pixel(g, 11, y, x) == f[y, x]


# ------------------------------------------------------------------------ Wiener
def _round_half_up_fraction(q: Fraction) -> int:
    return int((q + Fraction(1, 2)).__floor__())


@pytest.mark.parametrize("w", [1, 3, 5])
def test_wiener_exact_rational(w):
    rng = np.random.default_rng(w)
    for H, W in [(1, 1), (1, 7), (6, 1), (5, 8), (9, 6)]:
        f = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
        res = oracle.wiener(f, w)
        y_ex, nu2_ex, var = wiener_exact(f, w)
        # sum of D is n^2 * sum of local variances, exactly
        n = w * w
        assert res.sumD == sum(var[y][x] for y in range(H) for x in range(W)) * n * n
        assert res.nu2 == pytest.approx(float(nu2_ex), rel=4e-16, abs=0)
        # with the binary64 noise variance fed back in exactly, y matches per pixel
        y_ex2, _, _ = wiener_exact(f, w, noise_var=Fraction(res.nu2))
        for y in range(H):
            for x in range(W):
                assert abs(res.y64[y, x] - float(y_ex2[y, x])) <= 1e-9 * max(1.0, abs(float(y_ex2[y, x])))


def test_wiener_noise_variance_is_correctly_converted():
    # nu2 = fl(fl(sumD) / (n^2 H W)); Python's int->float is correctly rounded
    rng = np.random.default_rng(5)
    f = rng.integers(0, 65536, size=(128, 160)).astype(np.uint16)
    res = oracle.wiener(f, 7)
    assert res.sumD > 2 ** 53                  # exercises the rounding of the conversion
    assert res.nu2 == float(res.sumD) / float(49 * 49 * 128 * 160)


def test_wiener_constant_and_limits():
    for w in (3, 5, 7):
        f = np.full((12, 9), 77, np.uint8)
        r = oracle.wiener(f, w)
        assert r.nu2 == 0.0
        np.testing.assert_array_equal(r.out64, f)
        np.testing.assert_array_equal(r.out32, f)
        r = oracle.wiener(f, w, noise_var=5.0)
        np.testing.assert_array_equal(r.out64, f)
    rng = np.random.default_rng(2)
    f = rng.integers(0, 4096, size=(23, 19)).astype(np.uint16)
    # noise variance 0 -> identity
    r = oracle.wiener(f, 5, noise_var=0.0, bits=12)
    np.testing.assert_array_equal(r.out64, f)
    np.testing.assert_array_equal(r.out32, f)
    assert np.max(np.abs(r.y64 - f)) < 1e-9
    # huge noise variance -> box mean, rounded half up (exact integer rounding)
    S1, _ = oracle.wiener_stats(f, 5)
    r = oracle.wiener(f, 5, noise_var=1e30, bits=12)
    expect = (2 * S1.astype(np.int64) + 25) // 50
    np.testing.assert_array_equal(r.out64.astype(np.int64), expect)


@pytest.mark.parametrize("w", [3, 5, 7])
def test_wiener_checkerboard_closed_form(w):
    # c +- d checkerboard: interior windows hold one more cell of the centre's
    # colour, so mu = c +- d/n and sigma2 = d^2 (1 - 1/n^2): D = (n^2 - 1) d^2.
    c, d = 1000, 37
    H = W = 3 * w + 4
    yy, xx = np.mgrid[0:H, 0:W]
    f = np.where((yy + xx) % 2 == 0, c + d, c - d).astype(np.uint16)
    S1, D = oracle.wiener_stats(f, w)
    n = w * w
    r = w // 2
    inner = (slice(r, H - r), slice(r, W - r))
    np.testing.assert_array_equal(D[inner], np.full_like(D[inner], (n * n - 1) * d * d))
    centre_sign = np.where((yy + xx) % 2 == 0, 1, -1)[inner]
    np.testing.assert_array_equal(S1[inner].astype(np.int64), n * c + centre_sign * d)


@pytest.mark.parametrize("w", [3, 5])
def test_wiener_ramp_closed_form(w):
    # f = a*x + b: every interior window has variance a^2 r(r+1)/3
    a, b = 7, 11
    H, W = 9, 20
    f = (a * np.arange(W)[None, :] + b + np.zeros((H, 1), np.int64)).astype(np.uint16)
    S1, D = oracle.wiener_stats(f, w)
    n, r = w * w, w // 2
    inner = (slice(r, H - r), slice(r, W - r))
    assert np.all(D[inner] == n * n * a * a * r * (r + 1) // 3)
    assert np.all(S1[inner] == n * f[inner])


def test_wiener_matches_scipy_with_zero_border():
    from scipy.signal import wiener as scipy_wiener
    rng = np.random.default_rng(9)
    for w in (3, 5, 7):
        f = rng.integers(0, 256, size=(31, 44)).astype(np.uint8)
        r = oracle.wiener(f, w, border_zero=True)
        ref = scipy_wiener(f.astype(np.float64), mysize=w)
        np.testing.assert_allclose(r.y64, ref, rtol=1e-9, atol=1e-9)


# ---- rectangular windows: wh rows by ww columns
RECT = [(1, 3), (3, 1), (3, 5), (5, 3), (1, 7), (7, 3), (5, 9)]


@pytest.mark.parametrize("wh,ww", RECT)
def test_wiener_rect_exact_rational(wh, ww):
    rng = np.random.default_rng(wh * 100 + ww)
    for H, W in [(1, 1), (2, 9), (7, 2), (6, 8)]:
        f = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
        res = oracle.wiener(f, ww, wh=wh)
        y_ex, nu2_ex, var = wiener_exact(f, ww, wh=wh)
        n = wh * ww
        assert res.sumD == sum(var[y][x] for y in range(H) for x in range(W)) * n * n
        assert res.nu2 == pytest.approx(float(nu2_ex), rel=4e-16, abs=0)
        y_ex2, _, _ = wiener_exact(f, ww, noise_var=Fraction(res.nu2), wh=wh)
        for y in range(H):
            for x in range(W):
                assert abs(res.y64[y, x] - float(y_ex2[y, x])) <= 1e-9 * max(1.0, abs(float(y_ex2[y, x])))


@pytest.mark.parametrize("wh,ww", RECT)
def test_wiener_rect_checkerboard_closed_form(wh, ww):
    # n = wh * ww is odd: interior windows hold one more cell of the colour of
    # their corners (the centre's when ry + rx is even), so D = (n^2 - 1) d^2
    # and S1 = n c +- d
    c, d = 900, 23
    H, W = 2 * wh + 5, 2 * ww + 6
    yy, xx = np.mgrid[0:H, 0:W]
    f = np.where((yy + xx) % 2 == 0, c + d, c - d).astype(np.uint16)
    S1, D = oracle.wiener_stats(f, ww, wh=wh)
    n = wh * ww
    inner = (slice(wh // 2, H - wh // 2), slice(ww // 2, W - ww // 2))
    np.testing.assert_array_equal(D[inner], np.full_like(D[inner], (n * n - 1) * d * d))
    corner = -1 if (wh // 2 + ww // 2) % 2 else 1
    sign = corner * np.where((yy + xx) % 2 == 0, 1, -1)[inner]
    np.testing.assert_array_equal(S1[inner].astype(np.int64), n * c + sign * d)


@pytest.mark.parametrize("wh,ww", [(3, 5), (5, 3), (1, 7), (7, 1)])
def test_wiener_rect_ramps_fix_the_axes(wh, ww):
    # a ramp along x varies only across the window's ww columns, a ramp along y
    # only across its wh rows: variance a^2 r (r + 1) / 3 with r the radius of
    # that axis (swapping the axes fails these)
    a, b = 5, 40
    H, W = 15, 17
    n = wh * ww
    fx = (a * np.arange(W)[None, :] + b + np.zeros((H, 1), np.int64)).astype(np.uint16)
    S1, D = oracle.wiener_stats(fx, ww, wh=wh)
    rx, ry = ww // 2, wh // 2
    inner = (slice(ry, H - ry), slice(rx, W - rx))
    assert np.all(D[inner] == n * n * a * a * rx * (rx + 1) // 3)
    assert np.all(S1[inner] == n * fx[inner])
    fy = (a * np.arange(H)[:, None] + b + np.zeros((1, W), np.int64)).astype(np.uint16)
    S1, D = oracle.wiener_stats(fy, ww, wh=wh)
    assert np.all(D[inner] == n * n * a * a * ry * (ry + 1) // 3)
    assert np.all(S1[inner] == n * fy[inner])


def test_wiener_rect_matches_scipy_with_zero_border():
    from scipy.signal import wiener as scipy_wiener
    rng = np.random.default_rng(19)
    for wh, ww in [(3, 5), (5, 3), (1, 5), (7, 3)]:
        f = rng.integers(0, 256, size=(29, 41)).astype(np.uint8)
        r = oracle.wiener(f, ww, border_zero=True, wh=wh)
        ref = scipy_wiener(f.astype(np.float64), mysize=(wh, ww))
        np.testing.assert_allclose(r.y64, ref, rtol=1e-9, atol=1e-9)


def test_wiener_rect_transpose_symmetry():
    rng = np.random.default_rng(23)
    f = rng.integers(0, 4096, size=(33, 21)).astype(np.uint16)
    a = oracle.wiener(f, 7, bits=12, wh=3)
    b = oracle.wiener(np.ascontiguousarray(f.T), 3, bits=12, wh=7)
    np.testing.assert_array_equal(a.out64, b.out64.T)
    np.testing.assert_array_equal(a.y64, b.y64.T)
    assert a.sumD == b.sumD and a.nu2 == b.nu2
    # wh = ww is the square window
    np.testing.assert_array_equal(oracle.wiener(f, 5, bits=12, wh=5).y32, oracle.wiener(f, 5, bits=12).y32)


@pytest.mark.parametrize("bits,w", [(8, 3), (8, 7), (12, 5), (12, 7), (16, 3), (16, 7)])
def test_wiener_binary32_twin_error_bound(bits, w):
    rng = np.random.default_rng(bits * 10 + w)
    maxv = (1 << bits) - 1
    dtype = np.uint8 if bits == 8 else np.uint16
    base = rng.integers(0, maxv + 1, size=(60, 70))
    smooth = (base + np.roll(base, 1, 0) + np.roll(base, 1, 1)) // 3
    f = np.where(rng.random((60, 70)) < 0.5, base, smooth).astype(dtype)
    r = oracle.wiener(f, w, bits=bits)
    bound = maxv * 2.0 ** -20
    assert np.max(np.abs(r.y32.astype(np.float64) - r.y64)) <= bound
    # integer outputs agree except where binary64 sits within the bound of a tie
    diff = r.out32.astype(np.int64) != r.out64.astype(np.int64)
    frac = r.y64 - np.floor(r.y64)
    assert np.all(np.abs(frac[diff] - 0.5) <= bound)
    assert np.all(np.abs(r.out64.astype(np.float64) - r.y64) <= 0.5 + 1e-12)


def test_wiener_output_within_local_range():
    rng = np.random.default_rng(4)
    f = rng.integers(0, 4096, size=(25, 30)).astype(np.uint16)
    import scipy.ndimage as ndi
    for w in (3, 5):
        r = oracle.wiener(f, w, bits=12)
        lo = ndi.minimum_filter(f, w, mode="reflect")
        hi = ndi.maximum_filter(f, w, mode="reflect")
        assert np.all(r.out64 >= lo) and np.all(r.out64 <= hi)
        # y lies between mu and f
        S1, _ = oracle.wiener_stats(f, w)
        mu = S1 / (w * w)
        assert np.all((r.y64 - mu) * (f - mu) >= -1e-9)
        assert np.all(np.abs(r.y64 - mu) <= np.abs(f - mu) + 1e-9)


def test_hybrid_is_wiener_of_amf():
    rng = np.random.default_rng(8)
    g = rng.integers(0, 256, size=(20, 24)).astype(np.uint8)
    g[rng.random(g.shape) < 0.2] = 255
    f, r = oracle.hybrid(g, 7, 3)
    np.testing.assert_array_equal(f, oracle.amf(g, 7))
    r2 = oracle.wiener(f, 3)
    np.testing.assert_array_equal(r.out64, r2.out64)


# --------------------------------------------------------------------------- partitioned median
def test_strips_golden_worked_examples():
    for c in json.load(open(GOLDEN_STRIPS))["cases"]:
        g = np.array(c["image"], dtype=np.uint8)
        assert oracle.strip_bounds(g.shape[0], c["parts"]) == c["bounds"], c["name"]
        if "pixel" in c:
            y, x = c["pixel"]
            assert oracle.amf(g, c["smax"])[y, x] == c["whole_image"]
            assert oracle.amf_strips(g, c["smax"], c["parts"])[y, x] == c["strips"]


@pytest.mark.parametrize("seed", range(12))
def test_strips_match_brute_per_strip(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 14)), int(rng.integers(1, 9))
    parts = int(rng.integers(1, H + 1))
    smax = int(rng.choice([3, 5, 7]))
    g = rng.integers(0, 4, size=(H, W)).astype(np.uint8) * 60
    f = oracle.amf_strips(g, smax, parts)
    b = [(i * H) // parts for i in range(parts + 1)]
    for i in range(parts):
        want, _ = amf_brute(g[b[i]:b[i + 1]], smax)
        np.testing.assert_array_equal(f[b[i]:b[i + 1]], want)


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_strips_locality(parts):
    g = np.random.default_rng(parts).integers(0, 256, size=(64, 40)).astype(np.uint8)
    smax = 7
    f = oracle.amf_strips(g, smax, parts)
    whole = oracle.amf(g, smax)
    if parts == 1:
        np.testing.assert_array_equal(f, whole)
        _, r1 = oracle.hybrid_strips(g, smax, 5, 1)
        _, r2 = oracle.hybrid(g, smax, 5)
        np.testing.assert_array_equal(r1.out32, r2.out32)
    b = oracle.strip_bounds(64, parts)
    inner = [y for y in range(64) if all(abs(y - s) >= smax // 2 and abs(y - (s - 1)) >= smax // 2
                                         for s in b[1:-1])]
    np.testing.assert_array_equal(f[inner], whole[inner])
    if parts > 1:
        assert (f != whole).any()          # the seams do change some pixels


# --------------------------------------------------------------------------- reference noise variance
def test_reference_noise_variance_closed_forms():
    rng = np.random.default_rng(3)
    r = rng.integers(0, 200, size=(37, 53)).astype(np.uint8)
    for c in (0, 1, 7, 55):
        nu2, tot = oracle.reference_noise_variance((r + c).astype(np.uint8), r)
        assert nu2 == float(c * c) and tot == c * c * r.size
    d = 9
    sign = np.where((np.indices(r.shape).sum(axis=0) % 2) == 0, 1, -1)
    f = (r.astype(np.int64) + 20 + d * sign).astype(np.uint8)
    nu2, _ = oracle.reference_noise_variance(f, (r + 20).astype(np.uint8))
    assert nu2 == float(d * d)


def test_reference_noise_variance_exact_sum_and_rounding():
    rng = np.random.default_rng(4)
    for shape, hi in (((1, 1), 256), ((7, 9), 4096), ((300, 301), 65536)):
        f = rng.integers(0, hi, size=shape).astype(np.uint16)
        r = rng.integers(0, hi, size=shape).astype(np.uint16)
        nu2, tot = oracle.reference_noise_variance(f, r)
        want = int(((f.astype(np.int64) - r.astype(np.int64)) ** 2).sum())
        assert tot == want
        q = Fraction(want) if want < 2 ** 53 else Fraction(float(want))
        assert nu2 == float(q / f.size)          # fl(fl(sum) / N)
    # the largest possible sum: 65535^2 a pixel over many pixels stays exact
    f = np.full((1000, 1000), 65535, np.uint16)
    nu2, tot = oracle.reference_noise_variance(f, np.zeros_like(f))
    assert tot == 65535 ** 2 * 10 ** 6 and nu2 == float(65535 ** 2)


# --------------------------------------------------------------------------- contrast stretch
def test_contrast_golden_worked_examples():
    for c in json.load(open(GOLDEN_CONTRAST))["cases"]:
        dt = np.uint8 if c["bits"] == 8 else np.uint16
        x = np.array(c["image"], dtype=dt)
        out, lo, hi = oracle.contrast(x, c["tol"], bits=c["bits"])
        assert (lo, hi) == (c["lo"], c["hi"]), c["name"]
        np.testing.assert_array_equal(out, np.array(c["expected"]), err_msg=c["name"])


@pytest.mark.parametrize("seed", range(40))
def test_contrast_matches_sorted_brute(seed):
    rng = np.random.default_rng(seed)
    bits = int(rng.choice([3, 8, 10, 12, 16]))
    dt = np.uint8 if bits <= 8 and rng.random() < 0.5 else np.uint16
    H, W = int(rng.integers(1, 9)), int(rng.integers(1, 9))
    levels = int(rng.integers(1, 6)) if rng.random() < 0.4 else (1 << bits)
    x = (rng.integers(0, levels, size=(H, W)) * ((1 << bits) // max(levels, 1))).clip(0, (1 << bits) - 1)
    x = x.astype(dt)
    tol = float(rng.choice([0.0, 0.01, 0.1, 0.2, 0.25, 1 / 3, 0.49]))
    out, lo, hi = oracle.contrast(x, tol, bits=bits)
    ref, rlo, rhi = contrast_brute(x, bits, tol)
    assert (lo, hi) == (rlo, rhi)
    np.testing.assert_array_equal(out.astype(np.int64), ref)


@pytest.mark.parametrize("bits", [8, 12, 16])
def test_contrast_closed_forms(bits):
    maxv = (1 << bits) - 1
    dt = np.uint8 if bits == 8 else np.uint16
    # the full-range ramp is already stretched: identity for tol = 0
    ramp = np.arange(maxv + 1, dtype=np.int64).astype(dt).reshape(1, -1)
    np.testing.assert_array_equal(oracle.contrast(ramp, 0.0, bits=bits)[0], ramp)
    # an affine ramp a + b r, r = 0..m, maps to round-half-up(r maxv / m)
    for a, b, m in ((3, 2, 50), (100, 1, 7), (0, 5, 1)):
        r = np.arange(m + 1)
        x = (a + b * r).astype(dt).reshape(1, -1)
        want = (2 * r * maxv + m) // (2 * m)
        out, lo, hi = oracle.contrast(x, 0.0, bits=bits)
        assert (lo, hi) == (a, a + b * m)
        np.testing.assert_array_equal(out.astype(np.int64).ravel(), want)
    # two levels go to the two ends; constants and single pixels stay
    two = np.array([[9, 40, 40, 9, 9]], dtype=dt)
    np.testing.assert_array_equal(oracle.contrast(two, 0.0, bits=bits)[0], [[0, maxv, maxv, 0, 0]])
    for v in (0, 1, maxv):
        c = np.full((3, 4), v, dtype=dt)
        np.testing.assert_array_equal(oracle.contrast(c, 0.3, bits=bits)[0], c)
        np.testing.assert_array_equal(oracle.contrast(c[:1, :1], 0.0, bits=bits)[0], c[:1, :1])


@pytest.mark.parametrize("tol", [0.0, 0.01, 0.05, 0.3])
def test_contrast_invariants(tol):
    rng = np.random.default_rng(11)
    for bits, dt in ((8, np.uint8), (12, np.uint16)):
        maxv = (1 << bits) - 1
        x = np.clip(rng.normal(maxv * 0.4, maxv * 0.1, size=(37, 53)), 0, maxv).astype(dt)
        out, lo, hi = oracle.contrast(x, tol, bits=bits)
        k = int(np.floor(tol * x.size))
        assert (x < lo).sum() <= k and (x > hi).sum() <= k
        assert (x <= lo).sum() >= k + 1 and (x >= hi).sum() >= k + 1
        assert lo < hi and out.min() == 0 and out.max() == maxv
        order = np.argsort(x.ravel(), kind="stable")
        assert (np.diff(out.ravel()[order].astype(np.int64)) >= 0).all()   # order preserved
        assert (out[x <= lo] == 0).all() and (out[x >= hi] == maxv).all()


def test_contrast_rejects_bad_arguments():
    x = np.zeros((2, 2), np.uint8)
    for tol in (-0.1, 0.5, 0.7, float("nan")):
        with pytest.raises(oracle.OracleError):
            oracle.contrast(x, tol)
    with pytest.raises(oracle.OracleError):
        oracle.contrast(np.array([[5000]], np.uint16), 0.0, bits=12)     # above 2^bits - 1
