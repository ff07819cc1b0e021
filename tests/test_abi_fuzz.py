"""Seeded fuzz of the C ABI's argument checks (no GPU): for random image
descriptors the status returned before anything is launched must be the one
the header's rules give.  Only descriptors that some rule rejects are sent,
so no call reaches the device."""
import ctypes

import numpy as np
import pytest

import paper_2005_05371_gb300 as hd


def expected(H, W, dtype, bits, smax, w, pitch_s, pitch_d, src, dst, border, unresolved, need_amf, need_wiener):
    """The header's rules, in the order the library applies them (first failure wins)."""
    if dtype not in (hd.HD_U8, hd.HD_U16):
        return hd.HD_ERR_DTYPE
    if dtype == hd.HD_U8 and bits != 8:
        return hd.HD_ERR_DTYPE
    if dtype == hd.HD_U16 and not 1 <= bits <= 16:
        return hd.HD_ERR_DTYPE
    if H < 1 or W < 1:
        return hd.HD_ERR_ARG
    if H > 65535 or W > 65535:
        return hd.HD_ERR_OVERFLOW
    if not src or not dst:
        return hd.HD_ERR_ARG
    es = 1 if dtype == hd.HD_U8 else 2
    row = W * es
    if pitch_s < row or pitch_d < row:
        return hd.HD_ERR_ARG
    if es == 2 and ((pitch_s | pitch_d) & 1 or (src | dst) & 1):
        return hd.HD_ERR_ARG
    s0, s1 = src, src + (H - 1) * pitch_s + row
    d0, d1 = dst, dst + (H - 1) * pitch_d + row
    if s0 < d1 and d0 < s1:
        return hd.HD_ERR_ARG
    if need_amf:
        if smax < 3 or smax > hd.HD_SMAX_MAX or smax % 2 == 0:
            return hd.HD_ERR_SMAX
        if unresolved not in (0, 1):
            return hd.HD_ERR_ARG
    if need_wiener:
        if w < 1 or w > hd.HD_WIENER_W_MAX or w % 2 == 0:
            return hd.HD_ERR_WINDOW
        if border not in (0, 1):
            return hd.HD_ERR_ARG
    return hd.HD_OK


def draw(rng):
    dtype = int(rng.choice([hd.HD_U8, hd.HD_U16, hd.HD_U16, 3]))
    bits = int(rng.choice([8, 8, 12, 16, 0, 17]))
    H = int(rng.choice([0, 1, 7, 300, 65535, 65536]))
    W = int(rng.choice([-1, 1, 9, 640, 65536]))
    es = 2 if dtype == hd.HD_U16 else 1
    row = max(W, 0) * es
    pitch_s = int(rng.choice([row, row + 1, row + 64, max(row - 1, 0)]))
    pitch_d = int(rng.choice([row, row + 2, max(row - 2, 0)]))
    src = int(rng.choice([0, 0x10000000, 0x10000001]))
    dst = int(rng.choice([0, 0x20000000, src + 8]))
    smax = int(rng.choice([1, 2, 3, 9, 15, 17]))
    w = int(rng.choice([0, 1, 4, 5, 15, 17]))
    border = int(rng.choice([0, 1, 2]))
    unresolved = int(rng.choice([0, 1, 5]))
    return dict(H=H, W=W, dtype=dtype, bits=bits, smax=smax, w=w, pitch_s=pitch_s, pitch_d=pitch_d, src=src,
                dst=dst, border=border, unresolved=unresolved)


STATIC_BYTES = 36 * 1024 * 1024


def static_min_bytes(H, W, dtype):
    """hybrid_min_workspace_size with an estimated noise variance: the queue
    counters and control block (one 256-byte-rounded block) and the median plane
    with rows padded to 16 bytes."""
    es = 1 if dtype == hd.HD_U8 else 2
    ctl = -(-(256 + 64) // 256) * 256
    return ctl + -(-(H * (-(-W * es // 16) * 16)) // 256) * 256


@pytest.mark.parametrize("fn", ["amf_filter", "wiener_filter", "hybrid_denoise", "hybrid_denoise_static"])
def test_argument_checks_match_the_rules(fn):
    rng = np.random.default_rng({"amf_filter": 1, "wiener_filter": 2, "hybrid_denoise": 3,
                                 "hybrid_denoise_static": 4}[fn])
    need_amf = fn in ("amf_filter", "hybrid_denoise", "hybrid_denoise_static")
    need_wiener = fn in ("wiener_filter", "hybrid_denoise", "hybrid_denoise_static")
    checked = 0
    for _ in range(4000):
        a = draw(rng)
        want = expected(**a, need_amf=need_amf, need_wiener=need_wiener)
        if want == hd.HD_OK and fn == "hybrid_denoise_static":
            # after the shared checks: the fixed array's size limit
            if static_min_bytes(a["H"], a["W"], a["dtype"]) > STATIC_BYTES:
                want = hd.HD_ERR_OVERFLOW
        if want == hd.HD_OK:
            continue                        # would launch: not sent
        p = hd.hd_params(a["smax"], a["w"], -1.0, a["border"], a["unresolved"], a["bits"])
        img = hd.hd_image(a["src"] or None, a["dst"] or None, a["H"], a["W"], a["pitch_s"], a["pitch_d"], a["dtype"],
                          p, None, None)
        if fn == "amf_filter":
            got = hd._lib.amf_filter(ctypes.byref(img), None)
        elif fn == "hybrid_denoise_static":
            got = hd._lib.hybrid_denoise_static(ctypes.byref(img), None)
        else:
            got = getattr(hd._lib, fn)(ctypes.byref(img), 0x40000000, 1 << 40, None)
        assert got == want, (fn, a, got, want)
        checked += 1
    assert checked > 1000
