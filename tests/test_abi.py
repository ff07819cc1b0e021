"""The C-ABI library loads, exports every declared symbol, and validates
arguments on the host before any device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

from tests._lib import ROOT, ensure_built

ensure_built()
import paper_2005_05371_gb300 as hd  # noqa: E402

HEADER = os.path.join(ROOT, "include", "hybrid_denoise.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    assert set(hd.EXPORTS) == set(names), set(hd.EXPORTS) ^ set(names)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(hd.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_version():
    assert hd.hd_status_str(hd.HD_OK) == "ok"
    assert "Smax" in hd.hd_status_str(hd.HD_ERR_SMAX)
    assert hd.hd_status_str(99) == "unknown status"
    assert hd.hd_version() >= 100


def _img(H=16, W=16, dtype=hd.HD_U8, smax=5, w=3, bits=None, src=0x100000, dst=0x900000,
         pitch=None, noise_var=-1.0, border=0, unresolved=0):
    es = 1 if dtype == hd.HD_U8 else 2
    pitch = pitch if pitch is not None else W * es
    b = bits if bits is not None else (8 if dtype == hd.HD_U8 else 12)
    p = hd.hd_params(smax, w, noise_var, border, unresolved, b)
    return hd.hd_image(src, dst, H, W, pitch, pitch, dtype, p, None, None)


def call(fn, img, ws=None, nbytes=0):
    lib = hd._lib
    if fn == "amf_filter":
        return lib.amf_filter(ctypes.byref(img), None)
    return getattr(lib, fn)(ctypes.byref(img), ws, nbytes, None)


@pytest.mark.parametrize("fn", ["amf_filter", "hybrid_denoise"])
@pytest.mark.parametrize("smax", [-1, 0, 1, 2, 4, 10, 17, 101])
def test_smax_rejected(fn, smax):
    # Algorithm 1, step 6a: Smax must be an odd integer > 1 (and within the build's cap)
    assert call(fn, _img(smax=smax)) == hd.HD_ERR_SMAX


@pytest.mark.parametrize("w", [0, -1, 2, 4, 17])
def test_window_rejected(w):
    assert call("wiener_filter", _img(w=w)) == hd.HD_ERR_WINDOW
    assert call("hybrid_denoise", _img(w=w)) == hd.HD_ERR_WINDOW


@pytest.mark.parametrize("wh", [-1, 2, 4, 17])
def test_window_rows_rejected(wh):
    img = _img(w=5)
    img.p.wiener_h = wh
    assert call("wiener_filter", img) == hd.HD_ERR_WINDOW
    assert call("hybrid_denoise", img) == hd.HD_ERR_WINDOW
    assert call("amf_filter", img) != hd.HD_ERR_WINDOW           # the median ignores the Wiener window
    p = hd.Params(7, 5, wiener_h=wh).to_c(hd.HD_U8)
    n = ctypes.c_int()
    assert hd._lib.hd_part_halo_rows(ctypes.byref(p), ctypes.byref(n)) == hd.HD_ERR_WINDOW


def test_bad_arguments_rejected():
    assert call("amf_filter", _img(src=0)) == hd.HD_ERR_ARG
    assert call("amf_filter", _img(dst=0)) == hd.HD_ERR_ARG
    assert call("amf_filter", _img(H=0)) == hd.HD_ERR_ARG
    assert call("amf_filter", _img(W=-3)) == hd.HD_ERR_ARG
    assert call("amf_filter", _img(H=70000)) == hd.HD_ERR_OVERFLOW
    assert call("amf_filter", _img(pitch=15)) == hd.HD_ERR_ARG               # pitch < W
    assert call("amf_filter", _img(dtype=hd.HD_U16, pitch=33)) == hd.HD_ERR_ARG   # odd pitch
    assert call("amf_filter", _img(dtype=7)) == hd.HD_ERR_DTYPE
    assert call("amf_filter", _img(dtype=hd.HD_U8, bits=12)) == hd.HD_ERR_DTYPE
    assert call("amf_filter", _img(dtype=hd.HD_U16, bits=17)) == hd.HD_ERR_DTYPE
    assert call("amf_filter", _img(dtype=hd.HD_U16, bits=0)) == hd.HD_ERR_DTYPE
    assert call("amf_filter", _img(unresolved=5)) == hd.HD_ERR_ARG
    assert call("wiener_filter", _img(border=3)) == hd.HD_ERR_ARG
    assert call("wiener_filter", _img(noise_var=float("nan"))) == hd.HD_ERR_ARG
    # source and destination overlap
    assert call("amf_filter", _img(src=0x100000, dst=0x100000 + 40)) == hd.HD_ERR_ARG


def test_workspace_checks_before_launch():
    img = _img()
    assert call("hybrid_denoise", img, None, 0) == hd.HD_ERR_WORKSPACE
    assert call("hybrid_denoise", img, 0x1000 + 8, 1 << 20) == hd.HD_ERR_WORKSPACE   # misaligned
    need = hd.hybrid_min_workspace_size(16, 16, hd.HD_U8, hd.Params(5, 3))
    assert call("hybrid_denoise", img, 0x10000, need - 1) == hd.HD_ERR_WORKSPACE


def test_workspace_sizes():
    p = hd.Params(11, 5)
    n8 = hd.hybrid_min_workspace_size(1620, 1620, hd.HD_U8, p)
    n16 = hd.hybrid_min_workspace_size(4096, 4096, hd.HD_U16, p)
    assert n8 >= 1620 * 1620 and n8 < 1620 * 1620 + 64 * 1024
    assert n16 >= 4096 * 4096 * 2 and n16 < 4096 * 4096 * 2 + 64 * 1024
    # the full size adds the binary32 (mu, sigma2) plane: 8 bytes per pixel
    f8 = hd.hybrid_workspace_size(1620, 1620, hd.HD_U8, p)
    assert f8 - n8 >= 8 * 1620 * 1620 and f8 - n8 < 8 * 1620 * 1620 + 512
    assert hd.hybrid_min_workspace_size(512, 512, hd.HD_U8, hd.Params(7, 3, noise_var=25.0)) == 0
    # a supplied noise variance makes the hybrid one pass: no workspace
    assert hd.hybrid_workspace_size(512, 512, hd.HD_U8, hd.Params(7, 3, noise_var=25.0)) == 0
    assert hd.wiener_workspace_size(512, 512, hd.HD_U8, hd.Params(7, 3)) > 0
    assert hd.hybrid_host_workspace_size(100, 100, hd.HD_U16, p) >= 2 * 100 * 100 * 2


def test_tuning_validation():
    old = hd.hd_get_tuning()
    try:
        for bad in ((8, 0), (20, 0), (136, 0), (32, 9), (32, -1), (32, 0, 4), (32, 0, -1), (32, 0, 0, 33),
                    (32, 0, 0, -2), (32, 0, 0, 0, 3), (32, 0, 0, 0, 16), (32, 0, 0, 0, 0, 65), (32, 0, 0, 0, 0, -1),
                    (32, 0, 0, 0, 0, 0, 2)):
            with pytest.raises(hd.HDError):
                hd.hd_set_tuning(*bad)
        hd.hd_set_tuning(64, 2)
        assert hd.hd_get_tuning() == (64, 2, 0, 0, 0, 0, 0)
        hd.hd_set_tuning(48, 3, 1, -1, 8, 5, 1)
        assert hd.hd_get_tuning() == (48, 3, 1, -1, 8, 5, 1)
        for plane in (2, 3):        # the plane with its Wiener pass staged / read from L2
            hd.hd_set_tuning(32, 0, plane)
            assert hd.hd_get_tuning()[2] == plane
    finally:
        hd.hd_set_tuning(*old)


def test_batched_validation():
    imgs = (hd.hd_image * 2)(_img(), _img(smax=4))
    n = ctypes.c_size_t()
    assert hd._lib.hybrid_batched_workspace_size(imgs, 0, ctypes.byref(n)) == hd.HD_ERR_ARG
    assert hd._lib.hybrid_denoise_batched(imgs, 2, 0x10000, 1 << 30, None) == hd.HD_ERR_SMAX
    plan = ctypes.c_void_p()
    assert hd._lib.hd_batch_plan_create(imgs, 2, 0x10000, 1 << 30, ctypes.byref(plan)) == hd.HD_ERR_SMAX
    assert hd._lib.hd_batch_plan_launch(None, None) == hd.HD_ERR_ARG


def test_contrast_argument_checks_before_launch():
    lib = hd._lib
    img = _img()
    for tol in (-0.1, 0.5, float("nan")):
        assert lib.contrast_stretch(ctypes.byref(img), tol, 0x10000, 1 << 20, None) == hd.HD_ERR_ARG
    # in place is allowed only with the same pitch; partial overlap is refused
    ov = _img(src=0x100000, dst=0x100004)
    assert lib.contrast_stretch(ctypes.byref(ov), 0.01, 0x10000, 1 << 20, None) == hd.HD_ERR_ARG
    assert lib.contrast_stretch(ctypes.byref(img), 0.01, None, 0, None) == hd.HD_ERR_WORKSPACE
    assert lib.contrast_stretch(ctypes.byref(img), 0.01, 0x10008, 1 << 20, None) == hd.HD_ERR_WORKSPACE
    need = hd.contrast_workspace_size(16, 16, hd.HD_U8)
    assert need == 256 + 256 * 4
    assert lib.contrast_stretch(ctypes.byref(img), 0.01, 0x10000, need - 1, None) == hd.HD_ERR_WORKSPACE
    assert hd.contrast_workspace_size(16, 16, hd.HD_U16, 12) == 256 + 4096 * 4
    assert lib.contrast_stretch(ctypes.byref(_img(dtype=hd.HD_U8, bits=12)), 0.01, 0x10000, 1 << 20,
                                None) == hd.HD_ERR_DTYPE


def test_strips_argument_checks_before_launch():
    lib = hd._lib
    img = _img(H=16)
    for parts in (0, -2, 17):
        assert lib.hybrid_denoise_strips(ctypes.byref(img), parts, 0x10000, 1 << 30, None) == hd.HD_ERR_ARG
    assert lib.hybrid_denoise_strips(ctypes.byref(_img(smax=4)), 2, 0x10000, 1 << 30, None) == hd.HD_ERR_SMAX
    p = hd.Params(7, 5)
    # one part is the whole-image hybrid; more parts add the strip tables
    assert hd.hybrid_strips_workspace_size(64, 64, hd.HD_U8, p, 1) == hd.hybrid_workspace_size(64, 64, hd.HD_U8, p)
    assert hd.hybrid_strips_workspace_size(64, 64, hd.HD_U8, p, 8) > hd.hybrid_strips_workspace_size(64, 64, hd.HD_U8, p, 2)
    need = hd.hybrid_strips_workspace_size(16, 16, hd.HD_U8, hd.Params(5, 3), 4)
    assert lib.hybrid_denoise_strips(ctypes.byref(img), 4, 0x10000, need - 1, None) == hd.HD_ERR_WORKSPACE


def test_reference_and_pipeline_argument_checks():
    lib = hd._lib
    S = ctypes.c_size_t
    assert lib.reference_noise_variance(None, 16, 0x2000, 16, 16, 16, hd.HD_U8, 0x3000, 0x10000, 256,
                                        None) == hd.HD_ERR_ARG
    assert lib.reference_noise_variance(0x1000, 15, 0x2000, 16, 16, 16, hd.HD_U8, 0x3000, 0x10000, 256,
                                        None) == hd.HD_ERR_ARG
    assert lib.reference_noise_variance(0x1000, 16, 0x2000, 16, 16, 16, hd.HD_U8, 0x3004, 0x10000, 256,
                                        None) == hd.HD_ERR_ARG                       # misaligned output
    assert lib.reference_noise_variance(0x1000, 16, 0x2000, 16, 16, 16, hd.HD_U8, 0x3000, 0x10000, 255,
                                        None) == hd.HD_ERR_WORKSPACE
    assert lib.reference_noise_variance(0x1000, 32, 0x2001, 32, 16, 16, hd.HD_U16, 0x3000, 0x10000, 256,
                                        None) == hd.HD_ERR_ARG                       # odd u16 address
    n = S()
    c = hd.Params(7, 5).to_c(hd.HD_U8)
    for depth in (0, 9):
        assert lib.hd_host_pipeline_workspace_size(64, 64, hd.HD_U8, ctypes.byref(c), depth,
                                                   ctypes.byref(n)) == hd.HD_ERR_ARG
    assert lib.hd_host_pipeline_workspace_size(64, 64, hd.HD_U8, ctypes.byref(c), 2, ctypes.byref(n)) == hd.HD_OK
    core = hd.hybrid_workspace_size(64, 64, hd.HD_U8, hd.Params(7, 5))
    assert n.value == (core + 255) // 256 * 256 + 2 * 2 * ((64 * 64 + 255) // 256 * 256)
    pl = ctypes.c_void_p()
    bad = hd.Params(8, 5).to_c(hd.HD_U8)
    assert lib.hd_host_pipeline_create(64, 64, hd.HD_U8, ctypes.byref(bad), 2, 0x10000, 1 << 30,
                                       ctypes.byref(pl)) == hd.HD_ERR_SMAX
    assert lib.hd_host_pipeline_create(64, 64, hd.HD_U8, ctypes.byref(c), 2, 0x10000, n.value - 1,
                                       ctypes.byref(pl)) == hd.HD_ERR_WORKSPACE
    assert lib.hd_host_pipeline_submit(None, 0x1000, 64, 0x2000, 64) == hd.HD_ERR_ARG
    assert lib.hd_host_pipeline_wait(None) == hd.HD_ERR_ARG
    assert lib.hd_host_pipeline_destroy(None) == hd.HD_ERR_ARG


def test_batch_pipeline_argument_checks():
    lib = hd._lib
    S = ctypes.c_size_t
    shapes = [(64, 64, hd.HD_U16, hd.Params(7, 5, bits=12)), (30, 50, hd.HD_U16, hd.Params(5, 3, bits=12)),
              (17, 9, hd.HD_U8, hd.Params(9, 7))]
    arr = (hd.hd_image * 3)(*[hd._shape_image(*s) for s in shapes])
    n = S()
    for depth in (0, 9):
        assert lib.hd_batch_pipeline_workspace_size(arr, 3, depth, ctypes.byref(n)) == hd.HD_ERR_ARG
    assert lib.hd_batch_pipeline_workspace_size(arr, 0, 2, ctypes.byref(n)) == hd.HD_ERR_ARG
    assert lib.hd_batch_pipeline_workspace_size(arr, 3, 2, ctypes.byref(n)) == hd.HD_OK
    # per slot: the batch workspace, then the noisy and result planes packed
    # back to back (each aligned to its element size)
    ws = hd.hybrid_batched_workspace_size([hd.hd_image(0x10000, 0x20000000, H, W, W * (1 + c), W * (1 + c), c,
                                                       p.to_c(c), None, None) for H, W, c, p in shapes])
    planes = 64 * 64 * 2 + 30 * 50 * 2 + 17 * 9
    slot = (ws + 255) // 256 * 256 + 2 * ((planes + 255) // 256 * 256)
    assert n.value == 2 * slot
    pl = ctypes.c_void_p()
    assert lib.hd_batch_pipeline_create(arr, 3, 2, 0x10000, n.value - 1, ctypes.byref(pl)) == hd.HD_ERR_WORKSPACE
    assert lib.hd_batch_pipeline_create(arr, 3, 2, 0x10001, n.value, ctypes.byref(pl)) == hd.HD_ERR_WORKSPACE
    bad = (hd.hd_image * 1)(hd._shape_image(8, 8, 5, hd.Params(7, 5)))
    assert lib.hd_batch_pipeline_workspace_size(bad, 1, 2, ctypes.byref(n)) == hd.HD_ERR_DTYPE
    assert lib.hd_batch_pipeline_submit(None, None, None, None, None) == hd.HD_ERR_ARG
    assert lib.hd_batch_pipeline_wait(None) == hd.HD_ERR_ARG
    assert lib.hd_batch_pipeline_destroy(None) == hd.HD_ERR_ARG


def test_part_argument_checks():
    lib = hd._lib
    S = ctypes.c_size_t

    def part(**kw):
        a = dict(src=0x100000, src_pitch=64, dst=0x900000, dst_pitch=64, H=100, W=64, buf_row0=20, buf_rows=40,
                 own_row0=25, own_rows=30, dtype=hd.HD_U8, smax=7, w=5, nv=-1.0, border=0, unres=0, bits=8)
        a.update(kw)
        p = hd.hd_params(a["smax"], a["w"], a["nv"], a["border"], a["unres"], a["bits"])
        return hd.hd_part(a["src"], a["src_pitch"], a["dst"], a["dst_pitch"], a["H"], a["W"], a["buf_row0"],
                          a["buf_rows"], a["own_row0"], a["own_rows"], a["dtype"], p)

    n = S()
    halo = ctypes.c_int()
    assert lib.hd_part_halo_rows(ctypes.byref(hd.Params(7, 5).to_c(hd.HD_U8)), ctypes.byref(halo)) == hd.HD_OK
    assert halo.value == 5
    assert lib.hd_part_halo_rows(ctypes.byref(hd.Params(6, 5).to_c(hd.HD_U8)), ctypes.byref(halo)) == hd.HD_ERR_SMAX
    ok = part()
    assert lib.hybrid_part_workspace_size(ctypes.byref(ok), ctypes.byref(n)) == hd.HD_OK
    assert n.value >= 40 * 64 * 8
    cases = [
        (dict(buf_row0=21), hd.HD_ERR_ARG),              # buffer misses a halo row above
        (dict(buf_rows=39), hd.HD_ERR_ARG),              # ... and below
        (dict(own_row0=19), hd.HD_ERR_ARG),              # own rows outside the buffer
        (dict(buf_row0=70, own_row0=75, buf_rows=31), hd.HD_ERR_ARG),   # buffer beyond the image
        (dict(own_rows=0), hd.HD_ERR_ARG),
        (dict(nv=5.0), hd.HD_ERR_ARG),                   # a known noise variance needs no split
        (dict(smax=8), hd.HD_ERR_SMAX),
        (dict(w=4), hd.HD_ERR_WINDOW),
        (dict(dtype=hd.HD_U16, bits=12, src=0x100001, src_pitch=128, dst_pitch=128), hd.HD_ERR_ARG),
        (dict(bits=12), hd.HD_ERR_DTYPE),
        (dict(src_pitch=63), hd.HD_ERR_ARG),
        (dict(H=70000), hd.HD_ERR_OVERFLOW),
    ]
    for kw, want in cases:
        got = lib.hybrid_part_workspace_size(ctypes.byref(part(**kw)), ctypes.byref(n))
        assert got == want, (kw, got, want)
    # the buffer may start at row 0 when the halo would reach above the image
    assert lib.hybrid_part_workspace_size(ctypes.byref(part(buf_row0=0, own_row0=3, buf_rows=38)),
                                          ctypes.byref(n)) == hd.HD_OK
    sums = 0x3000
    assert lib.hybrid_part_stats(ctypes.byref(ok), 0x10000, 0, sums, None) == hd.HD_ERR_WORKSPACE
    assert lib.hybrid_part_stats(ctypes.byref(ok), 0x10000, 1 << 30, 0x3004, None) == hd.HD_ERR_ARG
    assert lib.hybrid_part_apply(ctypes.byref(part(dst=0)), sums, 0x10000, 1 << 30, None) == hd.HD_ERR_ARG
    assert lib.hybrid_part_apply(ctypes.byref(part(dst=0x100000 + 64 * 10)), sums, 0x10000, 1 << 30,
                                 None) == hd.HD_ERR_ARG                                   # dst overlaps src
    assert lib.hybrid_part_apply(ctypes.byref(ok), sums, 0x10010, 1 << 30, None) == hd.HD_ERR_WORKSPACE


def test_fourier_wiener_argument_checks():
    lib = hd._lib
    S = ctypes.c_size_t
    n = S()
    assert lib.wiener_deconv_workspace_size(1620, 1620, ctypes.byref(n)) == hd.HD_OK
    assert n.value >= 3 * 1620 * 1620 * 8
    for H, W in ((8192, 8192), (4096, 8), (3000, 4096), (1, 1)):
        assert lib.wiener_deconv_workspace_size(H, W, ctypes.byref(n)) == hd.HD_OK, (H, W)
    for H, W in ((16384, 8), (4097, 8), (8, 5000)):
        assert lib.wiener_deconv_workspace_size(H, W, ctypes.byref(n)) == hd.HD_ERR_OVERFLOW, (H, W)
    assert lib.wiener_deconv_workspace_size(0, 8, ctypes.byref(n)) == hd.HD_ERR_ARG
    img = _img(H=16, W=16)
    ws, big = 0x10000, 1 << 30
    assert lib.wiener_deconvolve(ctypes.byref(img), None, 3, 3, 0.1, ws, big, None) == hd.HD_ERR_ARG
    assert lib.wiener_deconvolve(ctypes.byref(img), 0x5002, 3, 3, 0.1, ws, big, None) == hd.HD_ERR_ARG
    for kh, kw in ((0, 3), (3, 0), (256, 1)):
        assert lib.wiener_deconvolve(ctypes.byref(img), 0x5000, kh, kw, 0.1, ws, big, None) == hd.HD_ERR_ARG
    for nsr in (-0.1, float("nan"), float("inf")):
        assert lib.wiener_deconvolve(ctypes.byref(img), 0x5000, 3, 3, nsr, ws, big, None) == hd.HD_ERR_ARG
    assert lib.wiener_deconvolve(ctypes.byref(img), 0x5000, 3, 3, 0.1, ws, 10, None) == hd.HD_ERR_WORKSPACE
    assert lib.wiener_deconvolve(ctypes.byref(_img(H=16, W=5000)), 0x5000, 3, 3, 0.1, ws, big,
                                 None) == hd.HD_ERR_OVERFLOW
    assert lib.wiener_deconvolve(ctypes.byref(_img(dtype=hd.HD_U8, bits=9)), 0x5000, 3, 3, 0.1, ws, big,
                                 None) == hd.HD_ERR_DTYPE
    assert lib.wiener_deconvolve(ctypes.byref(_img(dst=0x100000 + 8)), 0x5000, 3, 3, 0.1, ws, big,
                                 None) == hd.HD_ERR_ARG                   # dst overlaps src


def test_header_is_plain_c_and_links(tmp_path):
    """The ABI header compiles as C99 (no C++ in its declarations) and a C
    program that takes the address of every entry point links against the
    library."""
    import shutil
    import subprocess
    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = declared_functions()
    src = tmp_path / "use_abi.c"
    src.write_text('#include "hybrid_denoise.h"\n#include <stdio.h>\nint main(void) {\n'
                   + "".join(f'    printf("%p\\n", (void *)&{n});\n' for n in names)
                   + '    return hd_version() > 0 ? 0 : 1;\n}\n')
    exe = tmp_path / "use_abi"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"), str(src),
                        "-o", str(exe), os.path.join(root, "paper_2005_05371_gb300", "libhd.so"),
                        "-Wl,-rpath," + os.path.join(root, "paper_2005_05371_gb300")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
