"""Rectangular Wiener windows (wiener_h rows by wiener_w columns) on the GPU
against the oracle's rectangular statistics: integer output and binary32 value
bit for bit, the noise variance exactly, through every path that runs the
Wiener stage (statistics plane, recompute pass, one pass with a given noise
variance, the Wiener filter alone, batches and image parts)."""
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
from paper_2005_05371_gb300 import split  # noqa: E402

DEV = "cuda:0"
WINDOWS = [(1, 3), (3, 1), (3, 7), (7, 3), (5, 15), (15, 5), (1, 15), (9, 5)]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int16) if a.dtype == np.uint16 else np.ascontiguousarray(a))


def _host(t, dtype):
    a = t.cpu().numpy()
    return a.view(np.uint16) if dtype == np.uint16 else a


def _noisy(H, W, bits, seed, density=0.25):
    rng = np.random.default_rng(seed)
    maxv = (1 << bits) - 1
    g = rng.integers(0, maxv + 1, size=(H, W))
    g[H // 4:H // 2, W // 4:W // 2] = maxv // 3
    g[H // 2:, :W // 3] = rng.integers(0, 3, size=g[H // 2:, :W // 3].shape)
    u = rng.random((H, W))
    g[u < density / 2] = 0
    g[(u >= density / 2) & (u < density)] = maxv
    return g.astype(np.uint8 if bits == 8 else np.uint16)


def _check(out, nu2, y, ref, bits):
    assert nu2 == ref.nu2
    np.testing.assert_array_equal(out, ref.out32)
    if y is not None:
        np.testing.assert_array_equal(y, ref.y32)
        assert np.max(np.abs(y.astype(np.float64) - ref.y64)) <= ((1 << bits) - 1) * 2.0 ** -20


@pytest.mark.parametrize("wh,ww", WINDOWS)
@pytest.mark.parametrize("bits", [8, 12, 16])
@pytest.mark.parametrize("minimal", [False, True])
def test_hybrid_rect_window(wh, ww, bits, minimal):
    g = _noisy(97, 131, bits, seed=wh * 100 + ww + bits)
    smax = 9
    _, ref = oracle.hybrid(g, smax, ww, bits=bits, wh=wh)
    src = _t(g).to(DEV)
    dst = torch.full_like(src, 7)
    nv = torch.full((1,), -7.0, dtype=torch.float64, device=DEV)
    y = torch.empty(g.shape, dtype=torch.float32, device=DEV)
    code = hd.HD_U8 if bits == 8 else hd.HD_U16
    p = hd.Params(smax, ww, bits=bits, wiener_h=wh)
    n = hd.hybrid_min_workspace_size(*g.shape, code, p) if minimal else hd.hybrid_workspace_size(*g.shape, code, p)
    ws = hd._workspace(n, DEV)
    hd.hybrid_denoise(src, dst, smax, ww, bits=bits, workspace=ws, noise_var_out=nv, y_out=y, wiener_h=wh)
    assert hd.hd_get_device_error() == hd.HD_OK
    _check(_host(dst, g.dtype), float(nv.item()), y.cpu().numpy(), ref, bits)


@pytest.mark.parametrize("wh,ww", [(3, 7), (7, 3), (1, 5)])
def test_rect_given_noise_variance_zero_border_and_wiener_alone(wh, ww):
    g = _noisy(70, 90, 12, seed=3)
    f = oracle.amf(g, 7)
    for nv_in, bz in ((33.0, 0), (-1.0, 1), (0.0, 1)):
        _, ref = oracle.hybrid(g, 7, ww, noise_var=nv_in, bits=12, border_zero=bool(bz), wh=wh)
        src = _t(g).to(DEV)
        dst = torch.empty_like(src)
        nv = torch.zeros(1, dtype=torch.float64, device=DEV)
        hd.hybrid_denoise(src, dst, 7, ww, nv_in, bz, 0, 12, noise_var_out=nv, wiener_h=wh)
        assert hd.hd_get_device_error() == hd.HD_OK
        _check(_host(dst, np.uint16), float(nv.item()), None, ref, 12)
        # the Wiener filter alone, on the oracle's median
        fr = oracle.wiener(f, ww, noise_var=nv_in, bits=12, border_zero=bool(bz), wh=wh)
        fsrc = _t(f).to(DEV)
        fdst = torch.empty_like(fsrc)
        hd.wiener_filter(fsrc, fdst, ww, nv_in, bz, 12, noise_var_out=nv, wiener_h=wh)
        assert hd.hd_get_device_error() == hd.HD_OK
        _check(_host(fdst, np.uint16), float(nv.item()), None, fr, 12)


def test_rect_windows_in_a_batch():
    rng = np.random.default_rng(8)
    items, refs = [], []
    for i, (wh, ww) in enumerate(WINDOWS):
        H, W = int(rng.integers(20, 260)), int(rng.integers(20, 260))
        bits = 8 if i % 2 else 12
        g = _noisy(H, W, bits, seed=50 + i)
        p = hd.Params(int(rng.choice([5, 9, 11])), ww, -1.0, 0, 0, bits, wh)
        src = _t(g).to(DEV)
        items.append((src, torch.empty_like(src), p))
        refs.append((g, oracle.hybrid(g, p.smax, ww, bits=bits, wh=wh)[1]))
    hd.hybrid_denoise_batched(items)
    assert hd.hd_get_device_error() == hd.HD_OK
    for (_, dst, _), (g, ref) in zip(items, refs):
        np.testing.assert_array_equal(_host(dst, g.dtype), ref.out32)


@pytest.mark.parametrize("wh,ww,P", [(7, 3, 3), (3, 9, 4), (15, 1, 2)])
def test_rect_windows_in_image_parts(wh, ww, P):
    g = _noisy(88, 75, 12, seed=wh + ww)
    p = hd.Params(9, ww, -1.0, 0, 0, 12, wh)
    H, W = g.shape
    halo = hd.part_halo_rows(p)
    assert halo == 9 // 2 + wh // 2
    tg = _t(g).to(DEV)
    parts = split.all_parts(H, P, halo)
    total = torch.zeros(4, dtype=torch.int64, device=DEV)
    bes, bufs = [], []
    for me in parts:
        be = split.CudaPartBackend()
        buf = tg[me.buf0:me.buf1].clone()
        total += be.stats(buf, me, H, W, p)
        bes.append(be)
        bufs.append(buf)
    out = torch.cat([be.apply(b, me, H, W, p, total.clone()) for be, b, me in zip(bes, bufs, parts)])
    assert hd.hd_get_device_error() == hd.HD_OK
    _, ref = oracle.hybrid(g, 9, ww, bits=12, wh=wh)
    np.testing.assert_array_equal(_host(out, np.uint16), ref.out32)
