"""Parity of the contrast stretch kernel (Algorithm 1, step 4e) with the oracle.

The stretch is integer work (a histogram, two order statistics and an exact
integer map), so the bar is bit-exact output, on images that span many CTA
shares with ragged row pieces, at every bit depth the ABI takes, in place and
between distinct pitched buffers, and at the full sizes of the 1620 x 1620
and 4096 x 4096 workloads (the oracle computes those whole: it is linear).
"""
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


def to_dev(a, pad=0):
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a)
    if pad:
        big = torch.zeros((a.shape[0], a.shape[1] + pad), dtype=t.dtype, device=DEV)
        big[:, :a.shape[1]] = t.to(DEV)
        return big[:, :a.shape[1]]
    return t.to(DEV).contiguous()


def to_host(t, dtype):
    a = t.cpu().contiguous().numpy()
    return a.view(np.uint16) if dtype == np.uint16 else a


def image(H, W, bits, seed, kind="normal"):
    rng = np.random.default_rng(seed)
    maxv = (1 << bits) - 1
    dt = np.uint8 if bits == 8 else np.uint16
    if kind == "normal":
        x = rng.normal(maxv * 0.45, maxv * 0.12, size=(H, W))
    elif kind == "uniform":
        x = rng.integers(0, maxv + 1, size=(H, W))
    elif kind == "levels":          # few distinct values: long runs of equal lanes
        x = rng.choice([3, 9, maxv // 2, maxv - 4], size=(H, W))
    else:                           # flat with a few outliers
        x = np.full((H, W), maxv // 3)
        x.ravel()[rng.integers(0, H * W, size=max(1, H * W // 500))] = maxv
    return np.clip(np.rint(x), 0, maxv).astype(dt)


def gpu_stretch(x, tol, bits, pad_src=0, pad_dst=0, in_place=False, workspace=None):
    src = to_dev(x, pad_src)
    if in_place:
        hd.contrast_stretch(src, None, tol=tol, bits=bits, workspace=workspace)
        out = src
    else:
        dt = torch.uint8 if x.dtype == np.uint8 else torch.int16
        out = torch.full((x.shape[0], x.shape[1] + pad_dst), 5, dtype=dt, device=DEV)[:, :x.shape[1]]
        hd.contrast_stretch(src, out, tol=tol, bits=bits, workspace=workspace)
    assert hd.hd_get_device_error() == hd.HD_OK
    return to_host(out, x.dtype)


@pytest.mark.parametrize("bits", [8, 10, 12, 16])
@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (9, 1), (37, 91), (333, 517), (1111, 1303)])
def test_matches_oracle(bits, shape):
    for i, (kind, tol) in enumerate((("normal", 0.01), ("uniform", 0.0), ("levels", 0.1), ("flat", 0.0),
                                     ("normal", 0.49))):
        x = image(*shape, bits, seed=100 * bits + i, kind=kind)
        want, lo, hi = oracle.contrast(x, tol, bits=bits)
        got = gpu_stretch(x, tol, bits)
        np.testing.assert_array_equal(got, want, err_msg=f"{kind} tol={tol} lo={lo} hi={hi}")


@pytest.mark.parametrize("bits", [8, 12, 16])
def test_in_place_and_pitched(bits):
    x = image(301, 203, bits, seed=7)
    want, _, _ = oracle.contrast(x, 0.02, bits=bits)
    np.testing.assert_array_equal(gpu_stretch(x, 0.02, bits, in_place=True), want)
    np.testing.assert_array_equal(gpu_stretch(x, 0.02, bits, pad_src=9, pad_dst=0), want)
    np.testing.assert_array_equal(gpu_stretch(x, 0.02, bits, pad_src=0, pad_dst=17), want)
    np.testing.assert_array_equal(gpu_stretch(x, 0.02, bits, pad_src=4, pad_dst=4, in_place=True), want)


def test_workspace_is_zero_again_after_each_call():
    """The same workspace serves calls of different sizes and bit depths in a row."""
    ws = hd._workspace(hd.contrast_workspace_size(1, 1, hd.HD_U16, 16), DEV)
    for bits, shape, seed in ((12, (500, 700), 1), (8, (64, 64), 2), (16, (800, 999), 3), (12, (3, 5), 4),
                              (12, (500, 700), 1)):
        x = image(*shape, bits, seed=seed)
        want, _, _ = oracle.contrast(x, 0.05, bits=bits)
        np.testing.assert_array_equal(gpu_stretch(x, 0.05, bits, workspace=ws), want)
    assert int(ws.count_nonzero()) == 0


@pytest.mark.parametrize("name", ["paper1620", "stress4096"])
def test_full_size_after_hybrid(name):
    """The paper's full step 4 (hybrid then stretch) at the benchmark sizes:
    the stretch of the GPU hybrid output equals the oracle's stretch of the
    same image, and the hybrid output itself is the oracle's (checked in the
    hybrid parity tests), so the chain matches end to end."""
    spec, _, g = synth.config_image(name)
    src = to_dev(g)
    mid = torch.empty_like(src)
    hd.hybrid_denoise(src, mid, spec.smax, spec.wiener_w, bits=spec.bits)
    f = to_host(mid, g.dtype)
    want, lo, hi = oracle.contrast(f, 0.01, bits=spec.bits)
    assert lo < hi
    hd.contrast_stretch(mid, None, tol=0.01, bits=spec.bits)
    assert hd.hd_get_device_error() == hd.HD_OK
    np.testing.assert_array_equal(to_host(mid, g.dtype), want)


def test_argument_errors():
    x = torch.zeros((40, 50), dtype=torch.uint8, device=DEV)
    y = torch.zeros_like(x)
    for tol in (-0.01, 0.5, 1.0, float("nan")):
        with pytest.raises(hd.HDError) as e:
            hd.contrast_stretch(x, y, tol=tol)
        assert e.value.status == hd.HD_ERR_ARG
    big = torch.zeros((40, 60), dtype=torch.uint8, device=DEV)
    with pytest.raises(hd.HDError) as e:            # partial overlap
        hd.contrast_stretch(big[:, :50], big[:, 5:55])
    assert e.value.status == hd.HD_ERR_ARG
    need = hd.contrast_workspace_size(40, 50, hd.HD_U8)
    ws = hd._workspace(need, DEV)
    with pytest.raises(hd.HDError) as e:            # too small
        hd.contrast_stretch(x, y, workspace=ws[:need - 1 + (256 - ws.data_ptr() % 256) % 256])
    assert e.value.status == hd.HD_ERR_WORKSPACE
    with pytest.raises(hd.HDError) as e:            # bits above 8 for a uint8 image
        hd.contrast_stretch(x, y, bits=12)
    assert e.value.status == hd.HD_ERR_DTYPE


def test_wait_timeout_is_reported_and_recoverable():
    """A spin limit of one poll makes CTAs give up waiting for the others'
    histograms: the kernel returns, the error word says TIMEOUT, the
    workspace is still left zeroed, and the next call is exact."""
    x = image(2048, 2048, 12, seed=9)
    ws = hd._workspace(hd.contrast_workspace_size(2048, 2048, hd.HD_U16, 12), DEV)
    src = to_dev(x)
    dst = torch.empty_like(src)
    try:
        hd.hd_set_spin_limit(1)
        hd.contrast_stretch(src, dst, tol=0.01, bits=12, workspace=ws)
        assert hd.hd_get_device_error() == hd.HD_ERR_TIMEOUT
    finally:
        hd.hd_set_spin_limit(0)
    assert hd.hd_get_device_error() == hd.HD_OK
    assert int(ws.count_nonzero()) == 0
    want, _, _ = oracle.contrast(x, 0.01, bits=12)
    np.testing.assert_array_equal(gpu_stretch(x, 0.01, 12, workspace=ws), want)
