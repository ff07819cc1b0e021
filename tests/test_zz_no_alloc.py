"""hybrid_denoise_static: the hybrid with no device allocation.

Some callers cannot allocate device memory (a real-time loop with a fixed
memory budget, a plug-in whose host application owns the CUDA allocator).
This entry point keeps its scratch in a fixed array inside the library, so
the caller passes only its own input and output buffers.  These tests call
it through the C ABI and check that it returns exactly what hybrid_denoise
(with a caller-provided workspace) returns, on two calls in a row, and that
images too large for the fixed array are refused.  This file is collected
last so that, if it fails, a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ensure_built()
import paper_2005_05371_gb300 as hd  # noqa: E402
import synth  # noqa: E402

STATIC_BYTES = 36 * 1024 * 1024


def _dev(a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).to("cuda:0")


def _call_static(src, dst, p: "hd.Params"):
    img = hd.make_image(src, dst, p)
    return hd._lib.hybrid_denoise_static(ctypes.byref(img), hd._stream_ptr(None))


@pytest.mark.parametrize("name", ["plain512", "paper1620"])
def test_static_matches_workspace_path_twice(name):
    spec, _, g = synth.config_image(name)
    p = hd.Params(spec.smax, spec.wiener_w, bits=spec.bits)
    src = _dev(g)
    ref = torch.empty_like(src)
    hd.hybrid_denoise(src, ref, spec.smax, spec.wiener_w, bits=spec.bits)
    for _ in range(2):
        out = torch.full_like(src, 3)
        assert _call_static(src, out, p) == hd.HD_OK
        assert hd.hd_get_device_error() == hd.HD_OK
        torch.testing.assert_close(out, ref, rtol=0, atol=0)


def test_static_mixed_sizes_and_given_noise_variance():
    rng = np.random.default_rng(1)
    for H, W, bits in ((37, 91, 12), (300, 200, 8), (1, 5, 12)):
        dt = np.uint8 if bits == 8 else np.uint16
        g = rng.integers(0, (1 << bits), size=(H, W)).astype(dt)
        g[rng.random((H, W)) < 0.3] = 0
        src = _dev(g)
        for nv in (-1.0, 44.0):
            p = hd.Params(7, 5, noise_var=nv, bits=bits)
            ref = torch.empty_like(src)
            hd.hybrid_denoise(src, ref, 7, 5, noise_var=nv, bits=bits)
            for _ in range(2):
                out = torch.empty_like(src)
                assert _call_static(src, out, p) == hd.HD_OK
                torch.testing.assert_close(out, ref, rtol=0, atol=0)
    assert hd.hd_get_device_error() == hd.HD_OK


def test_static_rejects_images_beyond_the_fixed_scratch():
    p = hd.Params(7, 5, bits=12)
    need = hd.hybrid_min_workspace_size(4096, 4800, hd.HD_U16, p)
    assert need > STATIC_BYTES
    src = torch.zeros((4096, 4800), dtype=torch.int16, device="cuda:0")
    dst = torch.empty_like(src)
    assert _call_static(src, dst, p) == hd.HD_ERR_OVERFLOW
    assert hd.hybrid_min_workspace_size(4096, 4096, hd.HD_U16, p) <= STATIC_BYTES


def test_static_large_image_takes_the_recompute_path():
    """4096 x 4096 at 12 bits: the median plane fits the fixed array but the
    statistics plane does not, so the Wiener pass recomputes its window sums;
    the output still equals hybrid_denoise with its full workspace."""
    p = hd.Params(7, 5, bits=12)
    assert hd.hybrid_workspace_size(4096, 4096, hd.HD_U16, p) > STATIC_BYTES
    rng = np.random.default_rng(77)
    g = rng.integers(0, 4096, size=(4096, 4096)).astype(np.uint16)
    g[rng.random(g.shape) < 0.2] = 4095
    src = _dev(g)
    ref = torch.empty_like(src)
    hd.hybrid_denoise(src, ref, 7, 5, bits=12)
    out = torch.empty_like(src)
    assert _call_static(src, out, p) == hd.HD_OK
    torch.testing.assert_close(out, ref, rtol=0, atol=0)
    assert hd.hd_get_device_error() == hd.HD_OK
