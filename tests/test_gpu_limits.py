"""Every entry point at the largest dimension the ABI accepts (65535 rows, or
65535 columns), against the oracle on the whole image: the index arithmetic
along each axis (tile grid, row pieces, strip bounds, phase-2 shares) reaches
its limit, and the results stay exact."""
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
from tests.test_gpu_parity import (check_wiener, empty_like_dev, gpu_amf, gpu_hybrid, noisy_image,  # noqa: E402
                                   to_dev, to_host)

LIMIT = 65535


@pytest.mark.parametrize("shape,dtype,bits", [((LIMIT, 48), np.uint8, 8), ((40, LIMIT), np.uint16, 12)])
def test_largest_dimension(shape, dtype, bits):
    g = noisy_image(*shape, dtype, seed=11, density=0.3)
    if bits == 12:
        g = np.minimum(g, 4095).astype(np.uint16)
    smax, w = 9, 5
    f_ref, ref = oracle.hybrid(g, smax, w, bits=bits)
    np.testing.assert_array_equal(gpu_amf(g, smax), f_ref)
    out, nu2, y = gpu_hybrid(g, smax, w, bits=bits, want_y=True)
    check_wiener(out, nu2, y, ref, bits)
    # the stretch of the result, in place
    want, _, _ = oracle.contrast(ref.out32, 0.01, bits=bits)
    t = to_dev(ref.out32)
    hd.contrast_stretch(t, None, tol=0.01, bits=bits)
    assert hd.hd_get_device_error() == hd.HD_OK
    np.testing.assert_array_equal(to_host(t, g.dtype), want)
    # the partitioned median with more parts than a tile grid has rows
    parts = 16 if shape[0] > 1000 else 8
    _, sref = oracle.hybrid_strips(g, smax, w, parts, bits=bits)
    src = to_dev(g)
    dst = empty_like_dev(g)
    nv = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    hd.hybrid_denoise_strips(src, dst, parts, smax=smax, wiener_w=w, bits=bits, noise_var_out=nv)
    assert hd.hd_get_device_error() == hd.HD_OK
    np.testing.assert_array_equal(to_host(dst, g.dtype), sref.out32)
    assert float(nv.item()) == sref.nu2
    # the reference noise variance of the median output against the input
    nvr = hd.reference_noise_variance(to_dev(f_ref), src)
    assert float(nvr.item()) == oracle.reference_noise_variance(f_ref, g)[0]
