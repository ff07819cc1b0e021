"""Parity of the reference noise variance (Algorithm 1, step 4d with the
original image handed to the Wiener stage) with the oracle, and the hybrid
run with it.

The sum is an exact integer and the quotient one binary64 division on both
sides, so the bar is equality of the binary64 values; the hybrid that uses
the value then meets the hybrid's own bar (integer output and binary32 value
equal to the oracle's twin).
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
from tests.test_gpu_parity import check_wiener, gpu_hybrid, to_dev  # noqa: E402

DEV = "cuda:0"


@pytest.mark.parametrize("shape", [(1, 1), (1, 999), (777, 1), (37, 91), (640, 480), (1031, 2049)])
@pytest.mark.parametrize("bits", [8, 12, 16])
def test_matches_oracle(shape, bits):
    rng = np.random.default_rng(shape[0] * 7 + shape[1] + bits)
    dt = np.uint8 if bits == 8 else np.uint16
    r = rng.integers(0, 1 << bits, size=shape).astype(dt)
    noise = rng.normal(0, (1 << bits) * 0.05, size=shape)
    f = np.clip(r + np.rint(noise), 0, (1 << bits) - 1).astype(dt)
    want, _ = oracle.reference_noise_variance(f, r)
    ws = hd._workspace(hd.HD_REFNOISE_WORKSPACE_BYTES, DEV)
    for pad_f, pad_r in ((0, 0), (5, 0), (0, 3)):
        got = hd.reference_noise_variance(to_dev(f, pad_f), to_dev(r, pad_r), workspace=ws)
        assert hd.hd_get_device_error() == hd.HD_OK
        assert float(got.item()) == want
    assert int(ws.count_nonzero()) == 0


def test_extremes():
    f = torch.full((300, 400), -1, dtype=torch.int16, device=DEV)       # every pixel 65535
    z = torch.zeros_like(f)
    assert float(hd.reference_noise_variance(f, z).item()) == float(65535 ** 2)
    assert float(hd.reference_noise_variance(z, z).item()) == 0.0


def test_hybrid_with_the_reference_noise_variance():
    """The paper's step 4d as it passes the original: the median output's
    noise variance against the clean phantom, then the one-pass hybrid with
    that variance, equal to the oracle's hybrid with the oracle's variance."""
    spec, clean, g = synth.config_image("paper1620")
    f_ref = oracle.amf(g, spec.smax)
    nu2_ref, _ = oracle.reference_noise_variance(f_ref, clean)
    src = to_dev(g)
    f = torch.empty_like(src)
    hd.amf_filter(src, f, smax=spec.smax)
    nu2 = float(hd.reference_noise_variance(f, to_dev(clean)).item())
    assert nu2 == nu2_ref
    _, ref = oracle.hybrid(g, spec.smax, spec.wiener_w, noise_var=nu2, bits=spec.bits)
    out, used, y = gpu_hybrid(g, spec.smax, spec.wiener_w, noise_var=nu2, bits=spec.bits, want_y=True)
    check_wiener(out, used, y, ref, spec.bits)


def test_argument_errors():
    a = torch.zeros((10, 12), dtype=torch.uint8, device=DEV)
    b = torch.zeros((10, 12), dtype=torch.int16, device=DEV)
    with pytest.raises(ValueError):
        hd.reference_noise_variance(a, b)
    ws = hd._workspace(hd.HD_REFNOISE_WORKSPACE_BYTES, DEV)
    small = ws[:(256 - ws.data_ptr() % 256) % 256 + 255]
    with pytest.raises(hd.HDError) as e:
        hd.reference_noise_variance(a, a, workspace=small)
    assert e.value.status == hd.HD_ERR_WORKSPACE
