"""Parity of the partitioned hybrid (Algorithm 1, step 6 with `parts` strips)
with the oracle.

Each strip's median is integer-exact and the Wiener stage follows the same
binary32 contract as hybrid_denoise, so the bar is the hybrid's: the integer
output and the binary32 value equal the oracle's twin bit for bit and the
noise variance equals the oracle's binary64 value.
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
from tests.test_gpu_parity import check_wiener, empty_like_dev, noisy_image, to_dev, to_host  # noqa: E402

DEV = "cuda:0"


def gpu_strips(g, smax, w, parts, noise_var=-1.0, bits=None, pad=0, workspace=None):
    src = to_dev(g, pad)
    dst = empty_like_dev(g, pad)
    nv = torch.full((1,), -7.0, dtype=torch.float64, device=DEV)
    y = torch.empty(g.shape, dtype=torch.float32, device=DEV)
    hd.hybrid_denoise_strips(src, dst, parts, smax=smax, wiener_w=w, noise_var=noise_var, bits=bits,
                             noise_var_out=nv, y_out=y, workspace=workspace)
    assert hd.hd_get_device_error() == hd.HD_OK
    return to_host(dst, g.dtype), float(nv.item()), y.cpu().numpy()


@pytest.mark.parametrize("shape", [(9, 40), (97, 131), (256, 200), (301, 77)])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_matches_oracle(shape, dtype):
    bits = 8 if dtype == np.uint8 else 12
    g = noisy_image(*shape, dtype, seed=shape[0] + 7 * shape[1])
    for parts, smax, w, nv in ((1, 7, 3, -1.0), (2, 9, 5, -1.0), (3, 5, 3, 30.0), (4, 11, 5, -1.0),
                               (8, 7, 7, -1.0), (shape[0], 5, 3, -1.0)):
        if parts > shape[0]:
            continue
        _, ref = oracle.hybrid_strips(g, smax, w, parts, noise_var=nv, bits=bits)
        out, nu2, y = gpu_strips(g, smax, w, parts, noise_var=nv, bits=bits, pad=3 if parts == 3 else 0)
        check_wiener(out, nu2, y, ref, bits)


def test_seams_differ_from_whole_image():
    g = noisy_image(120, 90, np.uint8, seed=5)
    whole, _, _ = gpu_strips(g, 9, 5, 1)
    four, _, _ = gpu_strips(g, 9, 5, 4)
    _, ref1 = oracle.hybrid(g, 9, 5)
    np.testing.assert_array_equal(whole, ref1.out32)
    assert (four != whole).any()


@pytest.mark.parametrize("parts", [2, 4, 8])
def test_full_size_paper_partitions(parts):
    """The paper's worker counts on the 1620 x 1620 workload."""
    spec, _, g = synth.config_image("paper1620")
    _, ref = oracle.hybrid_strips(g, spec.smax, spec.wiener_w, parts, bits=spec.bits)
    out, nu2, y = gpu_strips(g, spec.smax, spec.wiener_w, parts, bits=spec.bits)
    check_wiener(out, nu2, y, ref, spec.bits)


def test_workspace_reuse_and_errors():
    g = noisy_image(200, 150, np.uint16, seed=8)
    p = hd.Params(7, 5, bits=12)
    ws = hd._workspace(hd.hybrid_strips_workspace_size(200, 150, hd.HD_U16, p, 16), DEV)
    for parts in (16, 2, 5, 16):
        _, ref = oracle.hybrid_strips(g, 7, 5, parts, bits=12)
        out, nu2, y = gpu_strips(g, 7, 5, parts, bits=12, workspace=ws)
        check_wiener(out, nu2, y, ref, 12)
    src = to_dev(g)
    dst = torch.empty_like(src)
    for parts in (0, 201, -1):
        with pytest.raises(hd.HDError) as e:
            hd.hybrid_denoise_strips(src, dst, parts, smax=7, wiener_w=5, bits=12)
        assert e.value.status == hd.HD_ERR_ARG
    need = hd.hybrid_strips_workspace_size(200, 150, hd.HD_U16, p, 4)
    small = hd._workspace(need, DEV)
    small = small[:(256 - small.data_ptr() % 256) % 256 + need - 1]
    with pytest.raises(hd.HDError) as e:
        hd.hybrid_denoise_strips(src, dst, 4, smax=7, wiener_w=5, bits=12, workspace=small)
    assert e.value.status == hd.HD_ERR_WORKSPACE
