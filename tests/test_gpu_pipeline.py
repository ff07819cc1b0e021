"""The host pipeline (hd_host_pipeline_*): many host images of one size through
the hybrid with copies overlapping kernels.  Every result must equal the
oracle's (the hybrid's bar: integer output equal to the binary32 twin), for
every depth, with tight and padded host rows, and with more steps than slots
so that every slot is reused."""
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
from tests.test_gpu_parity import noisy_image  # noqa: E402


def pinned(a):
    t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).pin_memory()
    return t


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("dtype,bits", [(np.uint8, 8), (np.uint16, 12)])
def test_pipeline_matches_oracle(depth, dtype, bits):
    H, W, smax, w = 150, 211, 9, 5
    imgs = [noisy_image(H, W, dtype, seed=100 + i, density=0.1 + 0.05 * i) for i in range(7)]
    refs = [oracle.hybrid(g, smax, w, bits=bits)[1].out32 for g in imgs]
    code = hd.HD_U8 if dtype == np.uint8 else hd.HD_U16
    pl = hd.HostPipeline(H, W, code, hd.Params(smax, w, bits=bits), depth=depth)
    outs = []
    for i, g in enumerate(imgs):
        if i % 3 == 0:                       # numpy, padded rows on both sides
            src = np.zeros((H, W + 5), dtype)[:, :W]
            src[:] = g
            out = np.full((H, W + 3), 9, dtype)[:, :W]
        elif i % 3 == 1:                     # pinned tensors
            src = pinned(g)
            out = torch.empty_like(src).pin_memory()
        else:                                # plain numpy
            src = g.copy()
            out = np.zeros_like(g)
        pl.submit(src, out)
        outs.append(out)
    pl.wait()
    assert hd.hd_get_device_error() == hd.HD_OK
    for out, ref in zip(outs, refs):
        o = out.numpy() if isinstance(out, torch.Tensor) else out
        o = o.view(np.uint16) if dtype == np.uint16 else o
        np.testing.assert_array_equal(o, ref)
    pl.close()


def test_pipeline_with_given_noise_variance():
    """A supplied noise variance: the hybrid needs no workspace of its own, so
    the slots start at the front of the pipeline's workspace."""
    H, W = 97, 133
    imgs = [noisy_image(H, W, np.uint8, seed=300 + i) for i in range(5)]
    pl = hd.HostPipeline(H, W, hd.HD_U8, hd.Params(7, 3, noise_var=40.0), depth=2)
    outs = [np.zeros_like(g) for g in imgs]
    for g, o in zip(imgs, outs):
        pl.submit(g, o)
    pl.wait()
    pl.close()
    for g, o in zip(imgs, outs):
        np.testing.assert_array_equal(o, oracle.hybrid(g, 7, 3, noise_var=40.0)[1].out32)


def test_pipeline_argument_errors():
    pl = hd.HostPipeline(40, 50, hd.HD_U8, hd.Params(7, 3), depth=2)
    with pytest.raises(ValueError):
        pl.submit(np.zeros((40, 51), np.uint8), np.zeros((40, 51), np.uint8))
    pl.close()
    with pytest.raises(hd.HDError) as e:
        hd.HostPipeline(40, 50, hd.HD_U8, hd.Params(7, 3), depth=0)
    assert e.value.status == hd.HD_ERR_ARG
    with pytest.raises(hd.HDError) as e:
        hd.HostPipeline(40, 50, hd.HD_U8, hd.Params(8, 3), depth=2)
    assert e.value.status == hd.HD_ERR_SMAX
