"""One image split into row-strip parts (hybrid_part_stats / hybrid_part_apply)
on one GPU: the parts run one after another through the C ABI, their four
sums are added on the device (what the all-reduce does across GPUs), and the
reassembled image must equal the oracle's whole-image hybrid bit for bit
(and hybrid_denoise of the whole image).  Covers strips thinner than the
halo, odd widths (the statistics plane's pair alignment), 8-, 12- and 16-bit
images, both border rules, the literal unresolved rule and the largest
windows."""
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
from paper_2005_05371_gb300 import split  # noqa: E402

DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int16) if a.dtype == np.uint16 else np.ascontiguousarray(a))


def run_parts(g, P, p):
    """The P parts of g one after another; returns the reassembled result."""
    H, W = g.shape
    halo = hd.part_halo_rows(p)
    tg = _t(g).to(DEV)
    backends, bufs, parts = [], [], split.all_parts(H, P, halo)
    total = torch.zeros(4, dtype=torch.int64, device=DEV)
    for me in parts:
        be = split.CudaPartBackend()
        buf = tg[me.buf0:me.buf1].clone()
        total += be.stats(buf, me, H, W, p)
        backends.append(be)
        bufs.append(buf)
    outs = [be.apply(buf, me, H, W, p, total.clone()) for be, buf, me in zip(backends, bufs, parts)]
    assert hd.hd_get_device_error() == hd.HD_OK
    out = torch.cat(outs).cpu().numpy()
    return out.view(np.uint16) if g.dtype == np.uint16 else out, total.cpu().numpy()


def _noisy(H, W, bits, seed, density=0.3):
    rng = np.random.default_rng(seed)
    maxv = (1 << bits) - 1
    g = rng.integers(0, maxv + 1, size=(H, W))
    g[H // 4:H // 2, W // 4:W // 2] = maxv // 3
    u = rng.random((H, W))
    g[u < density / 2] = 0
    g[(u >= density / 2) & (u < density)] = maxv
    return g.astype(np.uint8 if bits == 8 else np.uint16)


@pytest.mark.parametrize("H,W,bits,smax,w,P,border,unres", [
    (200, 131, 8, 9, 5, 2, 0, 0),
    (97, 64, 12, 11, 5, 4, 0, 0),
    (61, 45, 12, 15, 15, 5, 0, 0),     # strips of 12 rows, halo 14
    (130, 257, 16, 7, 3, 3, 0, 0),     # full 16-bit range: the scalar median path
    (90, 77, 8, 7, 7, 3, 1, 0),        # zero border
    (75, 50, 12, 5, 3, 7, 0, 1),       # unresolved pixels keep their input
    (3, 40, 8, 5, 3, 3, 0, 0),         # one row per part
])
def test_parts_equal_the_whole_image(H, W, bits, smax, w, P, border, unres):
    g = _noisy(H, W, bits, seed=H * 31 + W)
    p = hd.Params(smax, w, -1.0, border, unres, bits)
    out, words = run_parts(g, P, p)
    _, ref = oracle.hybrid(g, smax, w, bits=bits, keep_unresolved=bool(unres), border_zero=bool(border))
    np.testing.assert_array_equal(out, ref.out32)
    A, B = split.sums_total(words)
    assert w * w * B - A == ref.sumD
    whole = torch.empty_like(_t(g).to(DEV))
    hd.hybrid_denoise(_t(g).to(DEV), whole, smax, w, -1.0, border, unres, bits)
    np.testing.assert_array_equal(out, whole.cpu().numpy().view(np.uint16) if bits > 8 else whole.cpu().numpy())


@pytest.mark.parametrize("P", [2, 4, 8])
def test_parts_of_the_paper_sized_image(P):
    spec, _, g = synth.config_image("paper1620")
    p = hd.Params(spec.smax, spec.wiener_w, bits=spec.bits)
    out, _ = run_parts(g, P, p)
    _, ref = oracle.hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits)
    np.testing.assert_array_equal(out, ref.out32)


def test_parts_of_the_stress_image_equal_hybrid_denoise():
    """4096 x 4096 12-bit, density 0.40, Smax 11 in 4 parts against the
    whole-image hybrid (itself bit-exact against the oracle in the parity tests)."""
    spec, _, g = synth.config_image("stress4096")
    p = hd.Params(spec.smax, spec.wiener_w, bits=spec.bits)
    out, _ = run_parts(g, 4, p)
    src = _t(g).to(DEV)
    whole = torch.empty_like(src)
    hd.hybrid_denoise(src, whole, spec.smax, spec.wiener_w, bits=spec.bits)
    np.testing.assert_array_equal(out, whole.cpu().numpy().view(np.uint16))


def test_part_calls_again_on_the_same_workspace():
    """A part's workspace serves later calls of any part (the statistics call
    clears its sums first)."""
    g = _noisy(120, 90, 12, seed=5)
    p = hd.Params(9, 5, bits=12)
    first, _ = run_parts(g, 3, p)
    second, _ = run_parts(g, 3, p)
    np.testing.assert_array_equal(first, second)
