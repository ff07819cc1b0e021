"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars (the method's definition fixes them):
  * adaptive median output: bit-exact (integer order statistics);
  * Wiener: the integer output and the binary32 value equal the oracle's
    binary32 twin bit for bit (the rounding decision is taken in the same
    precision on both sides), the noise variance equals the oracle's binary64
    value exactly, and the binary32 value is within maxv * 2^-20 of the binary64
    definition (so the integer output is within 0.5 + maxv * 2^-20 LSB of it).
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


def to_dev(a: np.ndarray, pad: int = 0):
    """Copy a host image to the GPU; pad > 0 gives a row pitch wider than W."""
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a)
    if pad:
        big = torch.zeros((a.shape[0], a.shape[1] + pad), dtype=t.dtype, device=DEV)
        big[:, :a.shape[1]] = t.to(DEV)
        return big[:, :a.shape[1]]
    return t.to(DEV).contiguous()


def empty_like_dev(a: np.ndarray, pad: int = 0):
    dt = torch.uint8 if a.dtype == np.uint8 else torch.int16
    if pad:
        return torch.full((a.shape[0], a.shape[1] + pad), 7, dtype=dt, device=DEV)[:, :a.shape[1]]
    return torch.full(a.shape, 7, dtype=dt, device=DEV)


def to_host(t, dtype) -> np.ndarray:
    a = t.cpu().contiguous().numpy()
    return a.view(np.uint16) if dtype == np.uint16 else a


def noisy_image(H, W, dtype, seed, density=0.4, flat=True):
    rng = np.random.default_rng(seed)
    maxv = 255 if dtype == np.uint8 else 4095
    g = rng.integers(0, maxv + 1, size=(H, W))
    if flat and H > 6 and W > 6:
        g[H // 4:H // 2, W // 4:W // 2] = maxv // 3            # flat patch: growth to Smax
        g[H // 2:, :W // 3] = rng.integers(0, 3, size=g[H // 2:, :W // 3].shape)   # dark, clamped
    u = rng.random((H, W))
    g[u < density / 2] = 0
    g[(u >= density / 2) & (u < density)] = maxv
    return g.astype(dtype)


def gpu_amf(g, smax, unresolved=0, pad=0, bits=None):
    src = to_dev(g, pad)
    dst = empty_like_dev(g, pad)
    hd.amf_filter(src, dst, smax=smax, unresolved=unresolved, bits=bits)
    assert hd.hd_get_device_error() == hd.HD_OK
    return to_host(dst, g.dtype)


def exact_workspace(n):
    """A zeroed workspace whose usable length (after 256-byte alignment) is exactly n."""
    buf = hd._workspace(n, DEV)
    p = buf.data_ptr()
    return buf[:(p + 255) // 256 * 256 - p + n]


def min_workspace(H, W, code, p):
    """A workspace of the least accepted size (no statistics plane)."""
    n = hd.hybrid_min_workspace_size(H, W, code, p)
    return exact_workspace(n) if n else None


def gpu_hybrid(g, smax, w, noise_var=-1.0, border=0, unresolved=0, bits=None, pad=0, want_y=False,
               minimal=False):
    src = to_dev(g, pad)
    dst = empty_like_dev(g, pad)
    nv = torch.full((1,), -7.0, dtype=torch.float64, device=DEV)
    y = torch.empty(g.shape, dtype=torch.float32, device=DEV) if want_y else None
    ws = None
    if minimal:
        code = hd.HD_U8 if g.dtype == np.uint8 else hd.HD_U16
        b = bits if bits is not None else (8 if g.dtype == np.uint8 else 16)
        ws = min_workspace(*g.shape, code, hd.Params(smax, w, noise_var=noise_var, bits=b))
    hd.hybrid_denoise(src, dst, smax=smax, wiener_w=w, noise_var=noise_var, border=border,
                      unresolved=unresolved, bits=bits, noise_var_out=nv, y_out=y, workspace=ws)
    assert hd.hd_get_device_error() == hd.HD_OK
    return to_host(dst, g.dtype), float(nv.item()), (y.cpu().numpy() if want_y else None)


def gpu_wiener(f, w, noise_var=-1.0, border=0, bits=None, pad=0, minimal=False):
    src = to_dev(f, pad)
    dst = empty_like_dev(f, pad)
    nv = torch.full((1,), -7.0, dtype=torch.float64, device=DEV)
    y = torch.empty(f.shape, dtype=torch.float32, device=DEV)
    ws = None
    if minimal and noise_var < 0:
        # the full size less the 8-byte-per-pixel statistics plane (256-byte rounded)
        code = hd.HD_U8 if f.dtype == np.uint8 else hd.HD_U16
        b = bits if bits is not None else (8 if f.dtype == np.uint8 else 16)
        full = hd.wiener_workspace_size(*f.shape, code, hd.Params(3, w, noise_var=noise_var, bits=b))
        ws = exact_workspace(full - (8 * f.shape[0] * f.shape[1] + 255) // 256 * 256)
    hd.wiener_filter(src, dst, wiener_w=w, noise_var=noise_var, border=border, bits=bits, noise_var_out=nv,
                     y_out=y, workspace=ws)
    assert hd.hd_get_device_error() == hd.HD_OK
    return to_host(dst, f.dtype), float(nv.item()), y.cpu().numpy()


def check_wiener(out, nu2, y, ref: "oracle.WienerResult", bits):
    maxv = (1 << bits) - 1
    assert nu2 == ref.nu2
    np.testing.assert_array_equal(out, ref.out32)
    if y is not None:
        np.testing.assert_array_equal(y, ref.y32)
        assert np.max(np.abs(y.astype(np.float64) - ref.y64)) <= maxv * 2.0 ** -20
    assert np.all(np.abs(out.astype(np.float64) - ref.y64) <= 0.5 + maxv * 2.0 ** -20)


SHAPES = [(1, 1), (1, 17), (23, 1), (2, 3), (5, 7), (31, 33), (32, 64), (33, 65), (97, 130), (130, 257)]


# ------------------------------------------------------------------ adaptive median
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_amf_bit_exact_shapes(shape, dtype):
    g = noisy_image(*shape, dtype, seed=shape[0] * 1000 + shape[1])
    for smax in (3, 5, 7, 11, 15):
        for unresolved in (0, 1):
            ref = oracle.amf(g, smax, keep_unresolved=bool(unresolved))
            got = gpu_amf(g, smax, unresolved)
            np.testing.assert_array_equal(got, ref, err_msg=f"smax={smax} unresolved={unresolved}")


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_amf_pitched_rows(dtype):
    g = noisy_image(45, 77, dtype, seed=5)
    ref = oracle.amf(g, 9)
    np.testing.assert_array_equal(gpu_amf(g, 9, pad=19), ref)


def test_amf_full_range_16bit_and_constant():
    rng = np.random.default_rng(12)
    g = rng.integers(0, 65536, size=(70, 90)).astype(np.uint16)
    g[rng.random(g.shape) < 0.3] = 65535
    np.testing.assert_array_equal(gpu_amf(g, 7), oracle.amf(g, 7))
    c = np.full((40, 50), 123, np.uint8)
    np.testing.assert_array_equal(gpu_amf(c, 11), c)


@pytest.mark.parametrize("tile", [(16, 0), (24, 1), (32, 0), (64, 3), (128, 0)])
def test_amf_independent_of_tiling(tile):
    g = noisy_image(150, 211, np.uint16, seed=9)
    ref = oracle.amf(g, 11)
    old = hd.hd_get_tuning()
    try:
        hd.hd_set_tuning(*tile)
        np.testing.assert_array_equal(gpu_amf(g, 11), ref)
        f, nu2, _ = gpu_hybrid(g, 11, 5, bits=12)
        _, r = oracle.hybrid(g, 11, 5, bits=12)
        assert nu2 == r.nu2
        np.testing.assert_array_equal(f, r.out32)
    finally:
        hd.hd_set_tuning(*old)


# ------------------------------------------------------------------ Wiener
@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (7, 7), (33, 65), (130, 257)])
@pytest.mark.parametrize("dtype,bits", [(np.uint8, 8), (np.uint16, 12), (np.uint16, 16)])
def test_wiener_matches_oracle(shape, dtype, bits):
    rng = np.random.default_rng(shape[0] + 7 * shape[1] + bits)
    maxv = (1 << bits) - 1
    f = rng.integers(0, maxv + 1, size=shape).astype(dtype)
    for w in (1, 3, 5, 7, 15):
        for border in (0, 1):
            for nv in (-1.0, 0.0, 37.5, 1e9):
                ref = oracle.wiener(f, w, noise_var=nv, bits=bits, border_zero=bool(border))
                out, nu2, y = gpu_wiener(f, w, noise_var=nv, border=border, bits=bits)
                check_wiener(out, nu2, y, ref, bits)


# ------------------------------------------------------------------ hybrid
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype,bits", [(np.uint8, 8), (np.uint16, 12)])
def test_hybrid_matches_oracle(shape, dtype, bits):
    g = noisy_image(*shape, dtype, seed=3 * shape[0] + shape[1])
    for smax, w in ((3, 3), (5, 7), (11, 5), (15, 15)):
        for nv in (-1.0, 50.0):
            for border in (0, 1):
                f, ref = oracle.hybrid(g, smax, w, noise_var=nv, bits=bits, border_zero=bool(border))
                out, nu2, y = gpu_hybrid(g, smax, w, noise_var=nv, border=border, bits=bits, want_y=True)
                check_wiener(out, nu2, y, ref, bits)


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (31, 33), (33, 65), (130, 257)])
@pytest.mark.parametrize("dtype,bits", [(np.uint8, 8), (np.uint16, 12), (np.uint16, 16)])
def test_recompute_path_matches_oracle(shape, dtype, bits):
    """With the least workspace (no statistics plane) the Wiener pass
    recomputes the window sums; the output is the same as the oracle's."""
    g = noisy_image(*shape, dtype, seed=5 * shape[0] + shape[1])
    for smax, w in ((3, 3), (7, 5), (15, 15)):
        for border in (0, 1):
            f, ref = oracle.hybrid(g, smax, w, noise_var=-1.0, bits=bits, border_zero=bool(border))
            out, nu2, y = gpu_hybrid(g, smax, w, border=border, bits=bits, want_y=True, minimal=True)
            check_wiener(out, nu2, y, ref, bits)
            ref_w = oracle.wiener(f, w, noise_var=-1.0, bits=bits, border_zero=bool(border))
            out, nu2, y = gpu_wiener(f, w, border=border, bits=bits, minimal=True)
            check_wiener(out, nu2, y, ref_w, bits)


@pytest.mark.parametrize("plane", [2, 3])
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (31, 33), (33, 65), (130, 257), (257, 130)])
@pytest.mark.parametrize("dtype,bits", [(np.uint8, 8), (np.uint16, 12)])
def test_plane_pass_staged_and_direct_match_oracle(plane, shape, dtype, bits):
    """The Wiener pass from the statistics plane, forced to stage it in shared
    memory (plane knob 2) or to read it straight from L2 (3), on ragged shapes,
    pitched buffers, both borders, with the binary32 value."""
    g = noisy_image(*shape, dtype, seed=11 * shape[0] + shape[1] + plane)
    old = hd.hd_get_tuning()
    try:
        hd.hd_set_tuning(old[0], old[1], plane, *old[3:])
        for smax, w, pad in ((3, 3, 0), (7, 5, 5), (11, 7, 1)):
            for border in (0, 1):
                f, ref = oracle.hybrid(g, smax, w, bits=bits, border_zero=bool(border))
                out, nu2, y = gpu_hybrid(g, smax, w, border=border, bits=bits, pad=pad, want_y=True)
                check_wiener(out, nu2, y, ref, bits)
                ref_w = oracle.wiener(f, w, noise_var=-1.0, bits=bits, border_zero=bool(border))
                out, nu2, y = gpu_wiener(f, w, border=border, bits=bits, pad=pad)
                check_wiener(out, nu2, y, ref_w, bits)
    finally:
        hd.hd_set_tuning(*old)


def test_plane_pass_staged_direct_and_recompute_identical():
    """paper1620 (the plane's working set fits L2: read straight from it by
    default) through all three Wiener passes."""
    spec, clean, g = synth.config_image("paper1620")
    old = hd.hd_get_tuning()
    try:
        outs = []
        for plane in (2, 3):
            hd.hd_set_tuning(old[0], old[1], plane, *old[3:])
            outs.append(gpu_hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits, want_y=True))
    finally:
        hd.hd_set_tuning(*old)
    outs.append(gpu_hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits, want_y=True, minimal=True))
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0][0], o[0])
        assert outs[0][1] == o[1]
        np.testing.assert_array_equal(outs[0][2], o[2])


def test_plane_and_recompute_paths_identical():
    spec, clean, g = synth.config_image("paper1620")
    a = gpu_hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits, want_y=True)
    b = gpu_hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits, want_y=True, minimal=True)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1] == b[1]
    np.testing.assert_array_equal(a[2], b[2])


def test_hybrid_pitched_and_repeated_workspace():
    g = noisy_image(100, 140, np.uint16, seed=21)
    f, ref = oracle.hybrid(g, 9, 5, bits=12)
    src = to_dev(g, 24)
    dst = empty_like_dev(g, 8)
    ws = hd._workspace(hd.hybrid_workspace_size(100, 140, hd.HD_U16, hd.Params(9, 5, bits=12)), DEV)
    for _ in range(3):
        hd.hybrid_denoise(src, dst, smax=9, wiener_w=5, bits=12, workspace=ws)
        assert hd.hd_get_device_error() == hd.HD_OK
        np.testing.assert_array_equal(to_host(dst, np.uint16), ref.out32)


@pytest.mark.parametrize("name", ["plain512", "paper1620"])
def test_configs_full_image(name):
    spec, clean, g = synth.config_image(name)
    f, ref = oracle.hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits)
    np.testing.assert_array_equal(gpu_amf(g, spec.smax), f)
    out, nu2, y = gpu_hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits, want_y=True)
    check_wiener(out, nu2, y, ref, spec.bits)


def test_stress4096_full_image():
    spec, clean, g = synth.config_image("stress4096")
    f, ref = oracle.hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits)
    np.testing.assert_array_equal(gpu_amf(g, spec.smax), f)
    out, nu2, y = gpu_hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits, want_y=True)
    check_wiener(out, nu2, y, ref, spec.bits)


# ------------------------------------------------------------------ host entry point
def test_hybrid_host_buffers():
    g = noisy_image(77, 101, np.uint8, seed=4)
    _, ref = oracle.hybrid(g, 7, 3)
    out = np.zeros_like(g)
    hd.hybrid_denoise_host(g, out, smax=7, wiener_w=3)
    np.testing.assert_array_equal(out, ref.out32)
    g16 = noisy_image(64, 80, np.uint16, seed=6)
    _, ref16 = oracle.hybrid(g16, 11, 5, bits=12)
    out16 = np.zeros_like(g16)
    hd.hybrid_denoise_host(g16, out16, smax=11, wiener_w=5, bits=12)
    np.testing.assert_array_equal(out16, ref16.out32)


def test_hybrid_host_buffers_with_row_padding():
    """Host rows wider than the image (views into padded arrays): the copies
    move row by row instead of as one block; tight and padded buffers mixed."""
    for dtype, bits, (H, W) in ((np.uint8, 8, (61, 93)), (np.uint16, 12, (45, 70))):
        g = noisy_image(H, W, dtype, seed=9)
        _, ref = oracle.hybrid(g, 9, 5, bits=bits)
        gp = np.zeros((H, W + 13), dtype)
        gp[:, :W] = g
        for src in (g, gp[:, :W]):
            for pad in (0, 7):
                big = np.full((H, W + pad), 5, dtype)
                out = big[:, :W]
                hd.hybrid_denoise_host(src, out, smax=9, wiener_w=5, bits=bits)
                np.testing.assert_array_equal(out, ref.out32)
                assert (big[:, W:] == 5).all()


# ------------------------------------------------------------------ batches
def _batch_items(n, seed):
    rng = np.random.default_rng(seed)
    items, hosts = [], []
    for i in range(n):
        H, W = int(rng.integers(1, 300)), int(rng.integers(1, 300))
        dtype = np.uint8 if i % 3 == 0 else np.uint16
        bits = 8 if dtype == np.uint8 else int(rng.choice([10, 12, 16]))
        g = noisy_image(H, W, dtype, seed=seed * 100 + i, density=float(rng.uniform(0, 0.6)))
        if bits == 10:
            g = np.minimum(g, 1023).astype(np.uint16)
        p = hd.Params(int(rng.choice([3, 5, 7, 9, 11])), int(rng.choice([1, 3, 5, 7])),
                      float(rng.choice([-1.0, -1.0, 20.0])), int(rng.integers(0, 2)), int(rng.integers(0, 2)),
                      bits)
        src, dst = to_dev(g), empty_like_dev(g)
        items.append((src, dst, p))
        hosts.append(g)
    return items, hosts


def _oracle_of(g, p):
    return oracle.hybrid(g, p.smax, p.wiener_w, noise_var=p.noise_var, bits=p.bits,
                         keep_unresolved=bool(p.unresolved), border_zero=bool(p.border))[1]


def test_batched_equals_single_and_oracle():
    items, hosts = _batch_items(24, seed=77)
    hd.hybrid_denoise_batched(items)
    assert hd.hd_get_device_error() == hd.HD_OK
    for (src, dst, p), g in zip(items, hosts):
        batched = to_host(dst, g.dtype)
        ref = _oracle_of(g, p)
        np.testing.assert_array_equal(batched, ref.out32)
        single = empty_like_dev(g)
        hd.hybrid_denoise(src, single, p.smax, p.wiener_w, p.noise_var, p.border, p.unresolved, p.bits)
        np.testing.assert_array_equal(to_host(single, g.dtype), batched)


def test_batch_of_many_small_images():
    """600 images of 1..40 pixels a side with estimated noise variance: 1200
    segments of tickets, so the kernel's 32-way segment search takes three
    rounds; the images finish in a few tiles each, so many items of many
    images are in flight at once."""
    rng = np.random.default_rng(606)
    items, hosts = [], []
    for i in range(600):
        H, W = int(rng.integers(1, 41)), int(rng.integers(1, 41))
        dtype = np.uint8 if i % 2 == 0 else np.uint16
        bits = 8 if dtype == np.uint8 else 12
        g = noisy_image(H, W, dtype, seed=60600 + i, density=float(rng.uniform(0, 0.5)))
        p = hd.Params(int(rng.choice([3, 5, 7])), int(rng.choice([1, 3, 5])), -1.0, int(rng.integers(0, 2)), 0,
                      bits)
        items.append((to_dev(g), empty_like_dev(g), p))
        hosts.append(g)
    hd.hybrid_denoise_batched(items)
    assert hd.hd_get_device_error() == hd.HD_OK
    for (src, dst, p), g in zip(items, hosts):
        np.testing.assert_array_equal(to_host(dst, g.dtype), _oracle_of(g, p).out32)
    plan = hd.BatchPlan(items)
    try:
        for _, dst, _ in items:
            dst.fill_(3)
        plan.launch()
        assert hd.hd_get_device_error() == hd.HD_OK
        for (src, dst, p), g in zip(items, hosts):
            np.testing.assert_array_equal(to_host(dst, g.dtype), _oracle_of(g, p).out32)
    finally:
        plan.close()


def test_batch_plan_graph_replay():
    items, hosts = _batch_items(10, seed=5)
    plan = hd.BatchPlan(items)
    for rep in range(3):
        for _, dst, _ in items:
            dst.fill_(3)
        plan.launch()
        assert hd.hd_get_device_error() == hd.HD_OK
        for (src, dst, p), g in zip(items, hosts):
            np.testing.assert_array_equal(to_host(dst, g.dtype), _oracle_of(g, p).out32)
    plan.close()


# ------------------------------------------------------------------ bounded waits
def test_wait_timeout_is_reported_and_recoverable():
    """A spin limit of one poll makes the Wiener tiles give up waiting for the
    median tiles: the kernel returns, the error word says TIMEOUT, and the
    context stays usable."""
    g = noisy_image(2048, 2048, np.uint16, seed=1, density=0.3)
    src, dst = to_dev(g), empty_like_dev(g)
    try:
        hd.hd_set_spin_limit(1)
        hd.hybrid_denoise(src, dst, smax=11, wiener_w=5, bits=12)
        assert hd.hd_get_device_error() == hd.HD_ERR_TIMEOUT
    finally:
        hd.hd_set_spin_limit(0)
    assert hd.hd_get_device_error() == hd.HD_OK
    small = noisy_image(64, 64, np.uint8, seed=2)
    _, ref = oracle.hybrid(small, 5, 3)
    out, _, _ = gpu_hybrid(small, 5, 3)
    np.testing.assert_array_equal(out, ref.out32)


def test_launches_with_varying_shared_memory():
    """Launch sizes above 48 KB of shared memory in the order large, small,
    middle, large: every launch must keep a valid dynamic shared-memory limit
    (the limit only grows)."""
    old = hd.hd_get_tuning()
    try:
        hd.hd_set_tuning(64, 0)
        g = noisy_image(90, 150, np.uint16, seed=44)
        for smax in (15, 11, 13, 15, 9, 15):
            f, ref = oracle.hybrid(g, smax, 5, bits=12)
            out, nu2, _ = gpu_hybrid(g, smax, 5, bits=12)
            check_wiener(out, nu2, None, ref, 12)
    finally:
        hd.hd_set_tuning(*old)
