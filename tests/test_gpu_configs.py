"""Parity with the oracle on the batched and served workloads at their own sizes.

* The batched workload: all 256 uneven 12-bit slices (256^2 .. 1024^2, Smax
  up to 11, Wiener window up to 7, salt & pepper density up to 0.5), through
  one batched launch, through a replayed batch plan and through the batch
  pipeline from host buffers.
* The served workload: a pool of images 512^2 .. 4096^2, uint8 and 12-bit,
  density up to 0.3, through the continuous-batching server.

Every result is compared with the oracle (run on every host core, one image
per worker): the integer output and the binary32 value bit for bit (by
SHA-256 of the arrays), the noise variance exactly, and the binary32 value
within maxv * 2^-20 of the binary64 definition.  The count of pixels whose
integer output differs from round-half-up of the binary64 value is reported.
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
from oracle import parallel  # noqa: E402

DEV = "cuda:0"


def _t(a: np.ndarray):
    return torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a)


def _host(t, dtype) -> np.ndarray:
    a = t.cpu().contiguous().numpy()
    return a.view(np.uint16) if dtype == np.uint16 else a


def _params(spec):
    return hd.Params(spec.smax, spec.wiener_w, -1.0, hd.HD_BORDER_SYMMETRIC, hd.HD_UNRESOLVED_ZMED, spec.bits)


def _check_against(refs, outs, ys=None, nu2s=None, specs=None):
    """outs / ys: host arrays per image; refs: the oracle workers' records."""
    bad = [i for i, (r, o) in enumerate(zip(refs, outs)) if parallel.digest(o) != r["out32_sha"]]
    assert not bad, f"images whose output differs from the oracle: {bad[:10]}"
    if ys is not None:
        bad = [i for i, (r, y) in enumerate(zip(refs, ys)) if parallel.digest(y) != r["y32_sha"]]
        assert not bad, f"images whose binary32 value differs from the oracle's: {bad[:10]}"
    if nu2s is not None:
        bad = [i for i, (r, v) in enumerate(zip(refs, nu2s)) if v != r["nu2"]]
        assert not bad, f"images whose noise variance differs: {bad[:10]}"
    if specs is not None:
        for r, s in zip(refs, specs):
            assert r["max_err_y32_y64"] <= s.maxv * 2.0 ** -20
    rounding = sum(r["round_diff"] for r in refs)
    px = sum(r["pixels"] for r in refs)
    print(f"max |y32 - y64| = {max(r['max_err_y32_y64'] for r in refs):.3e} LSB; "
          f"{rounding} of {px} pixels differ from round(y64)")


@pytest.fixture(scope="module")
def batch():
    specs = synth.batch_specs(256, master_seed=400)
    hosts = [s.noisy() for s in specs]
    refs = parallel.run_specs(specs)
    return specs, hosts, refs


def test_batched_workload_full_size(batch):
    specs, hosts, refs = batch
    items, ys = [], []
    nv = torch.full((len(specs),), -7.0, dtype=torch.float64, device=DEV)
    for i, (s, g) in enumerate(zip(specs, hosts)):
        src = _t(g).to(DEV)
        dst = torch.full_like(src, 5)
        y = torch.empty(g.shape, dtype=torch.float32, device=DEV)
        items.append(hd.make_image(src, dst, _params(s), nv[i:i + 1], y))
        ys.append((src, dst, y))
    hd.hybrid_denoise_batched(items)
    assert hd.hd_get_device_error() == hd.HD_OK
    outs = [_host(d, np.uint16) for _, d, _ in ys]
    _check_against(refs, outs, [y.cpu().numpy() for _, _, y in ys], nv.cpu().tolist(), specs)
    # the same slices replayed from a batch plan (CUDA graph), twice
    plan = hd.BatchPlan(items)
    try:
        for _ in range(2):
            for _, d, _ in ys:
                d.fill_(9)
            plan.launch()
            assert hd.hd_get_device_error() == hd.HD_OK
            _check_against(refs, [_host(d, np.uint16) for _, d, _ in ys])
    finally:
        plan.close()


def test_batch_pipeline_host_buffers_full_size(batch):
    specs, hosts, refs = batch
    pipe = hd.BatchPipeline([(s.H, s.W, hd.HD_U16, _params(s)) for s in specs], depth=2)
    try:
        # all slices in one pinned buffer, back to back: one copy each way a step
        sizes = [g.size for g in hosts]
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        h_in = torch.empty(int(offs[-1]), dtype=torch.int16).pin_memory()
        for g, o in zip(hosts, offs[:-1]):
            h_in[int(o):int(o) + g.size].copy_(_t(g).reshape(-1))
        srcs = [h_in[int(o):int(o) + s.H * s.W].view(s.H, s.W) for s, o in zip(specs, offs[:-1])]
        outs = []
        for step in range(3):
            h_out = torch.full((int(offs[-1]),), 3, dtype=torch.int16).pin_memory()
            dsts = [h_out[int(o):int(o) + s.H * s.W].view(s.H, s.W) for s, o in zip(specs, offs[:-1])]
            pipe.submit(srcs, dsts)
            outs.append(dsts)
        pipe.wait()
        assert hd.hd_get_device_error() == hd.HD_OK
        for dsts in outs:
            _check_against(refs, [d.numpy().view(np.uint16) for d in dsts])
    finally:
        pipe.close()


def test_served_workload_images_against_oracle():
    """Served pool images (512^2 .. 4096^2, uint8 and 12-bit) through the
    continuous-batching server, each result against the oracle."""
    from paper_2005_05371_gb300.serve import Server, poisson_arrivals
    import time
    specs = synth.served_specs(12, seed=501)
    hosts = [s.noisy() for s in specs]
    refs = parallel.run_specs(specs)
    pinned = [_t(g).pin_memory() for g in hosts]
    outs = [torch.empty_like(p).pin_memory() for p in pinned]
    srv = Server(budget_bytes=2 << 30, max_inflight=3, device=DEV)
    try:
        t0 = time.perf_counter()
        reqs = []
        for i, t in enumerate(poisson_arrivals(2000.0, len(specs), 7)):
            wait = t - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            reqs.append(srv.submit(pinned[i], _params(specs[i]), outs[i]))
        for r in reqs:
            assert r.done.wait(300)
            assert r.error is None, r.error
    finally:
        srv.close()
    assert hd.hd_get_device_error() == hd.HD_OK
    got = [o.numpy().view(np.uint16) if s.dtype == "u16" else o.numpy() for o, s in zip(outs, specs)]
    _check_against(refs, got, specs=specs)
