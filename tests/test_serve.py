"""Continuous-batching server: every result in the mix equals the same image
denoised alone; admission never exceeds the device-memory budget."""
import numpy as np
import pytest

from tests._lib import ensure_built

torch = pytest.importorskip("torch")


def test_arena_first_fit_and_merge():
    ensure_built()
    from paper_2005_05371_gb300.serve import DeviceArena
    a = DeviceArena(4096, buffer=torch.zeros(4096, dtype=torch.uint8))
    x = a.alloc(1000)
    y = a.alloc(1000)
    z = a.alloc(1000)
    assert x == (0, 1024) and y == (1024, 1024) and z == (2048, 1024)
    assert a.alloc(2000) is None                 # only 1024 left
    a.release(*y)
    assert a.alloc(600) == (1024, 768)           # first fit reuses the hole
    a.release(*x)
    a.release(1024, 768)
    a.release(*z)
    assert a.used == 0 and a.free == [(0, 4096)]  # holes merged back


gpu = pytest.mark.gpu


def _pool(seed, n):
    rng = np.random.default_rng(seed)
    pool, specs = [], []
    for i in range(n):
        side_h, side_w = int(rng.integers(40, 700)), int(rng.integers(40, 700))
        if i % 2:
            g = rng.integers(0, 4096, size=(side_h, side_w)).astype(np.uint16)
            g[rng.random(g.shape) < 0.25] = 4095
            t = torch.from_numpy(g.view(np.int16)).pin_memory()
            bits = 12
        else:
            g = rng.integers(0, 256, size=(side_h, side_w)).astype(np.uint8)
            g[rng.random(g.shape) < 0.25] = 0
            t = torch.from_numpy(g).pin_memory()
            bits = 8
        pool.append(t)
        specs.append(bits)
    return pool, specs


@gpu
def test_served_results_equal_alone_results():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    ensure_built()
    import paper_2005_05371_gb300 as hd
    from paper_2005_05371_gb300.serve import Server, poisson_arrivals, replay
    pool, bits = _pool(3, 12)
    params = [hd.Params(int(s), int(w), -1.0 if i % 3 else 30.0, 0, 0, b)
              for i, (s, w, b) in enumerate(zip([5, 7, 9, 11] * 3, [3, 5, 7] * 4, bits))]
    srv = Server(budget_bytes=256 << 20, max_inflight=3)
    try:
        reqs = replay(srv, pool, poisson_arrivals(20000.0, 60, 5), lambda i: params[i % len(pool)],
                      want_results=True)
        for r in reqs:
            assert r.done.wait(60)
        st = srv.stats()
    finally:
        srv.close()
    assert st["requests"] == 60 and st["rejected"] == 0
    assert st["rounds"] < 60                      # requests were batched together
    for r in reqs:
        i = r.rid % len(pool)
        src = pool[i].cuda()
        alone = torch.empty_like(src)
        p = params[i]
        hd.hybrid_denoise(src, alone, p.smax, p.wiener_w, p.noise_var, p.border, p.unresolved, p.bits)
        torch.testing.assert_close(r.out, alone.cpu(), rtol=0, atol=0)


@gpu
def test_admission_respects_budget_and_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    ensure_built()
    import paper_2005_05371_gb300 as hd
    from paper_2005_05371_gb300.serve import Server, poisson_arrivals, replay
    pool, bits = _pool(4, 8)
    budget = 6 << 20
    srv = Server(budget_bytes=budget, max_inflight=2)
    try:
        reqs = replay(srv, pool, poisson_arrivals(50000.0, 40, 6), lambda i: hd.Params(7, 5, bits=bits[i % 8]))
        big = torch.zeros((2048, 2048), dtype=torch.int16).pin_memory()
        rej = srv.submit(big, hd.Params(7, 5, bits=12))
        for r in reqs:
            assert r.done.wait(60)
        st = srv.stats()
    finally:
        srv.close()
    assert rej.error is not None
    assert st["requests"] == 40
    assert st["peak_device_bytes"] <= budget
    assert hd.hd_get_device_error() == hd.HD_OK
