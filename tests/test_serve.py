"""Continuous-batching server: every result in the mix equals the same image
denoised alone; admission never exceeds the device-memory budget."""
import time

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


class _FakeEvent:
    def __init__(self, polls):
        self.polls = polls

    def query(self):
        self.polls -= 1
        return self.polls <= 0


class _FakeBackend:
    """The server's device side without a GPU: a round completes after a few
    polls; every launch checks that the arena regions it uses (each request's
    block and the round's workspace) overlap no region of a round in flight."""

    def __init__(self, seed):
        self.rng = np.random.default_rng(seed)
        self.live = []          # (lo, hi, round id) of regions in flight
        self.launches = []
        self.round_px = []      # pixels of each round, in launch order
        self.overlaps = 0

    def thread_init(self):
        pass

    def arena(self, nbytes):
        from paper_2005_05371_gb300.serve import DeviceArena
        return DeviceArena(nbytes, allocate=False)

    @staticmethod
    def workspace_bytes(reqs):
        # like the batched workspace: tables plus a median plane per image
        return 4096 + sum(r.shape[0] * ((r.shape[1] * r.elem + 15) // 16 * 16) for r in reqs)

    def launch(self, arena, reqs, ws_off, ws_len, si):
        rid = len(self.launches)
        regions = [(r.dev["alloc"][0], r.dev["alloc"][0] + r.dev["alloc"][1]) for r in reqs]
        own = len(reqs) == 1 and ws_off == reqs[0].dev["ws"]
        if not own:
            regions.append((ws_off, ws_off + ws_len))
        else:
            assert ws_off + ws_len <= regions[0][1]          # inside the request's own block
        self.live = [x for x in self.live if not x[3].polls <= 0]
        for lo, hi in regions:
            assert 0 <= lo < hi <= arena.size
            for a, b, _, _ in self.live:
                if lo < b and a < hi:
                    self.overlaps += 1
        ev = _FakeEvent(int(self.rng.integers(1, 6)))
        self.live += [(lo, hi, rid, ev) for lo, hi in regions]
        self.launches.append((len(reqs), own, si))
        self.round_px.append(sum(r.pixels for r in reqs))
        return ev


def test_scheduler_finishes_every_request_in_a_fragmented_arena():
    """A small arena and a seeded mix of sizes: requests of every size are
    admitted and finish, rounds never share arena space, and rounds of one
    request in its own block keep the scheduler going when no gap can hold a
    round's workspace (no GPU: the device side is a fake)."""
    ensure_built()
    from paper_2005_05371_gb300 import Params
    from paper_2005_05371_gb300.serve import Server
    rng = np.random.default_rng(11)
    fake = _FakeBackend(12)
    srv = Server(budget_bytes=3 << 20, max_inflight=3, backend=fake)
    try:
        reqs = []
        for i in range(300):
            H, W = int(rng.integers(8, 700)), int(rng.integers(8, 700))
            dt = np.uint8 if rng.random() < 0.5 else np.uint16
            reqs.append(srv.submit(np.zeros((H, W), dt), Params(7, 5, bits=8 if dt == np.uint8 else 12)))
            if rng.random() < 0.3:
                time.sleep(0.0005)
        for r in reqs:
            assert r.done.wait(30), "a request never finished"
        st = srv.stats()
    finally:
        srv.close()
    too_big = [r for r in reqs if r.error is not None]
    assert all(r.dev["block"] > srv.arena.size for r in too_big)
    assert st["requests"] == len(reqs) - len(too_big) > 250
    assert fake.overlaps == 0
    assert srv.arena.used == 0 and srv.arena.free == [(0, srv.arena.size)]
    assert st["peak_device_bytes"] <= srv.arena.size
    assert st["solo_rounds"] > 0 and st["rounds"] < st["requests"]
    busy_streams = [si for _, _, si in fake.launches]
    assert set(busy_streams) <= {0, 1, 2}


def test_rounds_hold_at_most_the_pixel_cap():
    """After a burst, rounds take admitted requests in order up to the pixel
    cap (a request larger than the cap runs alone), so no round holds the
    whole backlog."""
    ensure_built()
    from paper_2005_05371_gb300 import Params
    from paper_2005_05371_gb300.serve import Server
    rng = np.random.default_rng(12)
    fake = _FakeBackend(13)
    cap = 300_000
    srv = Server(budget_bytes=64 << 20, max_inflight=2, backend=fake, max_round_px=cap)
    try:
        sizes = [(int(rng.integers(50, 400)), int(rng.integers(50, 400))) for _ in range(200)]
        sizes[7] = (700, 700)                       # larger than the cap alone
        reqs = [srv.submit(np.zeros(hw, np.uint8), Params(5, 3, bits=8)) for hw in sizes]
        for r in reqs:
            assert r.done.wait(30), "a request never finished"
    finally:
        srv.close()
    assert fake.overlaps == 0 and all(r.error is None for r in reqs)
    assert sum(n for n, _, _ in fake.launches) == len(reqs)
    for (n, _, _), px in zip(fake.launches, fake.round_px):
        assert px <= cap or n == 1            # only a lone request may exceed the cap
    assert any(n > 1 for n, _, _ in fake.launches)           # rounds still batch
    assert 700 * 700 in fake.round_px                         # the large one ran alone


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
