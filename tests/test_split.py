"""One image split across ranks by row strips (host logic, CPU ranks over gloo).

`paper_2005_05371_gb300.split` owns the row bounds, the halo exchange and the
all-reduce of the four exact sums between the statistics and apply calls.
Here the device calls are replaced by a stand-in built on the oracle (test
infrastructure), so the host logic runs on CPU ranks: world sizes 2 and 3,
strips thinner than the halo, 8- and 12-bit images, both border rules.  Each
rank checks that its buffer holds exactly its rows of the image, the reduced
sum of local variances equals the whole image's, and the reassembled result
equals the oracle's whole-image hybrid bit for bit.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleParts:
    """Stand-in for the device calls: the same sums and rows from the oracle.

    stats: the oracle's median of the part's buffer (its edges reflect only
    where the buffer ends at the image's edge), then S1 and S2 of the own rows;
    the words carry A = sum S1^2 and S = sum S2 (whose total gives the image's
    sum of D = n S - A).  apply: the Wiener filter of the buffer's median with
    the noise variance of the summed words, own rows kept."""

    def __init__(self, border_zero):
        self.border_zero = border_zero

    def halo_rows(self, p):
        return p.smax // 2 + p.wiener_w // 2

    def _median(self, buf, p):
        import oracle
        a = buf.numpy()
        return oracle.amf(a.view(np.uint16) if a.dtype == np.int16 else a, p.smax)

    def stats(self, buf, me, H, W, p):
        import oracle
        f = self._median(buf, p)
        S1, D = oracle.wiener_stats(f, p.wiener_w, border_zero=self.border_zero)
        n = p.wiener_w ** 2
        own = slice(me.own0 - me.buf0, me.own1 - me.buf0)
        s1 = [int(x) for x in S1[own].ravel()]
        d = [int(x) for x in D[own].ravel()]
        A = sum(x * x for x in s1)
        S = sum((dd + x * x) // n for dd, x in zip(d, s1))
        m = (1 << 32) - 1
        return torch.tensor([A & m, A >> 32, S & m, S >> 32], dtype=torch.int64)

    def apply(self, buf, me, H, W, p, sums):
        import oracle
        from paper_2005_05371_gb300.split import sums_total
        A, S = sums_total(sums.numpy())
        n = p.wiener_w ** 2
        nu2 = float(n * S - A) / float(n * n * H * W)
        f = self._median(buf, p)
        r = oracle.wiener(f, p.wiener_w, noise_var=nu2, bits=p.bits, border_zero=self.border_zero)
        out = r.out32[me.own0 - me.buf0:me.own1 - me.buf0]
        return torch.from_numpy(out.view(np.int16) if out.dtype == np.uint16 else out.copy())


def _image(H, W, bits, seed):
    rng = np.random.default_rng(seed)
    maxv = (1 << bits) - 1
    g = rng.integers(0, maxv + 1, size=(H, W))
    g[H // 4:H // 2, W // 4:W // 2] = maxv // 3
    u = rng.random((H, W))
    g[u < 0.15] = 0
    g[(u >= 0.15) & (u < 0.3)] = maxv
    return g.astype(np.uint8 if bits == 8 else np.uint16)


def _rank_main(rank, world, port, case, q):
    try:
        import torch.distributed as dist
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import oracle
        from paper_2005_05371_gb300 import Params
        from paper_2005_05371_gb300 import split
        H, W, bits, smax, w, bz = case
        g = _image(H, W, bits, seed=H * 7 + W)
        p = Params(smax, w, -1.0, int(bz), 0, bits)
        halo = smax // 2 + w // 2
        me = split.part_rows(H, world, rank, halo)
        tg = torch.from_numpy(g.view(np.int16) if g.dtype == np.uint16 else g)
        own = tg[me.own0:me.own1].clone()
        backend = OracleParts(bool(bz))
        buf, me2 = split.exchange_halo(own, H, halo)
        assert me2 == me
        assert torch.equal(buf, tg[me.buf0:me.buf1]), "buffer rows differ from the image's"
        sums = backend.stats(buf, me, H, W, p)
        split.reduce_sums(sums)
        A, S = split.sums_total(sums.numpy())
        _, ref = oracle.hybrid(g, smax, w, bits=bits, border_zero=bool(bz))
        assert w * w * S - A == ref.sumD, "reduced sum of D differs from the whole image's"
        out = split.denoise_split(own, H, W, p, backend)
        ref_own = ref.out32[me.own0:me.own1]
        got = out.numpy().view(np.uint16) if bits > 8 else out.numpy()
        assert np.array_equal(got, ref_own), "rows differ from the whole-image oracle"
        dist.destroy_process_group()
        q.put((rank, "ok"))
    except Exception as e:  # reported to the parent
        import traceback
        q.put((rank, traceback.format_exc()))


@pytest.mark.parametrize("world,case", [
    (2, (37, 23, 8, 7, 5, 0)),
    (3, (40, 31, 12, 9, 3, 0)),
    (3, (13, 17, 8, 11, 7, 1)),        # strips of 4 rows, halo 8: rows come from two ranks away
    (2, (2, 9, 12, 5, 3, 0)),          # one row per rank
])
def test_split_over_gloo_ranks_matches_whole_image(world, case):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    results = {}
    for _ in range(world):
        rank, msg = q.get(timeout=240)
        results[rank] = msg
    for pr in procs:
        pr.join(timeout=60)
    for r in range(world):
        assert results.get(r) == "ok", results.get(r)


def test_part_rows_and_transfers_cover_every_buffer():
    from paper_2005_05371_gb300 import split
    for H, world, halo in ((100, 4, 7), (9, 9, 3), (50, 3, 30), (1, 1, 5)):
        parts = split.all_parts(H, world, halo)
        assert parts[0].own0 == 0 and parts[-1].own1 == H
        assert all(a.own1 == b.own0 for a, b in zip(parts, parts[1:]))
        got = {p.rank: set(range(p.own0, p.own1)) for p in parts}
        for s, d, a, b in split.transfers(H, world, halo):
            assert parts[s].own0 <= a < b <= parts[s].own1          # a sender sends its own rows
            assert not (got[d] & set(range(a, b)))                  # never twice
            got[d] |= set(range(a, b))
        for p in parts:
            assert got[p.rank] == set(range(p.buf0, p.buf1))
            assert p.buf0 == max(0, p.own0 - halo) and p.buf1 == min(H, p.own1 + halo)
