"""One image split across GPUs by row strips (one rank per GPU).

The paper parallelises its hybrid by cutting the image into sub-images that
workers filter side by side (Algorithm 1, step 6: parfor over the image's
strips; Fig. 5).  Here the cut keeps the whole-image result:

1. Rank r owns rows [own0, own1) = [floor(r H / P), floor((r+1) H / P)).
2. Halo exchange: each rank needs the rows its own rows' windows read, h =
   smax/2 + w/2 above and below; it receives them from the ranks that own
   them (point-to-point sends of whole rows into its own memory: no remote
   reads of a peer's memory by a kernel) and assembles its buffer of rows
   [max(0, own0 - h), min(H, own1 + h)).
3. Statistics (`hybrid_part_stats`): the median and the local statistics of
   the own rows, and four 64-bit words of exact partial sums.
4. One all-reduce (SUM) of the four words: the whole image's sums, from
   which the noise variance (the mean local variance) follows exactly.
5. Apply (`hybrid_part_apply`): the Wiener output of the own rows.

The integer reduction makes the reassembled image bit-identical to the
single-GPU hybrid.  This module holds only the host logic: row bounds,
the exchange and the reduction over ``torch.distributed``, and the order of
the calls.  The device work goes through a backend; `CudaPartBackend` calls
the library's C ABI.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class PartRows:
    """Rows of one part (all [begin, end)): the rows it owns and the rows its
    buffer holds (own rows plus halo, clipped to the image)."""
    rank: int
    own0: int
    own1: int
    buf0: int
    buf1: int


def part_rows(H: int, world: int, rank: int, halo: int) -> PartRows:
    """Rank `rank`'s rows of an H-row image split into `world` strips."""
    if not (1 <= world <= H):
        raise ValueError("need 1 <= world size <= image rows")
    own0, own1 = rank * H // world, (rank + 1) * H // world
    return PartRows(rank, own0, own1, max(0, own0 - halo), min(H, own1 + halo))


def all_parts(H: int, world: int, halo: int) -> list[PartRows]:
    return [part_rows(H, world, r, halo) for r in range(world)]


def transfers(H: int, world: int, halo: int):
    """(sender, receiver, row0, row1): every block of rows a rank sends from
    its own rows to fill another rank's buffer."""
    parts = all_parts(H, world, halo)
    out = []
    for dst in parts:
        for src in parts:
            if src.rank == dst.rank:
                continue
            a, b = max(dst.buf0, src.own0), min(dst.buf1, src.own1)
            if a < b:
                out.append((src.rank, dst.rank, a, b))
    return out


def exchange_halo(own, H: int, halo: int, group=None):
    """This rank's buffer (rows [buf0, buf1)) assembled from its own rows
    `own` (a tensor of shape (own1 - own0, W)) and the halo rows received
    from the ranks that own them.  The tensors stay on their device: CPU
    tensors over gloo, CUDA tensors over NCCL."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    me = part_rows(H, world, rank, halo)
    if own.shape[0] != me.own1 - me.own0:
        raise ValueError("own rows do not match this rank's strip")
    buf = torch.empty((me.buf1 - me.buf0, own.shape[1]), dtype=own.dtype, device=own.device)
    buf[me.own0 - me.buf0:me.own1 - me.buf0] = own
    ops = []
    for s, d, a, b in transfers(H, world, halo):
        if s == rank:
            ops.append(dist.P2POp(dist.isend, own[a - me.own0:b - me.own0].contiguous(), d, group))
        elif d == rank:
            ops.append(dist.P2POp(dist.irecv, buf[a - me.buf0:b - me.buf0], s, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return buf, me


def reduce_sums(sums, group=None):
    """Sum the parts' four 64-bit words over all ranks, in place (one all-reduce)."""
    import torch.distributed as dist
    dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return sums


def denoise_split(own, H: int, W: int, params, backend, group=None):
    """The hybrid of an H x W image split over the ranks of `group`: `own` is
    this rank's own rows of the noisy image; returns its own rows of the
    result.  `backend` runs the two device calls (`stats`, `apply`)."""
    halo = backend.halo_rows(params)
    buf, me = exchange_halo(own, H, halo, group)
    sums = backend.stats(buf, me, H, W, params)
    reduce_sums(sums, group)
    return backend.apply(buf, me, H, W, params, sums)


class CudaPartBackend:
    """The device calls of a part through the library's C ABI."""

    def __init__(self, stream=None):
        import torch
        import paper_2005_05371_gb300 as hd
        self.hd = hd
        self.torch = torch
        self.stream = stream
        self.ws = None

    def halo_rows(self, params) -> int:
        return self.hd.part_halo_rows(params)

    def _part(self, buf, dst, me: PartRows, H, W, params):
        return self.hd.make_part(buf, dst, H, W, me.buf0, me.own0, me.own1 - me.own0, params)

    def stats(self, buf, me: PartRows, H, W, params):
        hd, torch = self.hd, self.torch
        part = self._part(buf, None, me, H, W, params)
        need = hd.hybrid_part_workspace_size(part)
        if self.ws is None or hd._ws_len(self.ws) < need:
            self.ws = hd._workspace(need, buf.device)
        sums = torch.zeros(4, dtype=torch.int64, device=buf.device)
        hd.hybrid_part_stats(part, self.ws, sums, self.stream)
        return sums

    def apply(self, buf, me: PartRows, H, W, params, sums):
        dst = self.torch.empty((me.own1 - me.own0, W), dtype=buf.dtype, device=buf.device)
        part = self._part(buf, dst, me, H, W, params)
        self.hd.hybrid_part_apply(part, sums, self.ws, self.stream)
        return dst


def sums_total(words) -> tuple[int, int]:
    """(A, B) as exact integers from the four words {A lo32, A hi32, B lo32, B hi32}."""
    w = [int(x) & 0xFFFFFFFFFFFFFFFF for x in np.asarray(words, dtype=np.int64).tolist()]
    return w[0] + (w[1] << 32), w[2] + (w[3] << 32)
