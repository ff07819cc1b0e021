"""The N-GPU bench path, host side, on CPU ranks (gloo, world size 2).

Each rank denoises its own replica (independent seeded images: the path has
no data-path collective); the timing takes the slowest rank and the reported
value counts the pixels of every rank.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.replica_seeds("paper1620", rank)
        bseeds = bench.replica_seeds("batched", rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, (seeds, bseeds[:4]))
        t = bench.max_over_ranks(10.0 + rank * 5.0)
        out[rank] = (gathered, t)
    finally:
        dist.destroy_process_group()


def test_two_ranks_distinct_replicas_and_max_time():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    (g0, t0), (g1, t1) = out[0], out[1]
    assert g0 == g1                                  # every rank saw the same gathered list
    assert g0[0][0] != g0[1][0]                      # single-image replicas differ by rank
    assert g0[0][1] != g0[1][1]                      # batched replicas differ by rank
    assert t0 == t1 == 15.0                          # the slowest rank's time everywhere


def test_weak_value_counts_every_rank():
    import bench
    assert bench.weak_value(1_000_000, 10, 2.0, 1) == pytest.approx(5000.0)
    assert bench.weak_value(1_000_000, 10, 2.0, 4) == pytest.approx(20000.0)
    assert bench.max_over_ranks(3.5) == 3.5          # no process group: identity
