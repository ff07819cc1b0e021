"""The oracle over many seeded images at once, on every host core.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the parity tests and
the benchmark's CPU-baseline leg call it; the CUDA library never does.

Each image is named by its ``synth.SliceSpec`` and redrawn from its seeds
inside the worker, so no image crosses a process boundary.  A worker runs
the unchanged oracle (``oracle.hybrid``: Algorithm 1, step 4 without the
contrast stretch) on it and returns what a comparison with the GPU needs,
small enough to send back:

* ``out32_sha`` / ``y32_sha``: SHA-256 of the integer output and of the
  binary32 twin (the GPU path must match both bit for bit);
* ``nu2``: the binary64 noise variance;
* ``max_err_y32_y64``: max |y32 - y64|, the binary32 twin against the
  binary64 definition;
* ``round_diff``: pixels where the integer output differs from
  round-half-up(y64), i.e. from ``out64``;
* ``t0`` / ``t1``: perf_counter around the oracle call alone (the clock is
  system-wide, so spans of different workers compare).

The pool is started with ``spawn``: a process forked after CUDA is
initialised in the parent can hang.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def run_spec(task) -> dict:
    """The oracle's hybrid of one seeded image (runs in a worker).  ``task``
    is a spec, or (spec, noisy image) when the caller already drew it."""
    import oracle
    spec, g = task if isinstance(task, tuple) else (task, None)
    if g is None:
        g = spec.noisy()
    t0 = time.perf_counter()
    _, r = oracle.hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits)
    t1 = time.perf_counter()
    return {
        "out32_sha": _digest(r.out32), "y32_sha": _digest(r.y32), "nu2": r.nu2,
        "max_err_y32_y64": float(np.max(np.abs(r.y32.astype(np.float64) - r.y64))),
        "round_diff": int(np.count_nonzero(r.out32 != r.out64)),
        "pixels": int(g.size), "t0": t0, "t1": t1,
    }


def run_band(task) -> dict:
    """The oracle's hybrid of one row band of an image (runs in a worker);
    times the work only.  The band carries the halo rows its windows read,
    so its own rows cost what they cost in the whole image (their values
    near the band's edges differ: the band's edges reflect)."""
    import oracle
    g, smax, w, bits, own_px = task
    t0 = time.perf_counter()
    oracle.hybrid(g, smax, w, bits=bits)
    t1 = time.perf_counter()
    return {"pixels": int(own_px), "t0": t0, "t1": t1}


def band_tasks(g: np.ndarray, smax: int, w: int, bits: int, rows: int) -> list[tuple]:
    """An image cut into bands of ``rows`` output rows, each with the halo rows
    its windows read."""
    H, W = g.shape
    halo = smax // 2 + w // 2
    tasks = []
    for y0 in range(0, H, rows):
        y1 = min(H, y0 + rows)
        tasks.append((np.ascontiguousarray(g[max(0, y0 - halo):min(H, y1 + halo)]), smax, w, bits, (y1 - y0) * W))
    return tasks


class Runner:
    """A pool of ``processes`` spawned workers (default: every host core),
    kept for several calls.  A worker that dies raises ``BrokenProcessPool``
    instead of leaving a call waiting."""

    def __init__(self, processes: int | None = None):
        import oracle
        oracle.build()          # compile once here, not in every worker
        self.n = max(1, processes or host_cores())
        self.ex = ProcessPoolExecutor(max_workers=self.n, mp_context=mp.get_context("spawn"))

    def run_specs(self, tasks) -> list[dict]:
        """``run_spec`` of every task (spec, or (spec, image)), in order."""
        return list(self.ex.map(run_spec, tasks, chunksize=1))

    def run_bands(self, tasks) -> list[dict]:
        """``run_band`` of every band task (from ``band_tasks``)."""
        return list(self.ex.map(run_band, tasks, chunksize=1))

    def close(self):
        self.ex.shutdown(wait=True)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_specs(specs, processes: int | None = None) -> list[dict]:
    """``run_spec`` for every spec, in order, on ``processes`` workers
    (default: every host core)."""
    n = max(1, min(processes or host_cores(), len(specs)))
    if n == 1:
        import oracle
        oracle.build()
        return [run_spec(s) for s in specs]
    with Runner(n) as r:
        return r.run_specs(specs)


def rate_mpx(results: list[dict]) -> tuple[float, float]:
    """(Mpixel/s over the whole run, wall seconds) from the workers' spans."""
    px = sum(r["pixels"] for r in results)
    wall = max(r["t1"] for r in results) - min(r["t0"] for r in results)
    return px / wall / 1e6, wall


def digest(a: np.ndarray) -> str:
    """SHA-256 of an array's bytes, as the workers compute it."""
    return _digest(a)
