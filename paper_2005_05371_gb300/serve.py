"""Continuous-batching request server over the batched hybrid-denoise kernel.

Requests (a host image plus filter parameters) arrive at any time.  A
scheduler thread admits them into a fixed device-memory arena as space
frees up, groups every admitted, not yet launched request into one round,
and launches the round as ONE persistent batched kernel on a stream that no
running round holds.  Up to `max_inflight` rounds run on the device at once,
so requests that arrive while others are on the GPU start on the next round
without waiting for the earlier ones to finish: their work overlaps on the
device.  A round's completion event marks its requests done; their arena
space is then freed.

Admission by a byte budget: each admitted request holds ONE arena block with
its input, its output and the workspace it would need as a batch of its own.
A round of several requests asks the arena for one workspace for the whole
round; when no free gap is large enough, the first admitted request runs as
a round of one inside its own block.  So admission never overcommits the
arena and the scheduler always makes progress, however fragmented the arena
is.

Latency of a request = arrival (submit) -> its round's completion event
observed by the scheduler, including the host->device copy of the input and
the device->host copy of the result.

Every stage runs in the CUDA library through the C ABI
(`hybrid_denoise_batched`); this module only schedules, copies and keeps time.
The device side sits behind a small backend object (`CudaBackend`), so the
scheduling and the arena can also be exercised without a GPU.
"""
from __future__ import annotations

import ctypes
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import (HD_U8, HD_U16, Params, _check, _lib, _stream_ptr, hd_image)

ALIGN = 256


def _align(n: int) -> int:
    return (int(n) + ALIGN - 1) // ALIGN * ALIGN


class DeviceArena:
    """First-fit allocator of offsets into one buffer of `nbytes` (the buffer,
    if any, is owned by the arena; offsets are multiples of 256)."""

    def __init__(self, nbytes: int, device="cuda:0", buffer=None, allocate: bool = True):
        self.size = int(nbytes) // ALIGN * ALIGN
        if buffer is None and allocate:
            import torch
            buffer = torch.zeros(self.size, dtype=torch.uint8, device=device)
        self.buf = buffer
        self.free = [(0, self.size)]          # sorted (offset, length)
        self.used = 0

    def alloc(self, nbytes: int):
        n = _align(nbytes)
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                self.used += n
                return off, n
        return None

    def release(self, off: int, n: int):
        self.used -= n
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((o, l))
        self.free = merged

    def largest_gap(self) -> int:
        return max((l for _, l in self.free), default=0)

    def view(self, off: int, nbytes: int):
        return self.buf[off:off + nbytes]


@dataclass
class Request:
    rid: int
    host: object                     # pinned torch CPU tensor (uint8 or int16 view of uint16)
    params: Params
    out: object | None               # pinned torch CPU tensor for the result, or None (stays on device)
    t_arrive: float
    t_done: float = 0.0
    done: threading.Event = field(default_factory=threading.Event)
    error: str | None = None
    dev: dict = field(default_factory=dict)     # arena block of this request and the offsets in it

    @property
    def shape(self) -> tuple[int, int]:
        return int(self.host.shape[0]), int(self.host.shape[1])

    @property
    def elem(self) -> int:
        h = self.host
        return int(h.element_size()) if hasattr(h, "element_size") else int(h.itemsize)

    @property
    def pixels(self) -> int:
        H, W = self.shape
        return H * W

    @property
    def nbytes(self) -> int:
        return self.pixels * self.elem

    @property
    def code(self) -> int:
        return HD_U8 if self.elem == 1 else HD_U16

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.t_done - self.t_arrive)


def _images(reqs, src_dst=None) -> ctypes.Array:
    """hd_image array for a round; src_dst(i) gives the device pointers (or
    placeholders for a size query)."""
    imgs = (hd_image * len(reqs))()
    for i, r in enumerate(reqs):
        H, W = r.shape
        s, d = src_dst(i) if src_dst else (0x1000, 0x1000 + _align(r.nbytes))
        imgs[i] = hd_image(s, d, H, W, W * r.elem, W * r.elem, r.code, r.params.to_c(r.code), None, None)
    return imgs


class CudaBackend:
    """The device side of the server: the arena buffer, the streams, and a
    round = copies in + one hybrid_denoise_batched launch + copies out."""

    def __init__(self, device, n_streams: int):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]

    def thread_init(self):
        self.torch.cuda.set_device(self.device)

    def arena(self, nbytes: int) -> DeviceArena:
        return DeviceArena(nbytes, self.device)

    @staticmethod
    def workspace_bytes(reqs) -> int:
        """hybrid_batched_workspace_size of the requests as one batch (a size
        query only: no pointer is used)."""
        imgs = _images(reqs)
        n = ctypes.c_size_t()
        _check(_lib.hybrid_batched_workspace_size(imgs, len(reqs), ctypes.byref(n)),
               "hybrid_batched_workspace_size")
        return int(n.value)

    def launch(self, arena: DeviceArena, reqs, ws_off: int, ws_len: int, si: int):
        torch = self.torch
        s = self.streams[si]
        base = arena.buf.data_ptr()
        imgs = _images(reqs, lambda i: (base + reqs[i].dev["src"], base + reqs[i].dev["dst"]))
        with torch.cuda.stream(s):
            for r in reqs:
                arena.view(r.dev["src"], r.nbytes).copy_(r.host.reshape(-1).view(torch.uint8), non_blocking=True)
        _check(_lib.hybrid_denoise_batched(imgs, len(reqs), base + ws_off, ws_len, _stream_ptr(s)),
               "hybrid_denoise_batched")
        with torch.cuda.stream(s):
            for r in reqs:
                if r.out is not None:
                    r.out.reshape(-1).view(torch.uint8).copy_(arena.view(r.dev["dst"], r.nbytes), non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(s)
        return ev


class Server:
    """Continuous batching with admission by a device-memory budget."""

    def __init__(self, budget_bytes: int = 8 << 30, max_inflight: int = 3, max_batch: int = 128,
                 device="cuda:0", backend=None, max_round_px: int = 64 << 20):
        self.backend = backend if backend is not None else CudaBackend(device, max_inflight)
        self.arena = self.backend.arena(budget_bytes)
        self.max_inflight = max_inflight
        self.max_batch = max_batch
        # a round holds at most this many pixels (at least one request): after
        # a burst, the backlog drains in rounds of bounded length instead of
        # one long round that every request in it waits for
        self.max_round_px = max_round_px
        self.lock = threading.Condition()
        self.waiting: deque[Request] = deque()     # arrived, not admitted
        self.admitted: deque[Request] = deque()    # on device, not launched
        self.inflight: list = []                   # (event, requests, round workspace or None, stream index)
        self.finished: list[Request] = []
        self.rounds = 0
        self.solo_rounds = 0                       # rounds of one run in the request's own block
        self.next_id = 0
        self.stop_flag = False
        self.peak_used = 0
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    # ------------------------------------------------------------------ client side
    def submit(self, host, params: Params, out=None) -> Request:
        """Queue one image (pinned CPU tensor) for denoising; returns its Request."""
        with self.lock:
            r = Request(self.next_id, host, params, out, time.perf_counter())
            self.next_id += 1
            self._layout(r)
            if r.dev["block"] > self.arena.size:
                r.error = "request larger than the device-memory budget"
                r.t_done = time.perf_counter()
                r.done.set()
                self.finished.append(r)
                return r
            self.waiting.append(r)
            self.lock.notify()
            return r

    def close(self):
        with self.lock:
            self.stop_flag = True
            self.lock.notify()
        self.thread.join()

    def drain(self, timeout: float = 60.0) -> bool:
        t_end = time.perf_counter() + timeout
        while time.perf_counter() < t_end:
            with self.lock:
                if not self.waiting and not self.admitted and not self.inflight:
                    return True
            time.sleep(0.0005)
        return False

    def stats(self) -> dict:
        ok = [r for r in self.finished if r.error is None]
        lat = np.array([r.latency_ms for r in ok]) if ok else np.zeros(1)
        px = sum(r.pixels for r in ok)
        span = (max(r.t_done for r in ok) - min(r.t_arrive for r in ok)) if ok else 1.0
        return {"requests": len(ok), "rejected": len(self.finished) - len(ok), "rounds": self.rounds,
                "solo_rounds": self.solo_rounds,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mpixel_s": px / span / 1e6, "peak_device_bytes": self.peak_used}

    # ------------------------------------------------------------------ scheduler
    def _layout(self, r: Request):
        """Offsets of the request's block: [input][output][own workspace]."""
        b = _align(r.nbytes)
        ws1 = _align(self.backend.workspace_bytes([r]))
        r.dev = {"block": 2 * b + ws1, "src_rel": 0, "dst_rel": b, "ws_rel": 2 * b, "ws_len": ws1}

    def _admit(self):
        # first come, first admitted: a request that does not fit waits for
        # space (the ones behind it wait too, so large requests are not starved)
        while self.waiting:
            r = self.waiting[0]
            a = self.arena.alloc(r.dev["block"])
            if a is None:
                return
            self.waiting.popleft()
            off = a[0]
            r.dev.update(alloc=a, src=off + r.dev["src_rel"], dst=off + r.dev["dst_rel"], ws=off + r.dev["ws_rel"])
            self.admitted.append(r)
            self.peak_used = max(self.peak_used, self.arena.used)

    def _launch_round(self) -> bool:
        """Launch admitted requests (up to max_batch, and up to max_round_px
        pixels) as one batched kernel.
        A round of several needs a workspace gap in the arena (the round is
        halved until one fits).  A lone request, or the first request when no
        gap fits and no round is running to free one, runs alone in its own
        block.  Returns False when the round has to wait for space."""
        take = min(len(self.admitted), self.max_batch)
        px = self.admitted[0].pixels
        for i in range(1, take):
            px += self.admitted[i].pixels
            if px > self.max_round_px:
                take = i
                break
        lone = take == 1
        a_ws = None
        while take >= 2:
            reqs = [self.admitted[i] for i in range(take)]
            a_ws = self.arena.alloc(self.backend.workspace_bytes(reqs))
            if a_ws is not None:
                break
            take //= 2
        if a_ws is None:
            if not lone and self.inflight:
                return False          # running rounds will free space
            take = 1
            reqs = [self.admitted[0]]
            ws_off, ws_len = reqs[0].dev["ws"], reqs[0].dev["ws_len"]
            self.solo_rounds += 1
        else:
            ws_off, ws_len = a_ws
        for _ in range(take):
            self.admitted.popleft()
        busy = {si for _, _, _, si in self.inflight}
        si = next(i for i in range(self.max_inflight) if i not in busy)
        ev = self.backend.launch(self.arena, reqs, ws_off, ws_len, si)
        self.inflight.append((ev, reqs, a_ws, si))
        self.rounds += 1
        self.peak_used = max(self.peak_used, self.arena.used)
        return True

    def _retire(self):
        still = []
        now_done = []
        for ev, reqs, a_ws, si in self.inflight:
            if ev.query():
                t = time.perf_counter()
                for r in reqs:
                    r.t_done = t
                    now_done.append(r)
                if a_ws is not None:
                    self.arena.release(*a_ws)
                for r in reqs:
                    self.arena.release(*r.dev["alloc"])
            else:
                still.append((ev, reqs, a_ws, si))
        self.inflight = still
        for r in now_done:
            self.finished.append(r)
            r.done.set()

    def _loop(self):
        self.backend.thread_init()
        while True:
            with self.lock:
                if self.stop_flag and not self.waiting and not self.admitted and not self.inflight:
                    return
                self._retire()
                self._admit()
                while self.admitted and len(self.inflight) < self.max_inflight:
                    if not self._launch_round():
                        break
                idle = not self.admitted and not self.waiting
            if idle and not self.inflight:
                with self.lock:
                    if not self.waiting and not self.stop_flag:
                        self.lock.wait(timeout=0.001)
            else:
                time.sleep(0.00005)


def poisson_arrivals(rate_hz: float, n: int, seed: int) -> np.ndarray:
    """Arrival offsets (seconds) of a Poisson stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def replay(server: Server, pool, arrivals, params_of, want_results: bool = False, outs=None):
    """Submit pool images at the given arrival offsets (paced by sleeping).
    Results go to ``outs[i % len(pool)]`` when given, to fresh pinned tensors
    with ``want_results``, else stay on the device."""
    t0 = time.perf_counter()
    reqs = []
    for i, t in enumerate(arrivals):
        # sleep to the arrival time: a busy wait would hold the interpreter
        # lock that the scheduler thread needs
        wait = t - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        host = pool[i % len(pool)]
        if outs is not None:
            out = outs[i % len(pool)]
        elif want_results:
            import torch
            out = torch.empty_like(host).pin_memory()
        else:
            out = None
        reqs.append(server.submit(host, params_of(i), out))
    return reqs
