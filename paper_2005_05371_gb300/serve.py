"""Continuous-batching request server over the batched hybrid-denoise kernel.

Requests (a host image plus filter parameters) arrive at any time.  A
scheduler thread admits them into a fixed device-memory arena as space
frees up (admission by a byte budget: input, output and workspace of the
request), groups every admitted, not yet launched request into one round,
and launches the round as ONE persistent batched kernel on its own stream.
Up to `max_inflight` rounds run on the device at once, so requests that
arrive while others are on the GPU start on the next round without waiting
for the earlier ones to finish: their work overlaps on the device.  A round's
completion event marks its requests done; their arena space is then freed.

Latency of a request = arrival (submit) -> its round's completion event
observed by the scheduler, including the host->device copy of the input and
the device->host copy of the result.

Every stage runs in the CUDA library through the C ABI
(`hybrid_denoise_batched`); this module only schedules, copies and keeps time.
"""
from __future__ import annotations

import ctypes
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import (HD_U8, HD_U16, Params, _check, _lib, _stream_ptr, hd_image, hybrid_batched_workspace_size)

ALIGN = 256


class DeviceArena:
    """First-fit allocator over one device buffer of `nbytes` (offsets only;
    the buffer is a torch tensor owned by the arena)."""

    def __init__(self, nbytes: int, device="cuda:0", buffer=None):
        import torch
        self.size = int(nbytes) // ALIGN * ALIGN
        self.buf = buffer if buffer is not None else torch.zeros(self.size, dtype=torch.uint8, device=device)
        self.free = [(0, self.size)]          # sorted (offset, length)
        self.used = 0

    def alloc(self, nbytes: int):
        n = (int(nbytes) + ALIGN - 1) // ALIGN * ALIGN
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
    dev: dict = field(default_factory=dict)     # device allocations of this request

    @property
    def pixels(self) -> int:
        return int(self.host.shape[0] * self.host.shape[1])

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.t_done - self.t_arrive)


class Server:
    """Continuous batching with admission by a device-memory budget."""

    def __init__(self, budget_bytes: int = 8 << 30, max_inflight: int = 3, max_batch: int = 128,
                 device="cuda:0"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.arena = DeviceArena(budget_bytes, self.device)
        self.max_inflight = max_inflight
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream(self.device) for _ in range(max_inflight)]
        self.lock = threading.Condition()
        self.waiting: deque[Request] = deque()     # arrived, not admitted
        self.admitted: deque[Request] = deque()    # on device, not launched
        self.inflight: list = []                   # (event, requests, ws_alloc, stream index)
        self.finished: list[Request] = []
        self.rounds = 0
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
            if self._request_bytes(r) > self.arena.size:
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
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mpixel_s": px / span / 1e6, "peak_device_bytes": self.peak_used}

    # ------------------------------------------------------------------ scheduler
    @staticmethod
    def _img_bytes(r: Request) -> int:
        return int(r.host.numel() * r.host.element_size())

    def _request_bytes(self, r: Request) -> int:
        # input + output + this image's share of a batched workspace (median plane, tables)
        b = self._img_bytes(r)
        H, W = r.host.shape
        es = r.host.element_size()
        return 2 * ((b + ALIGN - 1) // ALIGN * ALIGN) + H * ((W * es + 15) // 16 * 16) + 3 * 1024

    def _admit(self):
        # keep room for the workspaces of the requests already admitted
        reserve = sum(self._request_bytes(r) - 2 * self._img_bytes(r) for r in self.admitted)
        while self.waiting:
            r = self.waiting[0]
            b = self._img_bytes(r)
            free = self.arena.size - self.arena.used
            if free - reserve < self._request_bytes(r):
                return
            reserve += self._request_bytes(r) - 2 * b
            a_src = self.arena.alloc(b)
            if a_src is None:
                return
            a_dst = self.arena.alloc(b)
            if a_dst is None:
                self.arena.release(*a_src)
                return
            self.waiting.popleft()
            r.dev = {"src": a_src, "dst": a_dst}
            self.admitted.append(r)

    def _launch_round(self):
        """Launch the admitted requests (up to max_batch) as one batched kernel.
        If the arena has no room for the round's workspace, the round is halved
        until it fits; returns False when not even one request fits now."""
        torch = self.torch
        take = min(len(self.admitted), self.max_batch)
        while take > 0:
            reqs = [self.admitted[i] for i in range(take)]
            imgs = (hd_image * take)()
            for i, r in enumerate(reqs):
                H, W = r.host.shape
                es = r.host.element_size()
                code = HD_U8 if es == 1 else HD_U16
                src = self.arena.view(r.dev["src"][0], H * W * es)
                dst = self.arena.view(r.dev["dst"][0], H * W * es)
                imgs[i] = hd_image(src.data_ptr(), dst.data_ptr(), H, W, W * es, W * es, code,
                                   r.params.to_c(code), None, None)
            n = ctypes.c_size_t()
            _check(_lib.hybrid_batched_workspace_size(imgs, take, ctypes.byref(n)), "hybrid_batched_workspace_size")
            a_ws = self.arena.alloc(n.value)
            if a_ws is not None:
                break
            take //= 2
        if take == 0:
            return False
        for _ in range(take):
            self.admitted.popleft()
        si = self.rounds % self.max_inflight
        s = self.streams[si]
        for r in reqs:
            H, W = r.host.shape
            es = r.host.element_size()
            src = self.arena.view(r.dev["src"][0], H * W * es)
            with torch.cuda.stream(s):
                src.copy_(r.host.reshape(-1).view(torch.uint8), non_blocking=True)
        ws = self.arena.view(a_ws[0], a_ws[1])
        _check(_lib.hybrid_denoise_batched(imgs, take, ws.data_ptr(), a_ws[1], _stream_ptr(s)),
               "hybrid_denoise_batched")
        for r in reqs:
            if r.out is not None:
                H, W = r.host.shape
                es = r.host.element_size()
                dst = self.arena.view(r.dev["dst"][0], H * W * es)
                with torch.cuda.stream(s):
                    r.out.reshape(-1).view(torch.uint8).copy_(dst, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(s)
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
                self.arena.release(*a_ws)
                for r in reqs:
                    self.arena.release(*r.dev["src"])
                    self.arena.release(*r.dev["dst"])
            else:
                still.append((ev, reqs, a_ws, si))
        self.inflight = still
        for r in now_done:
            self.finished.append(r)
            r.done.set()

    def _loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                if self.stop_flag and not self.waiting and not self.admitted and not self.inflight:
                    return
                self._retire()
                self._admit()
                if self.admitted and len(self.inflight) < self.max_inflight:
                    self._launch_round()
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


def replay(server: Server, pool, arrivals, params_of, want_results: bool = False):
    """Submit pool images at the given arrival offsets (paced by sleeping)."""
    torch = server.torch
    t0 = time.perf_counter()
    reqs = []
    for i, t in enumerate(arrivals):
        # sleep to the arrival time: a busy wait would hold the interpreter
        # lock that the scheduler thread needs
        wait = t - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        host = pool[i % len(pool)]
        out = torch.empty_like(host).pin_memory() if want_results else None
        reqs.append(server.submit(host, params_of(i), out))
    return reqs
