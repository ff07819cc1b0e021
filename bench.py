#!/usr/bin/env python3
"""Throughput of the hybrid denoiser (adaptive median -> Wiener) on GB300.

One step = one pass of the whole hot path (adaptive median with window
growth, Wiener statistics, noise-variance reduction, Wiener apply) over one
input of the chosen workload, through the C ABI.  Prints ONE JSON line.

Workloads (seeded synthetic phantoms, see synth/):
  batched    (default) 256 uneven 12-bit slices (256^2..1024^2), per-slice
             sigma, density, Smax and Wiener window; one persistent launch
             replayed as a CUDA graph, against the per-slice launch loop
             (also replayed from CUDA graphs) on the same slices.
  paper1620  1620x1620 uint8, Gaussian sigma 20 + salt&pepper 0.20, Smax 9,
             5x5 Wiener, noise variance estimated.  The image is the size of
             the paper's 2.5 MB medical image (Section V).
  plain512   512x512 uint8, sigma 10, density 0.05, Smax 7, 3x3 Wiener.
  stress4096 4096x4096 12-bit, sigma 40, density 0.40, Smax 11, 5x5 Wiener.
  served     Poisson request stream (2000 req/s) over a pool of 256 images
             512^2..4096^2 through the continuous-batching server: p50/p99
             latency, throughput and a capacity sweep.
With --parts P a single-image step runs the listing's partitioned median
(hybrid_denoise_strips: P row strips median-filtered alone, then the Wiener
filter of the whole image), as the paper runs it with P workers.
With --stretch TOL a single-image step also runs the contrast stretch of
Algorithm 1, step 4e (contrast_stretch, in place on the result): the paper's
whole step 4.  The contrast kernel is then also timed alone.

Timing: W untimed warm-up steps, then K steps between barrier +
synchronize, timed with CUDA events on the launching stream.  Inputs rotate
over enough device copies that every step reads data not resident in the
129 MB L2.  `e2e` runs the same workload from pinned host buffers to pinned
host buffers through the library's host-buffer entry points (every step
copies its inputs in and its results out inside the timed region).  The
CPU legs (`cpu_baseline`, `accuracy`) run the oracle on the host cores: one
thread on a bounded sample, and every core on the whole workload (or, for a
single image, on row bands of it), where the oracle's outputs are also
compared with the GPU's.  `--impl reference` times the oracle instead, on
every host core (bounded sample per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
METRIC = "hybrid AMF+Wiener Mpixel/s on 1 GB300 (batched vs plain); p50/p99 served latency"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
# algorithmic operations per pixel: 3x3 level A/B with shared column sorts
# (about 20 min/max and 6 compare/select) and the Wiener stage (about 10
# integer and 10 FP32 operations); window growth is not counted
OPS_PER_PIXEL = 46
ALU_LANES_PER_SM = 128          # 32-bit INT/FP32 lanes of one SM (4 partitions x 32)
SM_MAX_GHZ = 2.07
WORKLOADS = ["batched", "paper1620", "plain512", "stress4096", "served"]


# --------------------------------------------------------------------------- helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(files=("hd_kernel.cu", "hd_internal.h")) -> str:
    """Hash of a kernel's sources (the counters in profiles/ refer to it)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2005_05371_gb300", "csrc")
    for name in files:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, source: str | None = None):
    """DRAM bytes per launch from an ncu capture, if taken on the current kernel source
    (`source`: the kernel's file; default the persistent kernel)."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    with open(PROFILE_TRAFFIC) as fh:
        rec = json.load(fh)
    ent = rec.get(workload)
    want = kernel_source_hash((source,)) if source else kernel_source_hash()
    if not ent or ent.get("source_hash") != want:
        return None
    return ent.get("dram_bytes_per_launch")


def recorded_issue(workload: str):
    """ncu instruction-issue figures of the persistent kernel for a workload
    (if taken on the current kernel source): the measured side of the
    integer-ALU roofline."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    with open(PROFILE_TRAFFIC) as fh:
        ent = json.load(fh).get(workload)
    if not ent or ent.get("source_hash") != kernel_source_hash() or "issue" not in ent:
        return None
    return ent["issue"]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- multi-rank helpers
def replica_seeds(name: str, rank: int):
    """(phantom, noise) seeds of rank `rank`'s replica: every rank denoises its
    own independent images (weak scaling, no data-path collective)."""
    import synth
    if name in synth.CONFIGS:
        s = synth.CONFIGS[name]
        return [(s.phantom_seed + 1000 * rank, s.noise_seed + 1000 * rank)]
    if name == "batched":
        return [(sp.phantom_seed, sp.noise_seed) for sp in synth.batch_specs(256, master_seed=400 + rank)]
    raise SystemExit(f"unknown workload {name}")


def max_over_ranks(ms: float, device=None) -> float:
    """The slowest rank's time (all_reduce MAX); the identity for one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(px_per_rank: int, steps: int, max_ms: float, world: int) -> float:
    """Whole-job Mpixel/s: pixels of all ranks over the slowest rank's time."""
    return world * px_per_rank * steps / (max_ms / 1e3) / 1e6


# --------------------------------------------------------------------------- workloads
SERVED_POOL = 256


BATCH_SLICES = 256


def workload_specs(name: str, rank: int):
    """The seeded specs of a workload.  Rank r draws its own replica (distinct seeds)."""
    import synth
    if name in synth.CONFIGS:
        spec = synth.CONFIGS[name]
        if rank:
            spec = synth.SliceSpec(**{**spec.__dict__, "phantom_seed": spec.phantom_seed + 1000 * rank,
                                      "noise_seed": spec.noise_seed + 1000 * rank})
        return [spec]
    if name == "batched":
        return synth.batch_specs(256, master_seed=400 + rank)[:BATCH_SLICES]
    if name == "served":
        return synth.served_specs(SERVED_POOL, seed=501 + rank)
    raise SystemExit(f"unknown workload {name}")


def build_workload(name: str, rank: int):
    """[(spec, noisy host image)] of a workload (drawn on every host core)."""
    import synth
    specs = workload_specs(name, rank)
    return list(zip(specs, synth.noisy_images(specs)))


def describe(name: str, items, stretch: float | None = None, parts: int = 1) -> dict:
    px = sum(s.H * s.W for s, _ in items)
    if name == "served":
        return {"workload": f"served: Poisson 2000 req/s over a pool of {len(items)} seeded phantoms, side "
                            "log-uniform [512, 4096], u8 / 12-bit 50/50, s&p up to 0.3, Smax {5..11}, Wiener "
                            "{3,5,7}, 8 GB device budget, continuous batching",
                "images": len(items), "megapixels": round(px / 1e6, 3)}
    if name == "batched":
        return {"workload": "batched: 256 uneven 12-bit slices {256^2,512^2,768x512,1024^2}, sigma U[10,60], "
                            "density U[0.01,0.5], Smax {5,7,9,11}, Wiener {3,5,7}, one persistent launch "
                            "(CUDA graph) vs the per-slice launch loop (CUDA graphs)",
                "images": len(items), "megapixels": round(px / 1e6, 3)}
    s = items[0][0]
    d = {"workload": f"{name}: {s.H}x{s.W} {s.dtype} {s.bits}-bit, sigma {s.sigma:g}, s&p {s.density:g}, "
                     f"Smax {s.smax}, Wiener {s.wiener_w}x{s.wiener_w}, noise variance estimated",
         "H": s.H, "W": s.W, "smax": s.smax, "wiener_w": s.wiener_w, "megapixels": round(px / 1e6, 3)}
    if parts > 1:
        d["workload"] += f", median partitioned into {parts} row strips"
        d["parts"] = parts
    if stretch is not None:
        d["workload"] += f", then contrast stretch (tol {stretch:g}) in place"
        d["contrast_stretch_tol"] = stretch
    return d


def quality(outs, cleans, noisies, bits) -> dict:
    """PSNR (dB) and max abs error of the denoised images against the clean
    phantoms, beside the same figures for the noisy inputs (all images pooled)."""
    maxv = float((1 << bits) - 1)

    def stats(imgs):
        se, n, mx = 0.0, 0, 0
        for a, c in zip(imgs, cleans):
            d = a.astype(np.int64) - c.astype(np.int64)
            se += float((d * d).sum())
            n += d.size
            mx = max(mx, int(np.abs(d).max()))
        mse = se / n
        return (round(10.0 * math.log10(maxv * maxv / mse), 3) if mse > 0 else float("inf")), mx

    p_out, m_out = stats(outs)
    p_in, m_in = stats(noisies)
    return {"psnr_db": p_out, "max_abs_error": m_out, "noisy_psnr_db": p_in, "noisy_max_abs_error": m_in,
            "against": "the clean synthetic phantom", "images": len(outs)}


def algorithmic_bytes(items) -> int:
    """Read the noisy input once and write the result once."""
    return sum(2 * s.H * s.W * (1 if s.dtype == "u8" else 2) for s, _ in items)


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


# --------------------------------------------------------------------------- CPU oracle legs
def oracle_sample_rate(items, budget_s: float, stretch: float | None = None, parts: int = 1):
    """Oracle Mpx/s on ONE host core, on a bounded sample: whole images (or row
    bands) until ~budget_s.  With `stretch`, each band's result also goes
    through the oracle's contrast stretch; with `parts` > 1 the band's median
    is partitioned."""
    import oracle

    def run(g, spec):
        if parts > 1:
            _, r = oracle.hybrid_strips(g, spec.smax, spec.wiener_w, min(parts, g.shape[0]), bits=spec.bits)
        else:
            _, r = oracle.hybrid(g, spec.smax, spec.wiener_w, bits=spec.bits)
        if stretch is not None:
            oracle.contrast(r.out32, stretch, bits=spec.bits)
    done_px, t_total = 0, 0.0
    descr = []
    for spec, g in items:
        # calibrate on a 32-row band, then size the band to the remaining budget
        rows = min(spec.H, 32)
        t0 = time.perf_counter()
        run(g[:rows], spec)
        dt = time.perf_counter() - t0
        done_px += rows * spec.W
        t_total += dt
        remaining = budget_s - t_total
        if remaining <= 0:
            descr.append(f"{rows} rows of {spec.H}x{spec.W}")
            break
        per_row = dt / rows
        more = int(min(spec.H, max(1, remaining / per_row)))
        if more > rows:
            t0 = time.perf_counter()
            run(g[:more], spec)
            t_total += time.perf_counter() - t0
            done_px += more * spec.W
            rows = more
        descr.append(f"{rows} rows of {spec.H}x{spec.W}")
        if t_total >= budget_s:
            break
    return done_px / t_total / 1e6, t_total, "; ".join(descr[:4]) + (" ..." if len(descr) > 4 else "")


def accuracy_of(refs, gpu_out_sha, gpu_y_sha=None, gpu_nu2=None, specs=None) -> dict:
    """The GPU results against the oracle's: bit-exact integer outputs and
    binary32 values (by SHA-256), exact noise variances, and the binary32
    value's distance from the binary64 definition."""
    n = len(refs)
    d = {"vs": "the oracle on the host cores: binary64 definition and its binary32 twin", "images": n,
         "out_bit_exact_images": sum(r["out32_sha"] == h for r, h in zip(refs, gpu_out_sha))}
    if gpu_y_sha is not None:
        d["y32_bit_exact_images"] = sum(r["y32_sha"] == h for r, h in zip(refs, gpu_y_sha))
    if gpu_nu2 is not None:
        d["nu2_exact_images"] = sum(r["nu2"] == v for r, v in zip(refs, gpu_nu2))
    d["max_abs_err_y32_vs_y64_lsb"] = max(r["max_err_y32_y64"] for r in refs)
    if specs is not None:
        d["bound_lsb"] = max(s.maxv for s in specs) * 2.0 ** -20
    d["pixels_out_ne_round_y64"] = sum(r["round_diff"] for r in refs)
    d["pixels"] = sum(r["pixels"] for r in refs)
    return d


def cpu_legs(items, budget_s: float, stretch=None, parts: int = 1, gpu=None):
    """cpu_baseline (the oracle on every host core, plus one thread beside it)
    and, when `gpu` gives the GPU's output digests, the accuracy record.

    Every core: the whole workload (every image once, one image per worker),
    or for a single image row bands of it; one thread: a bounded sample."""
    from oracle import parallel
    rate1, secs1, descr1 = oracle_sample_rate(items, budget_s, stretch, parts)
    single = {"value": round(rate1, 4), "unit": "Mpixel/s", "cores": 1,
              "sample": f"C oracle, one thread, {secs1:.1f} s on {descr1}"}
    specs = [s for s, _ in items]
    acc = None
    with parallel.Runner() as runner:
        if len(items) > 1:
            refs = runner.run_specs(list(items))
            rate, wall = parallel.rate_mpx(refs)
            sample = f"the whole workload ({len(items)} images), one image per worker"
        else:
            spec, g = items[0]
            bands = runner.run_bands(parallel.band_tasks(g, spec.smax, spec.wiener_w, spec.bits,
                                                         rows=max(8, spec.H // (4 * runner.n))))
            rate, wall = parallel.rate_mpx(bands)
            sample = f"{spec.H}x{spec.W} in row bands with their halo rows, one band per task"
            refs = runner.run_specs(list(items)) if gpu is not None and stretch is None and parts == 1 else None
        cores = runner.n
    if gpu is not None and refs is not None:
        acc = accuracy_of(refs, *gpu, specs=specs)
    cpu = {"value": round(rate, 4), "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
           "sample": f"C oracle (unchanged) on {cores} host cores, {wall:.1f} s wall: {sample}"
                     + ("; the hybrid only (no stretch, no strips)" if (stretch is not None or parts > 1) else ""),
           "single_thread": single}
    return cpu, acc


def run_reference(args, rank, world):
    """The oracle as it stands, on every host core of the box: each step a
    bounded sample of the workload (whole images one per worker, or row bands
    of a single image)."""
    if rank != 0:
        return 0
    from oracle import parallel
    import synth
    specs = workload_specs(args.workload, 0)
    per_step = max(0.3, min(10.0, args.ref_budget / max(1, args.steps + args.warmup)))
    rates = []
    with parallel.Runner() as runner:
        # the sample: row bands (with their halo rows) of the first images of
        # the workload, rotating; a step takes as many bands as fit its budget
        # (calibrated by the steps before it)
        imgs = synth.noisy_images(specs[:max(1, min(len(specs), 2 * runner.n))])
        tasks = []
        for spec, g in zip(specs, imgs):
            tasks += parallel.band_tasks(g, spec.smax, spec.wiener_w, spec.bits, rows=32)
        take, pos = runner.n, 0
        for k in range(args.warmup + args.steps):
            sub = [tasks[(pos + i) % len(tasks)] for i in range(take)]
            pos += take
            res = runner.run_bands(sub)
            rate, wall = parallel.rate_mpx(res)
            if k >= args.warmup:
                rates.append(rate)
            take = int(min(4 * len(tasks), max(runner.n, take * per_step / max(wall, 1e-3))))
        descr = (f"about {take} row bands of 32 rows (with halo rows) a step, from the first {len(imgs)} "
                 f"images of the workload, one band per task")
        cores = runner.n
    value = statistics.median(rates)
    px_step = describe(args.workload, [(s, None) for s in specs])["megapixels"]
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mpixel/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * px_step / value, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "data": "synthetic",
        "dtype": "u8+u16" if args.workload == "served" else ("u8" if specs[0].dtype == "u8" else "u16"),
        "config": describe(args.workload, [(s, None) for s in specs], args.stretch, args.parts),
        "cpu_baseline": {"value": round(value, 4), "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step ~{per_step:.1f} s of the C oracle on {cores} host cores: {descr}"
                                   + ("; the hybrid only" if (args.stretch is not None or args.parts > 1) else "")},
        "e2e": {"value": round(value, 4), "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- served
def run_served(args, rank, world, dev, hd, torch):
    """Poisson request stream (2000 req/s) through the continuous-batching
    server: 2 s of warm-up arrivals, then `--served-seconds` of arrivals;
    then a capacity sweep of short runs at higher rates."""
    from paper_2005_05371_gb300.serve import Server, poisson_arrivals, replay
    items = build_workload("served", rank)
    specs = [s for s, _ in items]
    hosts = [torch.from_numpy(g.view(np.int16) if g.dtype == np.uint16 else g).pin_memory() for _, g in items]
    outs = [torch.empty_like(h).pin_memory() for h in hosts]

    def params_of(i):
        s = specs[i % len(specs)]
        return hd.Params(s.smax, s.wiener_w, -1.0, hd.HD_BORDER_SYMMETRIC, hd.HD_UNRESOLVED_ZMED, s.bits)

    from paper_2005_05371_gb300 import autotune
    tuning = autotune.choose_batch()
    hd.hd_set_tuning(*tuning)
    rate = 2000.0
    bound_ms = 50.0

    def run(srv, r_hz, seconds, seed):
        n = max(1, int(r_hz * seconds))
        reqs = replay(srv, hosts, poisson_arrivals(r_hz, n, seed), params_of, outs=outs)
        for r in reqs:
            r.done.wait(600)
        lat = np.array([r.latency_ms for r in reqs if r.error is None])
        px = sum(r.pixels for r in reqs if r.error is None)
        span = max(r.t_done for r in reqs) - min(r.t_arrive for r in reqs)
        return reqs, {"offered_req_s": r_hz, "p50_ms": round(float(np.percentile(lat, 50)), 3),
                      "p99_ms": round(float(np.percentile(lat, 99)), 3), "mpixel_s": round(px / span / 1e6, 1),
                      "requests": len(reqs)}

    srv = Server(budget_bytes=8 << 30, max_inflight=max(1, args.inflight), device=dev)
    try:
        run(srv, rate, 2.0, 499)                            # warm-up: 2 s of arrivals
        srv.finished.clear()
        srv.rounds = srv.solo_rounds = 0
        with ClockSampler(dev.index or 0) as clk:
            reqs, main = run(srv, rate, args.served_seconds, 500 + rank)
        st = srv.stats()
        clocks = clk.summary()
        clocks["window"] = "request stream"
        # capacity: the highest offered rate whose p99 stays under the bound and
        # whose served rate keeps up with the offered one
        sweep, capacity = [], None
        for k, r_hz in enumerate((2000.0, 4000.0, 6000.0, 8000.0, 12000.0, 16000.0)):
            _, res = run(srv, r_hz, 2.0, 600 + k)
            offered_mpx = r_hz * sum(s.H * s.W for s in specs) / len(specs) / 1e6
            res["keeps_up"] = res["mpixel_s"] >= 0.9 * offered_mpx
            sweep.append(res)
            if res["p99_ms"] <= bound_ms and res["keeps_up"]:
                capacity = res
            else:
                break
    finally:
        srv.close()
    status = hd.hd_get_device_error()
    if status != hd.HD_OK:
        raise SystemExit(f"device error: {hd.hd_status_str(status)}")
    n_req = len(reqs)
    px = sum(r.pixels for r in reqs)
    bytes_in = sum(r.nbytes for r in reqs)
    span_ms = 1e3 * (max(r.t_done for r in reqs) - min(r.t_arrive for r in reqs))
    span_ms = max_over_ranks(span_ms, dev)
    value = weak_value(px, 1, span_ms, world)
    peak, peak_kind = peaks()
    achieved = 2 * bytes_in / (span_ms / 1e3) / 1e9
    cpu = acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # every pool image was served (the stream cycles through the pool);
        # the oracle checks the first 32 results and gives the CPU baseline
        sub = items[:32]
        got = [o.numpy().view(np.uint16) if s.dtype == "u16" else o.numpy() for o, (s, _) in zip(outs, sub)]
        cpu, acc = cpu_legs(sub, args.cpu_budget, gpu=([digest(a) for a in got],))
        cpu["sample"] += " (the first 32 pool images)"
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "Mpixel/s", "n_gpus": world, "steps": n_req,
            "warmup": int(rate * 2.0), "ms_per_step": round(span_ms / n_req, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8+u16", "data": "synthetic",
            "config": {**describe("served", items), "requests": n_req, "seconds_of_arrivals": args.served_seconds,
                       "rounds_in_flight": max(1, args.inflight),
                       "warmup_seconds": 2.0, "megapixels": round(px / 1e6, 1), "parallelism": f"replicas x{world}",
                       "tuning": dict(zip(autotune.FIELDS, tuning)),
                       "l2": f"every request moves its own input/output through HBM (pool {len(items)} images, "
                             f"{sum(h.numel() * h.element_size() for h in hosts) / 1e9:.1f} GB)"},
            "latency": {"p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                        "rounds": st["rounds"], "solo_rounds": st["solo_rounds"],
                        "peak_device_bytes": st["peak_device_bytes"]},
            "capacity": {"p99_bound_ms": bound_ms, "highest_rate_within_bound": capacity, "sweep": sweep,
                         "run_seconds": 2.0},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "kernel": "hd_persistent_kernel",
                         "peak_kind": peak_kind,
                         "note": "served rate equals the offered load at 2000 req/s: see capacity"},
            "cpu_baseline": cpu, "accuracy": acc,
            "e2e": {"value": round(value, 2), "unit": "Mpixel/s", "h2d_bytes_per_step": bytes_in // n_req,
                    "d2h_bytes_per_step": bytes_in // n_req,
                    "api": "Server.submit (pinned host in/out, copies and launches inside)"},
            "gpu_launches": 2 * st["rounds"], "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="batched", choices=WORKLOADS)
    ap.add_argument("--cpu-budget", type=float, default=10.0, help="seconds of single-thread oracle work")
    ap.add_argument("--ref-budget", type=float, default=90.0, help="total seconds of the reference arm")
    ap.add_argument("--served-seconds", type=float, default=10.0, help="seconds of arrivals of the served run")
    ap.add_argument("--inflight", type=int, default=3, help="served: rounds in flight on the device at once")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--parts", type=int, default=1,
                    help="row strips of the partitioned median (Algorithm 1, step 6); 1 = whole image")
    ap.add_argument("--stretch", type=float, default=None,
                    help="also run the contrast stretch (Algorithm 1, step 4e) with this tolerance every step")
    ap.add_argument("--slices", type=int, default=256,
                    help="batched: the first N slices of the 256 (smaller cases for profiling)")
    ap.add_argument("--fourier", type=float, default=None,
                    help="single image: also time the Wiener filter in the Fourier domain (wiener_deconvolve, "
                         "7x7 Gaussian PSF) with this noise-to-signal ratio")
    args = ap.parse_args()
    global BATCH_SLICES
    BATCH_SLICES = max(1, min(256, args.slices))
    if (args.stretch is not None or args.parts > 1 or args.fourier is not None) and \
            args.workload in ("batched", "served"):
        raise SystemExit("--stretch, --parts and --fourier apply to the single-image workloads")
    if args.parts < 1:
        raise SystemExit("--parts must be >= 1")
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__._buildlib().build()
    import paper_2005_05371_gb300 as hd

    if args.workload == "served":
        return run_served(args, rank, world, dev, hd, torch)

    items = build_workload(args.workload, rank)
    batched = args.workload == "batched"
    cfg = describe(args.workload, items, args.stretch, args.parts)
    # work-item shape from the autotuner's table (paper_2005_05371_gb300/tuning.json)
    from paper_2005_05371_gb300 import autotune
    s0 = items[0][0]
    tuning = autotune.choose_batch() if batched else autotune.choose(s0.H, s0.W, s0.dtype, s0.smax, s0.wiener_w,
                                                                       s0.density)
    hd.hd_set_tuning(*tuning)
    cfg["tuning"] = dict(zip(autotune.FIELDS, tuning))
    stream = torch.cuda.current_stream(dev)

    def to_dev(a):
        t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a)
        return t.to(dev)

    def params_of(spec):
        return hd.Params(spec.smax, spec.wiener_w, -1.0, hd.HD_BORDER_SYMMETRIC, hd.HD_UNRESOLVED_ZMED, spec.bits)

    def code_of(spec):
        return hd.HD_U8 if spec.dtype == "u8" else hd.HD_U16

    step_bytes = algorithmic_bytes(items)
    copies = 2 if batched else max(1, math.ceil(3 * L2_BYTES / step_bytes))
    px_per_step = sum(s.H * s.W for s, _ in items)

    if batched:
        # `copies` independent batch plans over distinct device buffers
        plans, bufs = [], []
        for c in range(copies):
            its = []
            for spec, g in items:
                src = to_dev(g)
                dst = torch.empty_like(src)
                its.append((src, dst, params_of(spec)))
            bufs.append(its)
            plans.append(hd.BatchPlan(its))

        def step(i, s):
            plans[i % copies].launch(s)

        launches_per_step = 1
        # plain: the per-slice launch loop (one hybrid_denoise call per slice, each
        # with its size class's tuning and a full workspace) on the same data
        ws_plain = [hd._workspace(hd.hybrid_workspace_size(s.H, s.W, code_of(s), params_of(s)), dev)
                    for s, _ in items]
        slice_tuning = [autotune.choose(s.H, s.W, s.dtype, s.smax, s.wiener_w, s.density) for s, _ in items]

        def plain_step(i, s):
            its = bufs[i % copies]
            try:
                for (src, dst, p), ws, tn in zip(its, ws_plain, slice_tuning):
                    hd.hd_set_tuning(*tn)
                    hd.hybrid_denoise(src, dst, p.smax, p.wiener_w, p.noise_var, p.border, p.unresolved, p.bits,
                                      workspace=ws, stream=s)
            finally:
                hd.hd_set_tuning(*tuning)
    else:
        spec, g = items[0]
        p = params_of(spec)
        srcs = [to_dev(g) for _ in range(copies)]
        dsts = [torch.empty_like(srcs[0]) for _ in range(copies)]
        code = code_of(spec)
        if args.parts > 1:
            ws = hd._workspace(hd.hybrid_strips_workspace_size(spec.H, spec.W, code, p, args.parts), dev)

            def hybrid_step(i, s):
                j = i % copies
                hd.hybrid_denoise_strips(srcs[j], dsts[j], args.parts, p.smax, p.wiener_w, p.noise_var, p.border,
                                         p.unresolved, p.bits, workspace=ws, stream=s)
            # strip medians, descriptor upload, Wiener
            launches_per_step = 3
        else:
            ws = hd._workspace(hd.hybrid_workspace_size(spec.H, spec.W, code, p), dev)

            def hybrid_step(i, s):
                j = i % copies
                hd.hybrid_denoise(srcs[j], dsts[j], p.smax, p.wiener_w, p.noise_var, p.border, p.unresolved,
                                  p.bits, workspace=ws, stream=s)
            launches_per_step = 1

        step = hybrid_step
        plain_step = None
        if args.stretch is not None:
            cws = hd._workspace(hd.contrast_workspace_size(spec.H, spec.W, code, spec.bits), dev)
            cdsts = [torch.empty_like(srcs[0]) for _ in range(copies)]

            def step(i, s):
                hybrid_step(i, s)
                j = i % copies
                hd.contrast_stretch(dsts[j], None, args.stretch, p.bits, workspace=cws, stream=s)

            def contrast_step(i, s):
                # the stretch alone, dsts -> cdsts (same data every time around)
                j = i % copies
                hd.contrast_stretch(dsts[j], cdsts[j], args.stretch, p.bits, workspace=cws, stream=s)

            launches_per_step += 1

    def capture(fn, first, count):
        """One CUDA graph holding `count` consecutive steps."""
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs):
                for i in range(count):
                    fn(first + i, cs)
        stream.wait_stream(cs)
        return g

    def timed(fn, K, W, graph, per_graph=400):
        """K steps after W warm-up steps; CUDA events on the launching stream.
        With graph=True the K steps replay from CUDA graphs of up to
        `per_graph` steps each (the host's launch cost is not timed; every
        kernel still launches)."""
        for i in range(W):
            fn(i, stream)
        torch.cuda.synchronize(dev)
        plan = []
        if graph:
            G = min(K, per_graph)
            g_main = capture(fn, W, G)
            plan = [g_main] * (K // G)
            if K % G:
                plan.append(capture(fn, W, K % G))
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            e0.record(stream)
            if graph:
                for g in plan:
                    g.replay()
            else:
                for i in range(K):
                    fn(W + i, stream)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        if world > 1:
            dist.barrier()
        return e0.elapsed_time(e1), plan, wall

    def soak(fn, plan, seconds):
        """Keep the same kernel running so the clock sampler sees it under load."""
        t_end = time.perf_counter() + seconds
        with torch.cuda.stream(stream):
            while time.perf_counter() < t_end:
                if plan:
                    for g in plan[:8]:
                        g.replay()
                else:
                    fn(0, stream)
                torch.cuda.synchronize(dev)

    # a batch plan is itself a CUDA graph: its steps launch directly
    with ClockSampler(local) as clk:
        total_ms, graphs, wall = timed(step, args.steps, args.warmup, not batched)
        soaked = max(0.0, 1.5 - wall)
        if soaked > 0:
            soak(step, graphs, soaked)
    clocks = clk.summary()
    clocks["window"] = "timed region" if soaked == 0 else f"timed region ({wall:.3f} s) + {soaked:.2f} s of the same step"
    status = hd.hd_get_device_error(stream)
    if status != hd.HD_OK:
        raise SystemExit(f"device error after the timed region: {hd.hd_status_str(status)}")

    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / args.steps
    value = weak_value(px_per_step, args.steps, total_ms, world)

    # dominant kernel: one persistent launch per step; events over
    # back-to-back launches give the average launch duration
    peak, peak_kind = peaks()
    extra = {}
    hybrid_ms = ms_per_step
    if args.stretch is not None:
        # each kernel alone, same launch configuration and rotation of copies
        K2 = max(10, args.steps)
        h_ms, _, _ = timed(hybrid_step, K2, args.warmup, True)
        c_ms, _, _ = timed(contrast_step, K2, args.warmup, True)
        hybrid_ms, contrast_ms = max_over_ranks(h_ms, dev) / K2, max_over_ranks(c_ms, dev) / K2
        c_ach = step_bytes / (contrast_ms / 1e3) / 1e9
        extra["contrast_kernel"] = {"kernel": "contrast_kernel", "ms": round(contrast_ms, 5),
                                    "bound": "hbm", "achieved": round(c_ach, 1), "peak": peak, "unit": "GB/s",
                                    "frac": round(c_ach / peak, 4), "traffic": recorded_traffic(
                                        args.workload + "_contrast", "hd_contrast.cu"),
                                    "algorithmic_bytes_per_launch": step_bytes,
                                    "hybrid_kernel_ms": round(hybrid_ms, 5)}
        status = hd.hd_get_device_error(stream)
        if status != hd.HD_OK:
            raise SystemExit(f"device error in the per-kernel timing: {hd.hd_status_str(status)}")
    if args.fourier is not None:
        # the Wiener filter in the Fourier domain alone (Section IV), same image
        # rotation; its traffic counts the binary32 complex planes (8 bytes a
        # pixel) each pass reads or writes: 5 for the PSF's transfer function
        # (row pass, transpose, column pass) and 9 for the image (row pass,
        # transpose, filtered column pass reading the PSF's plane too,
        # transpose, inverse row pass)
        r = np.arange(7) - 3
        kern = np.exp(-(r[:, None] ** 2 + r[None, :] ** 2) / (2 * 1.5 * 1.5))
        psf = torch.from_numpy((kern / kern.sum()).astype(np.float32)).to(dev)
        fws = hd._workspace(hd.wiener_deconv_workspace_size(spec.H, spec.W), dev)
        fdsts = [torch.empty_like(srcs[0]) for _ in range(copies)]

        def fourier_step(i, s):
            j = i % copies
            hd.wiener_deconvolve(srcs[j], fdsts[j], psf, args.fourier, bits=p.bits, workspace=fws, stream=s)
        K2 = max(10, args.steps)
        f_ms, _, _ = timed(fourier_step, K2, args.warmup, True)
        f_ms = max_over_ranks(f_ms, dev) / K2
        plane_traffic = 14 * spec.H * spec.W * 8
        f_ach = plane_traffic / (f_ms / 1e3) / 1e9
        extra["fourier_wiener"] = {"kernels": "fft_rows_kernel, fft_transpose_kernel, fft_tables_kernel",
                                   "ms": round(f_ms, 5), "mpixel_s": round(px_per_step / (f_ms / 1e3) / 1e6, 1),
                                   "nsr": args.fourier, "psf": "7x7 Gaussian, sigma 1.5",
                                   "bound": "hbm", "achieved": round(f_ach, 1), "peak": peak, "unit": "GB/s",
                                   "frac": round(f_ach / peak, 4), "bytes_per_call": plane_traffic,
                                   "bytes_note": "14 reads or writes of an H x W binary32 complex plane "
                                                 "(8 bytes a pixel)",
                                   "launches_per_call": 10}
        status = hd.hd_get_device_error(stream)
        if status != hd.HD_OK:
            raise SystemExit(f"device error in the Fourier-domain Wiener: {hd.hd_status_str(status)}")
    achieved = step_bytes / (hybrid_ms / 1e3) / 1e9
    # the integer/FP32 side of the roofline: algorithmic operations per pixel
    # of the 3x3 median stage and the Wiener stage (window growth not
    # counted, so this is a lower bound of the work) against the SMs' 32-bit
    # lanes at the maximum SM clock; the measured issue rate from ncu beside it
    props = torch.cuda.get_device_properties(dev)
    alu_peak = props.multi_processor_count * ALU_LANES_PER_SM * SM_MAX_GHZ * 1e9 / 1e12
    alu_achieved = px_per_step * OPS_PER_PIXEL / (hybrid_ms / 1e3) / 1e12
    traffic = recorded_traffic(args.workload) if args.parts == 1 else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": "hd_persistent_kernel", "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": step_bytes}
    roofline_alu = {"bound": "alu", "achieved": round(alu_achieved, 3), "peak": round(alu_peak, 2),
                    "unit": "Tops/s", "frac": round(alu_achieved / alu_peak, 4),
                    "ops_per_pixel": OPS_PER_PIXEL, "kernel": "hd_persistent_kernel",
                    "peak_kind": f"derived: {props.multi_processor_count} SMs x {ALU_LANES_PER_SM} lanes x "
                                 f"{SM_MAX_GHZ} GHz",
                    "ncu_issue": recorded_issue(args.workload) if args.parts == 1 else None}

    if batched:
        # the plain per-slice loop, replayed from CUDA graphs of 4 steps (1024 launches each)
        Kp = max(4, args.steps // 5 // 4 * 4)
        plain_ms, _, _ = timed(plain_step, Kp, 2, True, per_graph=4)
        plain_ms = max_over_ranks(plain_ms, dev)
        plain_value = weak_value(px_per_step, Kp, plain_ms, world)
        extra["plain_loop"] = {"value": round(plain_value, 1), "unit": "Mpixel/s",
                               "ms_per_step": round(plain_ms / Kp, 4), "launches_per_step": len(items),
                               "how": "one hybrid_denoise per slice (its size class's tuning, full workspace), "
                                      "replayed from CUDA graphs", "batched_over_plain": round(value / plain_value, 3)}
        status = hd.hd_get_device_error(stream)
        if status != hd.HD_OK:
            raise SystemExit(f"device error in the plain loop: {hd.hd_status_str(status)}")

    # end to end through the library's host-buffer entry points
    e2e = None
    if not args.no_e2e and (args.stretch is not None or args.parts > 1):
        # pinned host -> device, hybrid (strips), stretch, device -> pinned host, wait
        spec, g = items[0]
        hsrc = torch.from_numpy(g.view(np.int16) if g.dtype == np.uint16 else g).pin_memory()
        hdst = torch.empty_like(hsrc).pin_memory()

        def e2e_step(i):
            srcs[0].copy_(hsrc, non_blocking=True)
            hybrid_step(0, stream)
            if args.stretch is not None:
                hd.contrast_stretch(dsts[0], None, args.stretch, p.bits, workspace=cws, stream=stream)
            hdst.copy_(dsts[0], non_blocking=True)
            stream.synchronize()
        for i in range(args.warmup):
            e2e_step(i)
        t0 = time.perf_counter()
        for i in range(args.steps):
            e2e_step(i)
        dt = time.perf_counter() - t0
        e2e = {"value": round(world * px_per_step * args.steps / dt / 1e6, 2), "unit": "Mpixel/s",
               "h2d_bytes_per_step": g.nbytes, "d2h_bytes_per_step": g.nbytes,
               "api": "copy_ + " + ("hybrid_denoise_strips" if args.parts > 1 else "hybrid_denoise") +
                      (" + contrast_stretch" if args.stretch is not None else "") + " (pinned host buffers)"}
    elif not args.no_e2e and not batched:
        # the host pipeline: every step copies its noisy image in from pinned
        # host memory and its result back out; the copies of one step overlap
        # the kernels of its neighbours
        spec, g = items[0]
        p = params_of(spec)
        code = code_of(spec)
        hsrc = torch.from_numpy(g.view(np.int16) if g.dtype == np.uint16 else g).pin_memory()
        hdst = [torch.empty_like(hsrc).pin_memory() for _ in range(2)]
        pipe = hd.HostPipeline(spec.H, spec.W, code, p, depth=2, device=dev)
        for i in range(args.warmup):
            pipe.submit(hsrc, hdst[i % 2])
        pipe.wait()
        t0 = time.perf_counter()
        for i in range(args.steps):
            pipe.submit(hsrc, hdst[i % 2])
        pipe.wait()
        dt = time.perf_counter() - t0
        pipe.close()
        e2e = {"value": round(world * px_per_step * args.steps / dt / 1e6, 2), "unit": "Mpixel/s",
               "h2d_bytes_per_step": g.nbytes, "d2h_bytes_per_step": g.nbytes,
               "api": "hd_host_pipeline (pinned host buffers, depth 2: copies overlap neighbouring steps)"}
        # the synchronous call, one step at a time, for comparison
        wsh = hd._workspace(hd.hybrid_host_workspace_size(spec.H, spec.W, code, p), dev)
        t0 = time.perf_counter()
        K3 = max(3, args.steps // 5)
        for i in range(K3):
            hd.hybrid_denoise_host(hsrc, hdst[0], p.smax, p.wiener_w, p.noise_var, p.border, p.unresolved,
                                   p.bits, workspace=wsh, stream=stream)
        e2e["synchronous_call"] = {"value": round(world * px_per_step * K3 / (time.perf_counter() - t0) / 1e6, 2),
                                   "api": "hybrid_denoise_host, one blocking call a step"}
    elif not args.no_e2e:
        # the batch pipeline: every step copies all slices in from one pinned
        # host buffer (back to back: one copy) and the results back out;
        # depth 2, so one step's copies overlap its neighbours' kernels
        sizes = [g.size for _, g in items]
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        h_in = torch.empty(int(offs[-1]), dtype=torch.int16).pin_memory()
        for (_, g), o in zip(items, offs[:-1]):
            h_in[int(o):int(o) + g.size].copy_(torch.from_numpy(g.view(np.int16).reshape(-1)))
        h_out = [torch.empty_like(h_in).pin_memory() for _ in range(2)]
        views = lambda buf: [buf[int(o):int(o) + s.H * s.W].view(s.H, s.W) for (s, _), o in zip(items, offs[:-1])]
        in_v, out_v = views(h_in), [views(h) for h in h_out]
        pipe = hd.BatchPipeline([(s.H, s.W, code_of(s), params_of(s)) for s, _ in items], depth=2, device=dev)
        for i in range(args.warmup):
            pipe.submit(in_v, out_v[i % 2])
        pipe.wait()
        t0 = time.perf_counter()
        for i in range(args.steps):
            pipe.submit(in_v, out_v[i % 2])
        pipe.wait()
        dt = time.perf_counter() - t0
        pipe.close()
        nb = sum(g.nbytes for _, g in items)
        e2e = {"value": round(world * px_per_step * args.steps / dt / 1e6, 2), "unit": "Mpixel/s",
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
               "api": "hd_batch_pipeline (pinned host buffers, all slices back to back: one copy each way a "
                      "step; depth 2)"}
        status = hd.hd_get_device_error()
        if status != hd.HD_OK:
            raise SystemExit(f"device error in the batch pipeline: {hd.hd_status_str(status)}")

    # one more step outside the timed region, with the binary32 values and noise
    # variances kept, for the oracle comparison and the quality figures
    def host_image(t, spec):
        a = t.cpu().numpy()
        return a.view(np.uint16) if spec.dtype != "u8" else a
    gpu_rec = None
    if batched:
        nv = torch.full((len(items),), -7.0, dtype=torch.float64, device=dev)
        ys = [torch.empty((s.H, s.W), dtype=torch.float32, device=dev) for s, _ in items]
        imgs = [hd.make_image(src, dst, pp, nv[i:i + 1], ys[i]) for i, (src, dst, pp) in enumerate(bufs[0])]
        hd.hybrid_denoise_batched(imgs, stream=stream)
        torch.cuda.synchronize(dev)
        outs = [host_image(dst, spec) for (_, dst, _), (spec, _) in zip(bufs[0], items)]
        gpu_rec = ([digest(o) for o in outs], [digest(y.cpu().numpy()) for y in ys], nv.cpu().tolist())
        del ys
        extra["quality"] = quality(outs, [spec.clean() for spec, _ in items], [g for _, g in items], 12)
    else:
        spec0, g0 = items[0]
        nv = torch.full((1,), -7.0, dtype=torch.float64, device=dev)
        y = torch.empty((spec0.H, spec0.W), dtype=torch.float32, device=dev)
        hd.hybrid_denoise(srcs[0], dsts[0], p.smax, p.wiener_w, p.noise_var, p.border, p.unresolved, p.bits,
                          noise_var_out=nv, y_out=y, stream=stream)
        torch.cuda.synchronize(dev)
        out0 = host_image(dsts[0], spec0)
        gpu_rec = ([digest(out0)], [digest(y.cpu().numpy())], nv.cpu().tolist())
        extra["quality"] = quality([out0], [spec0.clean()], [g0], spec0.bits)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, acc = cpu_legs(items, args.cpu_budget, args.stretch, args.parts, gpu=gpu_rec)
        if acc is not None:
            extra["accuracy"] = acc
        # the paper's parallel metrics (Section 3.3): T_s = the serial oracle's
        # time for one step's pixels, T_p = this GPU's step, P = its SMs
        t_s = px_per_step / (cpu["single_thread"]["value"] * 1e6) * 1e3
        n_sm = props.multi_processor_count
        s_p = t_s / ms_per_step
        extra["paper_metrics"] = {"T_s_ms": round(t_s, 3), "T_p_ms": round(ms_per_step, 5), "P": n_sm,
                                  "S_P": round(s_p, 1), "EFF": round(s_p / n_sm, 2),
                                  "T_over_ms": round(ms_per_step - t_s / n_sm, 5),
                                  "defs": "Eq. 1 S_P = T_s/T_p, Eq. 2 EFF = S_P/P, Eq. 3 T_over = T_p - T_s/P; "
                                          "T_s: the C oracle on one host core, P: streaming multiprocessors"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8" if items[0][0].dtype == "u8" else "u16", "data": "synthetic",
            "config": {**cfg, "parallelism": f"replicas x{world}",
                       "l2": f"inputs rotate over {copies} device copies ({copies * step_bytes / 2**20:.0f} MiB "
                             f"of algorithmic traffic > 129 MB L2)"},
            "roofline": roofline, "roofline_alu": roofline_alu, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks, **extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
