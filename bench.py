#!/usr/bin/env python3
"""Throughput of the hybrid denoiser (adaptive median -> Wiener) on GB300.

One step = one pass of the whole hot path (adaptive median with window
growth, Wiener statistics, noise-variance reduction, Wiener apply) over one
input of the chosen workload, through the C ABI.  Prints ONE JSON line.

Workloads (seeded synthetic phantoms, see synth/):
  paper1620  (default) 1620x1620 uint8, Gaussian sigma 20 + salt&pepper 0.20,
             Smax 9, 5x5 Wiener, noise variance estimated.  The image is the
             size of the paper's 2.5 MB medical image (Section V).
  plain512   512x512 uint8, sigma 10, density 0.05, Smax 7, 3x3 Wiener.
  stress4096 4096x4096 12-bit, sigma 40, density 0.40, Smax 11, 5x5 Wiener.
  batched    256 uneven 12-bit slices (256^2..1024^2), per-slice parameters,
             one persistent launch replayed as a CUDA graph.
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
host buffers through the host pipeline (hd_host_pipeline: every step copies
its image in and its result out inside the timed region, overlapping the
neighbouring steps' kernels), and reports the one-blocking-call-a-step
hybrid_denoise_host beside it.  `--impl reference` times the CPU oracle
instead (bounded sample per step).
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
def build_workload(name: str, rank: int):
    """Host images + parameters.  Rank r draws its own replica (distinct seeds)."""
    import synth
    if name in synth.CONFIGS:
        spec = synth.CONFIGS[name]
        if rank:
            spec = synth.SliceSpec(**{**spec.__dict__, "phantom_seed": spec.phantom_seed + 1000 * rank,
                                      "noise_seed": spec.noise_seed + 1000 * rank})
        clean = spec.clean()
        return [(spec, spec.noisy(clean))]
    if name == "batched":
        specs = synth.batch_specs(256, master_seed=400 + rank)
        return [(s, s.noisy()) for s in specs]
    if name == "served":
        return served_pool(seed=501 + rank)
    raise SystemExit(f"unknown workload {name}")


def describe(name: str, items, stretch: float | None = None, parts: int = 1) -> dict:
    px = sum(s.H * s.W for s, _ in items)
    if name == "served":
        return {"workload": "served: pool of 16 seeded phantoms, side log-uniform [512, 4096], u8 / 12-bit "
                            "50/50, s&p up to 0.3, Smax {5..11}, Wiener {3,5,7} (the reference arm denoises "
                            "the pool's images one after another)", "images": len(items),
                "megapixels": round(px / 1e6, 3)}
    if name == "batched":
        return {"workload": "batched: 256 uneven 12-bit slices {256^2,512^2,768x512,1024^2}, sigma U[10,60], "
                            "density U[0.01,0.5], Smax {5,7,9,11}, Wiener {3,5,7}, one persistent launch "
                            "(CUDA graph)", "images": len(items), "megapixels": round(px / 1e6, 3)}
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


# --------------------------------------------------------------------------- CPU oracle
def oracle_sample_rate(items, budget_s: float, stretch: float | None = None, parts: int = 1):
    """Oracle Mpx/s on a bounded sample: whole images (or row bands) until ~budget_s.
    With `stretch`, each band's result also goes through the oracle's contrast
    stretch; with `parts` > 1 the band's median is partitioned."""
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


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    items = build_workload(args.workload, 0)
    per_step = max(0.2, min(5.0, args.ref_budget / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample_rate(items, per_step, args.stretch, args.parts)
    rates, tsum, descr = [], 0.0, ""
    for _ in range(args.steps):
        r, t, descr = oracle_sample_rate(items, per_step, args.stretch, args.parts)
        rates.append(r)
        tsum += t
    value = statistics.median(rates)
    px_step = describe(args.workload, items)["megapixels"]
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mpixel/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * px_step / value, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "data": "synthetic",
        "dtype": "u8+u16" if args.workload == "served" else ("u8" if items[0][0].dtype == "u8" else "u16"),
        "config": describe(args.workload, items, args.stretch, args.parts),
        "cpu_baseline": {"value": round(value, 4), "unit": "Mpixel/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step ~{per_step:.1f} s of the C oracle (single thread) on {descr}"},
        "e2e": {"value": round(value, 4), "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- served
def served_pool(n: int = 16, seed: int = 501):
    """Pool of requests: side log-uniform in [512, 4096], u8 or 12-bit 50/50,
    sigma U[5,25] (u8) / U[10,60] (12-bit), salt & pepper density U[0, 0.3]."""
    import synth
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(n):
        side = int(np.exp(rng.uniform(np.log(512), np.log(4096))))
        H = side
        W = int(side * rng.uniform(0.8, 1.25)) // 2 * 2
        if i % 2 == 0:
            spec = synth.SliceSpec(H, W, "u8", 8, float(rng.uniform(5, 25)), float(rng.uniform(0, 0.3)),
                                   int(rng.choice([5, 7, 9, 11])), int(rng.choice([3, 5, 7])),
                                   seed * 1000 + i, seed * 1000 + 500 + i, kind="ellipse")
        else:
            spec = synth.SliceSpec(H, W, "u16", 12, float(rng.uniform(10, 60)), float(rng.uniform(0, 0.3)),
                                   int(rng.choice([5, 7, 9, 11])), int(rng.choice([3, 5, 7])),
                                   seed * 1000 + i, seed * 1000 + 500 + i, kind="ct")
        pool.append((spec, spec.noisy()))
    return pool


def run_served(args, rank, world, dev, hd, torch):
    """Poisson request stream (2000 req/s) through the continuous-batching server."""
    from paper_2005_05371_gb300.serve import Server, poisson_arrivals, replay
    pool = served_pool()
    hosts = [torch.from_numpy(g.view(np.int16) if g.dtype == np.uint16 else g).pin_memory() for _, g in pool]
    outs = [torch.empty_like(h).pin_memory() for h in hosts]

    def params_of(i):
        s = pool[i % len(pool)][0]
        return hd.Params(s.smax, s.wiener_w, -1.0, hd.HD_BORDER_SYMMETRIC, hd.HD_UNRESOLVED_ZMED, s.bits)

    from paper_2005_05371_gb300 import autotune
    tuning = autotune.choose_batch()
    hd.hd_set_tuning(*tuning)
    srv = Server(budget_bytes=8 << 30, max_inflight=3, device=dev)
    try:
        warm = replay(srv, hosts, poisson_arrivals(2000.0, max(args.warmup, 3) * 10, 499), params_of)
        for r in warm:
            r.done.wait(120)
        srv.finished.clear()
        n_req = args.steps * 40
        arrivals = poisson_arrivals(2000.0, n_req, 500 + rank)
        with ClockSampler(dev.index or 0) as clk:
            reqs = []
            t0 = time.perf_counter()
            for i, t in enumerate(arrivals):
                # sleep to the arrival time: a busy wait would hold the
                # interpreter lock that the scheduler thread needs
                wait = t - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                j = i % len(hosts)
                reqs.append(srv.submit(hosts[j], params_of(j), outs[j]))
            for r in reqs:
                r.done.wait(300)
        st = srv.stats()
        clocks = clk.summary()
        clocks["window"] = "request stream"
    finally:
        srv.close()
    status = hd.hd_get_device_error()
    if status != hd.HD_OK:
        raise SystemExit(f"device error: {hd.hd_status_str(status)}")
    px = sum(r.pixels for r in reqs)
    bytes_in = sum(int(r.host.numel() * r.host.element_size()) for r in reqs)
    span_ms = 1e3 * (max(r.t_done for r in reqs) - min(r.t_arrive for r in reqs))
    span_ms = max_over_ranks(span_ms, dev)
    value = weak_value(px, 1, span_ms, world)
    peak, peak_kind = peaks()
    achieved = 2 * bytes_in / (span_ms / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "Mpixel/s", "n_gpus": world, "steps": n_req,
            "warmup": len(warm), "ms_per_step": round(span_ms / n_req, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8+u16", "data": "synthetic",
            "config": {"workload": "served: Poisson 2000 req/s, pool of 16 seeded phantoms, side log-uniform "
                                   "[512, 4096], u8 / 12-bit 50/50, s&p up to 0.3, Smax {5..11}, Wiener {3,5,7}, "
                                   "8 GB device budget, continuous batching (3 rounds in flight)",
                       "requests": n_req, "megapixels": round(px / 1e6, 1), "parallelism": f"replicas x{world}",
                       "tuning": {"region_h": tuning[0], "ctas_per_sm": tuning[1]},
                       "l2": "every request moves its own input/output through HBM (pool 16 images, ~120 MB)"},
            "latency": {"p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                        "rounds": st["rounds"], "peak_device_bytes": st["peak_device_bytes"]},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "kernel": "hd_persistent_kernel",
                         "peak_kind": peak_kind},
            "cpu_baseline": None,
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
    ap.add_argument("--workload", default="paper1620",
                    choices=["paper1620", "plain512", "stress4096", "batched", "served"])
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=90.0, help="total seconds of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--parts", type=int, default=1,
                    help="row strips of the partitioned median (Algorithm 1, step 6); 1 = whole image")
    ap.add_argument("--stretch", type=float, default=None,
                    help="also run the contrast stretch (Algorithm 1, step 4e) with this tolerance every step")
    args = ap.parse_args()
    if (args.stretch is not None or args.parts > 1) and args.workload in ("batched", "served"):
        raise SystemExit("--stretch and --parts apply to the single-image workloads")
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

    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__._buildlib().build()
    import paper_2005_05371_gb300 as hd

    if args.workload == "served":
        return run_served(args, rank, world, dev, hd, torch)

    items = build_workload(args.workload, rank)
    cfg = describe(args.workload, items, args.stretch, args.parts)
    # work-item shape from the autotuner's table (paper_2005_05371_gb300/tuning.json)
    from paper_2005_05371_gb300 import autotune
    if args.workload == "batched":
        tuning = autotune.choose_batch()
    else:
        tuning = autotune.choose(items[0][0].H, items[0][0].W)
    hd.hd_set_tuning(*tuning)
    cfg["tuning"] = {"region_h": tuning[0], "ctas_per_sm": tuning[1]}
    stream = torch.cuda.current_stream(dev)

    def to_dev(a):
        t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a)
        return t.to(dev)

    def params_of(spec):
        return hd.Params(spec.smax, spec.wiener_w, -1.0, hd.HD_BORDER_SYMMETRIC, hd.HD_UNRESOLVED_ZMED, spec.bits)

    step_bytes = algorithmic_bytes(items)
    copies = max(1, math.ceil(3 * L2_BYTES / step_bytes)) if args.workload != "batched" else 2
    px_per_step = sum(s.H * s.W for s, _ in items)

    if args.workload == "batched":
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
        # plain: per-slice launch loop (one hybrid_denoise call per slice) on the same data
        spec0 = None
        ws_plain = [hd._workspace(hd.hybrid_workspace_size(s.H, s.W, hd.HD_U16, params_of(s)), dev)
                    for s, _ in items]

        def plain_step(i, s):
            its = bufs[i % copies]
            for (src, dst, p), ws in zip(its, ws_plain):
                hd.hybrid_denoise(src, dst, p.smax, p.wiener_w, p.noise_var, p.border, p.unresolved, p.bits,
                                  workspace=ws, stream=s)
    else:
        spec, g = items[0]
        p = params_of(spec)
        srcs = [to_dev(g) for _ in range(copies)]
        dsts = [torch.empty_like(srcs[0]) for _ in range(copies)]
        code = hd.HD_U8 if spec.dtype == "u8" else hd.HD_U16
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

    use_graph = args.workload != "batched"

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

    def timed(fn, K, W, graph):
        """K steps after W warm-up steps; CUDA events on the launching stream.
        With graph=True the K steps replay from CUDA graphs (launch overhead of
        the host path is not timed; every step is still one kernel launch)."""
        for i in range(W):
            fn(i, stream)
        torch.cuda.synchronize(dev)
        plan = []
        if graph:
            G = min(K, 400)
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

    with ClockSampler(local) as clk:
        total_ms, graphs, wall = timed(step, args.steps, args.warmup, use_graph)
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
    # back-to-back launches (graph replay) give the average launch duration
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
    achieved = step_bytes / (hybrid_ms / 1e3) / 1e9
    # the integer/FP32 side of the roofline: algorithmic operations per pixel
    # of the 3x3 median stage and the Wiener stage (window growth not
    # counted, so this is a lower bound of the work) against the SMs' 32-bit
    # lanes at the maximum SM clock
    props = torch.cuda.get_device_properties(dev)
    alu_peak = props.multi_processor_count * ALU_LANES_PER_SM * SM_MAX_GHZ * 1e9 / 1e12
    alu_achieved = px_per_step * OPS_PER_PIXEL / (hybrid_ms / 1e3) / 1e12
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": recorded_traffic(args.workload) if args.parts == 1 else None,
                "kernel": "hd_persistent_kernel", "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": step_bytes}
    roofline_alu = {"bound": "alu", "achieved": round(alu_achieved, 3), "peak": round(alu_peak, 2),
                    "unit": "Tops/s", "frac": round(alu_achieved / alu_peak, 4),
                    "ops_per_pixel": OPS_PER_PIXEL, "kernel": "hd_persistent_kernel",
                    "peak_kind": f"derived: {props.multi_processor_count} SMs x {ALU_LANES_PER_SM} lanes x "
                                 f"{SM_MAX_GHZ} GHz"}

    if plain_step is not None:
        plain_ms, _, _ = timed(plain_step, max(3, args.steps // 5), args.warmup, False)
        extra["plain_loop"] = {"value": round(px_per_step * max(3, args.steps // 5) / (plain_ms / 1e3) / 1e6, 1),
                               "unit": "Mpixel/s", "launches_per_step": len(items)}

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e and (args.stretch is not None or args.parts > 1):
        # end to end through the public calls: pinned host -> device, hybrid,
        # stretch, device -> pinned host, wait
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
    elif not args.no_e2e and args.workload != "batched":
        # end to end through the host pipeline: every step copies its noisy
        # image in from pinned host memory and its result back out, and the
        # copies of one step overlap the kernels of its neighbours
        spec, g = items[0]
        p = params_of(spec)
        code = hd.HD_U8 if spec.dtype == "u8" else hd.HD_U16
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
        # batched end to end: all slices in one pinned host buffer and one
        # device buffer, so a step is one copy in, one plan launch and one copy
        # out; two buffer sets on two streams let one step's copies overlap the
        # other's kernel
        sizes = [g.size for _, g in items]
        offs = np.concatenate([[0], np.cumsum(sizes)])
        h_in = torch.empty(int(offs[-1]), dtype=torch.int16).pin_memory()
        for (_, g), o in zip(items, offs[:-1]):
            h_in[int(o):int(o) + g.size].copy_(torch.from_numpy(g.view(np.int16).reshape(-1)))
        h_out = [torch.empty_like(h_in).pin_memory() for _ in range(2)]
        sets = []
        for k in range(2):
            d_in, d_out = torch.empty(int(offs[-1]), dtype=torch.int16, device=dev), torch.empty(
                int(offs[-1]), dtype=torch.int16, device=dev)
            its = [(d_in[int(o):int(o) + s.H * s.W].view(s.H, s.W), d_out[int(o):int(o) + s.H * s.W].view(s.H, s.W),
                    params_of(s)) for (s, _), o in zip(items, offs[:-1])]
            sets.append((d_in, d_out, hd.BatchPlan(its), torch.cuda.Stream(dev)))

        def e2e_step(i):
            d_in, d_out, plan, st = sets[i % 2]
            with torch.cuda.stream(st):
                d_in.copy_(h_in, non_blocking=True)
                plan.launch(st)
                h_out[i % 2].copy_(d_out, non_blocking=True)
        for i in range(args.warmup):
            e2e_step(i)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        K2 = max(3, args.steps // 5)
        for i in range(K2):
            e2e_step(i)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        for _, _, plan, _ in sets:
            plan.close()
        nb = sum(g.nbytes for _, g in items)
        e2e = {"value": round(world * px_per_step * K2 / dt / 1e6, 2), "unit": "Mpixel/s",
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
               "api": "one copy in + hd_batch_plan_launch + one copy out a step (pinned host buffers, "
                      "two buffer sets on two streams)"}

    # output quality against the clean phantoms, from one more step outside the
    # timed region (the hybrid output, before any contrast stretch)
    def host_image(t, spec):
        a = t.cpu().numpy()
        return a.view(np.uint16) if spec.dtype != "u8" else a
    if args.workload == "batched":
        plans[0].launch(stream)
        torch.cuda.synchronize(dev)
        outs = [host_image(dst, spec) for (_, dst, _), (spec, _) in zip(bufs[0], items)]
        extra["quality"] = quality(outs, [spec.clean() for spec, _ in items], [g for _, g in items], 12)
    else:
        hybrid_step(0, stream)
        torch.cuda.synchronize(dev)
        spec0, g0 = items[0]
        extra["quality"] = quality([host_image(dsts[0], spec0)], [spec0.clean()], [g0], spec0.bits)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, secs, descr = oracle_sample_rate(items, args.cpu_budget, args.stretch, args.parts)
        cpu = {"value": round(rate, 4), "unit": "Mpixel/s", "cores": 1, "kind": "oracle",
               "sample": f"C oracle, single thread, {secs:.1f} s on {descr}"}
        # the paper's parallel metrics (Section 3.3): T_s = the serial oracle's
        # time for one step's pixels, T_p = this GPU's step, P = its SMs
        t_s = px_per_step / (rate * 1e6) * 1e3
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
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
