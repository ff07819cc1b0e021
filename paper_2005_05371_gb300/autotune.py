"""Autotuner for the persistent kernel's work-item shape.

The tunables are the rows per work item (`region_h`: the median/Wiener region
is 64 columns x region_h rows) and the grid size in CTAs per SM.  `sweep`
times every candidate on seeded images of each size class, and on a batch
plan of uneven slices, with CUDA events over CUDA-graph replays; `tune` keeps
the fastest per class and writes a JSON table; `choose` / `apply` pick the
entry for an image at call time and `choose_batch` the one for batches.  Results
never depend on the tuning (the tests check several shapes), only the speed.
"""
from __future__ import annotations

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE_PATH = os.path.join(HERE, "tuning.json")
REGION_H = (16, 24, 32, 40, 48, 56, 64)
CTAS_PER_SM = (0, 2, 3)


def size_class(H: int, W: int) -> str:
    px = H * W
    if px < 1_000_000:
        return "small"
    if px < 8_000_000:
        return "medium"
    return "large"


def _cases():
    import synth
    return {
        "small": [synth.CONFIGS["plain512"]],
        "medium": [synth.CONFIGS["paper1620"]],
        "large": [synth.CONFIGS["stress4096"]],
    }


def time_config(hd, torch, spec, g, region_h, ctas, steps=20, warmup=3):
    """Mean ms per hybrid_denoise launch for one tuning (CUDA-graph replay)."""
    hd.hd_set_tuning(region_h, ctas)
    src = torch.from_numpy(g.view(np.int16) if g.dtype == np.uint16 else g).cuda()
    dst = torch.empty_like(src)
    code = hd.HD_U8 if g.dtype == np.uint8 else hd.HD_U16
    p = hd.Params(spec.smax, spec.wiener_w, bits=spec.bits)
    ws = hd._workspace(hd.hybrid_workspace_size(spec.H, spec.W, code, p), "cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(warmup):
            hd.hybrid_denoise(src, dst, spec.smax, spec.wiener_w, bits=spec.bits, workspace=ws, stream=s)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for _ in range(steps):
            hd.hybrid_denoise(src, dst, spec.smax, spec.wiener_w, bits=spec.bits, workspace=ws, stream=s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        graph.replay()          # warm
        e0.record(s)
        graph.replay()
        e1.record(s)
    s.synchronize()
    return e0.elapsed_time(e1) / steps


def time_batch(hd, torch, items, region_h, ctas, launches=10):
    """Mean ms per launch of a batch plan for one tuning."""
    hd.hd_set_tuning(region_h, ctas)
    plan = hd.BatchPlan(items)
    s = torch.cuda.Stream()
    try:
        for _ in range(3):
            plan.launch(s)
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            e0.record(s)
            for _ in range(launches):
                plan.launch(s)
            e1.record(s)
        s.synchronize()
        return e0.elapsed_time(e1) / launches
    finally:
        plan.close()


def sweep():
    import torch
    import paper_2005_05371_gb300 as hd
    import synth
    old = hd.hd_get_tuning()
    out = {}
    try:
        for cls, specs in _cases().items():
            for spec in specs:
                g = spec.noisy()
                for rh in REGION_H:
                    for c in CTAS_PER_SM:
                        ms = time_config(hd, torch, spec, g, rh, c)
                        out.setdefault(cls, []).append({"region_h": rh, "ctas_per_sm": c, "ms": ms,
                                                        "H": spec.H, "W": spec.W})
        # batches: 64 uneven 12-bit slices of the batched workload's kind
        items = []
        for sp in synth.batch_specs(64, master_seed=400):
            src = torch.from_numpy(sp.noisy().view(np.int16)).cuda()
            items.append((src, torch.empty_like(src), hd.Params(sp.smax, sp.wiener_w, -1.0, 0, 0, sp.bits)))
        for rh in REGION_H:
            for c in CTAS_PER_SM:
                out.setdefault("batch", []).append({"region_h": rh, "ctas_per_sm": c,
                                                    "ms": time_batch(hd, torch, items, rh, c), "images": 64})
    finally:
        hd.hd_set_tuning(*old)
    return out


def tune(path: str = TABLE_PATH):
    res = sweep()
    table = {}
    for cls, rows in res.items():
        best = min(rows, key=lambda r: r["ms"])
        table[cls] = {"region_h": best["region_h"], "ctas_per_sm": best["ctas_per_sm"], "ms": best["ms"]}
    with open(path, "w") as fh:
        json.dump({"table": table, "sweep": res}, fh, indent=1)
    return table


_loaded: dict = {}


def _table(path: str) -> dict:
    """The tuned table at `path` (read once per path; {} if there is none)."""
    if path not in _loaded:
        tab = {}
        if os.path.exists(path):
            with open(path) as fh:
                tab = json.load(fh).get("table", {})
        _loaded[path] = tab
    return _loaded[path]


def choose(H: int, W: int, path: str = TABLE_PATH):
    """(region_h, ctas_per_sm) for an image, from the tuned table (default (32, 0))."""
    ent = _table(path).get(size_class(H, W))
    if not ent:
        return 32, 0
    return int(ent["region_h"]), int(ent["ctas_per_sm"])


def choose_batch(path: str = TABLE_PATH):
    """(region_h, ctas_per_sm) for batched launches (default: the large-image entry)."""
    ent = _table(path).get("batch")
    if not ent:
        return choose(4096, 4096, path)
    return int(ent["region_h"]), int(ent["ctas_per_sm"])


def apply(H: int, W: int):
    """Set the library's tuning for an H x W image from the table."""
    import paper_2005_05371_gb300 as hd
    hd.hd_set_tuning(*choose(H, W))


if __name__ == "__main__":
    print(json.dumps(tune(), indent=1))
