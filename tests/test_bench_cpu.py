"""The benchmark's CPU-side pieces: the reference arm (the oracle, timed on the
host) prints one valid JSON line for each workload option, and the workload
descriptions carry what the line reports."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "3",
           "--ref-budget", "2", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("extra", [(), ("--workload", "plain512", "--stretch", "0.01"),
                                   ("--workload", "plain512", "--parts", "4"), ("--workload", "batched"),
                                   ("--workload", "served")])
def test_reference_arm_line(extra):
    d = _reference_line(*extra)
    assert d["impl"] == "reference" and d["unit"] == "Mpixel/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    if "--stretch" in extra:
        assert d["config"]["contrast_stretch_tol"] == 0.01
    if "--parts" in extra:
        assert d["config"]["parts"] == 4


def test_describe_and_algorithmic_bytes():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    spec = synth.CONFIGS["paper1620"]
    items = [(spec, None)]
    d = bench.describe("paper1620", items, 0.01, 2)
    assert d["H"] == d["W"] == 1620 and d["parts"] == 2 and d["contrast_stretch_tol"] == 0.01
    assert bench.algorithmic_bytes(items) == 2 * 1620 * 1620
    s4 = synth.CONFIGS["stress4096"]
    assert bench.algorithmic_bytes([(s4, None)]) == 4 * 4096 * 4096


def test_quality_psnr_and_max_error():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    c = np.full((10, 10), 100, np.uint8)
    o = c.copy()
    o[0, 0] = 110                                    # one error of 10: MSE = 100 / 100 = 1
    n = c.copy()
    n[:] = 120                                       # MSE 400
    q = bench.quality([o], [c], [n], 8)
    assert q["max_abs_error"] == 10 and q["noisy_max_abs_error"] == 20
    assert q["psnr_db"] == round(10 * np.log10(255.0 ** 2 / 1.0), 3)
    assert q["noisy_psnr_db"] == round(10 * np.log10(255.0 ** 2 / 400.0), 3)
    assert bench.quality([c], [c], [n], 8)["psnr_db"] == float("inf")
    # pooled over images of different sizes, 12-bit scale
    a, b = np.zeros((2, 2), np.uint16), np.zeros((1, 4), np.uint16)
    a2, b2 = a + 1, b + 3                            # squared errors 4 x 1 and 4 x 9: MSE 5
    q = bench.quality([a2, b2], [a, b], [a2, b2], 12)
    assert q["psnr_db"] == round(10 * np.log10(4095.0 ** 2 / 5.0), 3) and q["max_abs_error"] == 3
