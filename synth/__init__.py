"""Seeded synthetic phantoms and noise for the hybrid denoiser.

This module only draws inputs.  It holds none of the method's arithmetic and
is shared by the CUDA path's tests and benchmark and by the oracle's tests,
so both sides see the same noisy image for the same seed.

The paper (Section V, Fig. 5) ran on a hand X-ray image that is not
available, and its noise model (Algorithm 1, step 3, a degradation step) is only
named.  The stand-ins below follow the workload shapes of the benchmark
configurations:

* ``ellipse_phantom``  - piecewise-constant ellipses (optionally annuli) on a
  linear background gradient, integer values in [lo, hi] (8-bit studies).
* ``ct_phantom``       - CT-like 12-bit slice: a body disc, bright bone-like
  rings and dark lung-like blobs on an air background.
* ``add_noise``        - additive Gaussian noise (rounded to nearest, clamped
  to [0, maxv]) followed by salt-and-pepper impulses at a given density, half
  pepper (0) and half salt (maxv).

Every function takes an explicit ``numpy.random.Generator`` or seed, so each
image is reproducible from its seed on any machine with the same numpy.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "ellipse_phantom", "ct_phantom", "add_noise", "SliceSpec", "batch_specs",
    "config_image", "CONFIGS", "served_specs", "noisy_images",
]


def _grid(H: int, W: int):
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    return yy, xx


def _paint_ellipse(img: np.ndarray, cy, cx, ry, rx, theta, value, ring_frac=None):
    """Set pixels inside an (optionally hollow) rotated ellipse to ``value``.

    Only the bounding box is evaluated, so large images stay cheap.
    """
    H, W = img.shape
    r = max(ry, rx)
    y0, y1 = max(0, int(cy - r) - 1), min(H, int(cy + r) + 2)
    x0, x1 = max(0, int(cx - r) - 1), min(W, int(cx + r) + 2)
    if y0 >= y1 or x0 >= x1:
        return
    yy = np.arange(y0, y1, dtype=np.float64)[:, None] - cy
    xx = np.arange(x0, x1, dtype=np.float64)[None, :] - cx
    c, s = math.cos(theta), math.sin(theta)
    u = (c * xx + s * yy) / rx
    v = (-s * xx + c * yy) / ry
    rr = u * u + v * v
    inside = rr <= 1.0
    if ring_frac is not None:
        inside &= rr >= ring_frac * ring_frac
    img[y0:y1, x0:x1][inside] = value


def ellipse_phantom(H: int, W: int, seed: int, n_ellipses=(8, 12), lo=20, hi=230,
                    rings: int = 0) -> np.ndarray:
    """Piecewise-constant ellipses (and ``rings`` annuli) on a linear gradient.

    Returns uint8 values in [lo, hi].
    """
    rng = np.random.default_rng(seed)
    yy, xx = _grid(H, W)
    a, b = rng.uniform(-1, 1, size=2)
    base = 0.5 * (lo + hi) + 0.25 * (hi - lo) * (a * (yy / max(H - 1, 1) - 0.5)
                                                 + b * (xx / max(W - 1, 1) - 0.5))
    img = np.broadcast_to(base, (H, W)).copy()
    n = int(rng.integers(n_ellipses[0], n_ellipses[1] + 1))
    for _ in range(n):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        ry = rng.uniform(0.03, 0.3) * H
        rx = rng.uniform(0.03, 0.3) * W
        _paint_ellipse(img, cy, cx, ry, rx, rng.uniform(0, math.pi), rng.uniform(lo, hi))
    for _ in range(rings):
        cy, cx = rng.uniform(0.2, 0.8) * H, rng.uniform(0.2, 0.8) * W
        rad = rng.uniform(0.05, 0.25) * min(H, W)
        _paint_ellipse(img, cy, cx, rad, rad * rng.uniform(0.8, 1.2), rng.uniform(0, math.pi),
                       rng.uniform(lo, hi), ring_frac=rng.uniform(0.7, 0.9))
    return np.clip(np.rint(img), lo, hi).astype(np.uint8)


def ct_phantom(H: int, W: int, seed: int, bits: int = 12) -> np.ndarray:
    """CT-like slice: air background, soft-tissue disc, bone rings, lung blobs.

    Intensities follow a 12-bit scale (body ~1000-1400, bone ~3000-3800,
    lung ~50-300) and are rescaled for other bit depths.  Returns uint16.
    """
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W), dtype=np.float64) + rng.uniform(0, 40)
    cy, cx = H * rng.uniform(0.45, 0.55), W * rng.uniform(0.45, 0.55)
    ry, rx = H * rng.uniform(0.38, 0.46), W * rng.uniform(0.38, 0.46)
    _paint_ellipse(img, cy, cx, ry, rx, rng.uniform(0, math.pi), rng.uniform(1000, 1400))
    # smooth soft-tissue variation inside the body
    yy, xx = _grid(H, W)
    body = img > 500
    img[body] += (60 * np.sin(yy / max(H, 1) * rng.uniform(2, 6)) *
                  np.cos(xx / max(W, 1) * rng.uniform(2, 6)))[body]
    for _ in range(int(rng.integers(2, 5))):       # lung-like dark blobs
        _paint_ellipse(img, cy + rng.uniform(-0.2, 0.2) * H, cx + rng.uniform(-0.25, 0.25) * W,
                       rng.uniform(0.06, 0.15) * H, rng.uniform(0.05, 0.12) * W,
                       rng.uniform(0, math.pi), rng.uniform(50, 300))
    for _ in range(int(rng.integers(3, 7))):       # bone-like rings
        rad = rng.uniform(0.03, 0.12) * min(H, W)
        _paint_ellipse(img, cy + rng.uniform(-0.3, 0.3) * H, cx + rng.uniform(-0.3, 0.3) * W,
                       rad, rad * rng.uniform(0.7, 1.3), rng.uniform(0, math.pi),
                       rng.uniform(3000, 3800), ring_frac=rng.uniform(0.6, 0.85))
    scale = ((1 << bits) - 1) / 4095.0
    maxv = (1 << bits) - 1
    return np.clip(np.rint(img * scale), 0, maxv).astype(np.uint16)


def add_noise(img: np.ndarray, sigma: float, density: float, seed: int, maxv: int) -> np.ndarray:
    """Gaussian noise (rounded, clamped to [0, maxv]) then salt & pepper.

    Each pixel independently becomes an impulse with probability ``density``:
    pepper (0) with probability density/2, salt (maxv) with density/2.
    """
    rng = np.random.default_rng(seed)
    x = img.astype(np.float64)
    if sigma > 0:
        x = x + sigma * rng.standard_normal(img.shape)
    x = np.clip(np.rint(x), 0, maxv)
    if density > 0:
        u = rng.random(img.shape)
        x[u < density / 2] = 0
        x[(u >= density / 2) & (u < density)] = maxv
    return x.astype(img.dtype)


@dataclass
class SliceSpec:
    """One image of a workload with its filter parameters."""
    H: int
    W: int
    dtype: str            # "u8" or "u16"
    bits: int
    sigma: float
    density: float
    smax: int
    wiener_w: int
    phantom_seed: int
    noise_seed: int
    kind: str = "ct"      # "ct" or "ellipse"
    rings: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def maxv(self) -> int:
        return (1 << self.bits) - 1

    def clean(self) -> np.ndarray:
        if self.kind == "ct":
            return ct_phantom(self.H, self.W, self.phantom_seed, bits=self.bits)
        return ellipse_phantom(self.H, self.W, self.phantom_seed, rings=self.rings)

    def noisy(self, clean: np.ndarray | None = None) -> np.ndarray:
        c = self.clean() if clean is None else clean
        return add_noise(c, self.sigma, self.density, self.noise_seed, self.maxv)


# The five benchmark workloads.  Sizes, noise levels and filter parameters are
# those of the paper-shaped study (Section V: a ~2.5 MB grayscale image, Smax up
# to 11) and larger CT/MR-like slices.
CONFIGS = {
    "plain512": SliceSpec(512, 512, "u8", 8, 10.0, 0.05, 7, 3, 101, 102, kind="ellipse"),
    "paper1620": SliceSpec(1620, 1620, "u8", 8, 20.0, 0.20, 9, 5, 201, 202, kind="ellipse",
                           rings=4),
    "stress4096": SliceSpec(4096, 4096, "u16", 12, 40.0, 0.40, 11, 5, 301, 302, kind="ct"),
}


def config_image(name: str):
    """(spec, clean, noisy) for one of the single-image workloads."""
    spec = CONFIGS[name]
    clean = spec.clean()
    return spec, clean, spec.noisy(clean)


_BATCH_SIZES = [(256, 256), (512, 512), (768, 512), (1024, 1024)]


def batch_specs(n: int = 256, master_seed: int = 400) -> list[SliceSpec]:
    """Uneven 12-bit slices: sizes from {256^2, 512^2, 768x512, 1024^2},
    sigma ~ U[10,60] LSB, density ~ U[0.01,0.5], Smax in {5,7,9,11},
    Wiener window in {3,5,7}.  Slice i uses phantom seed 1000*master+i and
    noise seed 1000*master+100000+i (400000+i and 500000+i for master 400)."""
    rng = np.random.default_rng(master_seed)
    out = []
    for i in range(n):
        H, W = _BATCH_SIZES[int(rng.integers(0, len(_BATCH_SIZES)))]
        out.append(SliceSpec(H, W, "u16", 12, float(rng.uniform(10, 60)),
                             float(rng.uniform(0.01, 0.5)), int(rng.choice([5, 7, 9, 11])),
                             int(rng.choice([3, 5, 7])), 1000 * master_seed + i, 1000 * master_seed + 100000 + i,
                             kind="ct"))
    return out


def served_specs(n: int = 256, seed: int = 501) -> list[SliceSpec]:
    """Request pool of the served workload: side log-uniform in [512, 4096]
    (width 0.8-1.25 x the height, even), uint8 and 12-bit alternating, sigma
    U[5,25] (uint8) / U[10,60] (12-bit), salt & pepper density U[0, 0.3], Smax
    in {5,7,9,11}, Wiener window in {3,5,7}.  Image i uses phantom seed
    1000*seed+i and noise seed 1000*seed+500+i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(np.exp(rng.uniform(np.log(512), np.log(4096))))
        H = side
        W = int(side * rng.uniform(0.8, 1.25)) // 2 * 2
        if i % 2 == 0:
            out.append(SliceSpec(H, W, "u8", 8, float(rng.uniform(5, 25)), float(rng.uniform(0, 0.3)),
                                 int(rng.choice([5, 7, 9, 11])), int(rng.choice([3, 5, 7])),
                                 seed * 1000 + i, seed * 1000 + 500 + i, kind="ellipse"))
        else:
            out.append(SliceSpec(H, W, "u16", 12, float(rng.uniform(10, 60)), float(rng.uniform(0, 0.3)),
                                 int(rng.choice([5, 7, 9, 11])), int(rng.choice([3, 5, 7])),
                                 seed * 1000 + i, seed * 1000 + 500 + i, kind="ct"))
    return out


def _noisy_of(spec: SliceSpec) -> np.ndarray:
    return spec.noisy()


def noisy_images(specs, processes: int | None = None) -> list[np.ndarray]:
    """The noisy images of many specs, drawn on ``processes`` spawned workers
    (default: every host core); the same arrays as ``[s.noisy() for s in specs]``."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    n = max(1, min(processes or cores, len(specs)))
    if n == 1:
        return [s.noisy() for s in specs]
    with ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_noisy_of, specs, chunksize=1))
