"""Seeded synthetic images and workload definitions.

This module holds no arithmetic of the filter: it only makes inputs.  It is the one piece
of code that feeds both the CUDA path and the FP64 oracle in the tests and the benchmark.

The paper filters 8-bit grayscale images (R = 255) from the BM3D set (Section III), which
are not available here.  Stand-ins are Voronoi mosaics: flat cells with uniform random
intensity (sharp edges, the case the range kernel exists for), a horizontal linear ramp,
additive Gaussian noise, clipped to [0, 255] and rounded to integers (uint8), returned as
float32.  Generator details:
  * RNG: numpy PCG64 ``default_rng(seed)``; draws in order: cell centres (cells x 2,
    uniform over [0,H) x [0,W)), cell intensities (uniform [0,255]), noise (H x W normal).
  * cell of a pixel = the nearest centre in Euclidean distance (pixel at integer (y, x)).
  * ramp(x) = A * x / (W - 1) (zero when W == 1).
  * rounding is rint (ties to even).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def voronoi_image(H: int, W: int, cells: int, ramp: float = 40.0, noise_std: float = 10.0,
                  seed: int = 0) -> np.ndarray:
    """H x W float32 image with integer values in [0, 255] (see the module docstring)."""
    if H < 1 or W < 1:
        return np.zeros((max(H, 0), max(W, 0)), np.float32)
    rng = np.random.default_rng(seed)
    cells = max(1, int(cells))
    centres = rng.uniform(size=(cells, 2)) * np.array([H, W], dtype=np.float64)
    values = rng.uniform(0.0, 255.0, size=cells)
    noise = rng.normal(0.0, noise_std, size=(H, W)) if noise_std > 0 else np.zeros((H, W))
    labels = _nearest(centres, H, W)
    x = np.arange(W, dtype=np.float64)[None, :]
    rampv = ramp * x / (W - 1) if W > 1 else np.zeros((1, W))
    img = values[labels] + rampv + noise
    img = np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8)
    return img.astype(np.float32)


def _nearest(centres: np.ndarray, H: int, W: int) -> np.ndarray:
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    pts = np.stack([yy.ravel(), xx.ravel()], axis=1)
    try:
        from scipy.spatial import cKDTree
        _, idx = cKDTree(centres).query(pts, k=1, workers=-1)
    except ImportError:  # pragma: no cover - scipy is present on both machines
        idx = np.empty(len(pts), np.int64)
        for s in range(0, len(pts), 1 << 16):
            d = ((pts[s:s + (1 << 16), None, :] - centres[None, :, :]) ** 2).sum(-1)
            idx[s:s + (1 << 16)] = np.argmin(d, axis=1)
    return np.asarray(idx, np.int64).reshape(H, W)


@dataclass(frozen=True)
class FilterJob:
    """One bilateral-filtering request: image shape/seed and the filter parameters."""
    H: int
    W: int
    cells: int
    ramp: float
    noise: float
    seed: int
    theta: float
    sigma: float
    K: int | None = None      # fixed order, T optimised (Fig. 1 construction)
    eps: float | None = None  # or: order chosen by Algorithm 1

    def image(self) -> np.ndarray:
        return voronoi_image(self.H, self.W, self.cells, self.ramp, self.noise, self.seed)

    @property
    def pixels(self) -> int:
        return self.H * self.W


def scaled_cells(H: int, W: int, per_256sq: float = 40.0) -> int:
    return max(1, int(round(per_256sq * H * W / (256.0 * 256.0))))


# --- the five workloads -------------------------------------------------------------
# 0: 256x256, 40 cells, ramp 40, noise 10; theta 3, sigma 30, K 4 (T optimised).
# 1: 1024x1024, 200 cells, ramp 40, noise 10; theta 5; sigma in {10,30,80}; K from eps 0.01.
# 2: 4096x4096, 2000 cells, ramp 60, noise 15; theta 10, sigma 10, K 16.
# 3: 64 images, sides log-uniform in [256, 2048] (H, W independent); theta in {2,5,10},
#    sigma in {10,30,80}; K from eps 0.01; cells scaled by area.
# 4: Poisson stream 500 req/s for 60 s, sides log-uniform in [512, 4096]; theta {2,5,10},
#    sigma {10,30,80}, K {4,8,16}.
# Seeds: workload c, image i uses seed 1000 c + i.

def workload_small() -> FilterJob:
    return FilterJob(256, 256, 40, 40.0, 10.0, 0, theta=3.0, sigma=30.0, K=4)


def workload_sigma_sweep() -> list[FilterJob]:
    return [FilterJob(1024, 1024, 200, 40.0, 10.0, 1000, theta=5.0, sigma=s, eps=0.01)
            for s in (10.0, 30.0, 80.0)]


def workload_large() -> FilterJob:
    return FilterJob(4096, 4096, 2000, 60.0, 15.0, 2000, theta=10.0, sigma=10.0, K=16)


def workload_batch(n: int = 64, lo: int = 256, hi: int = 2048) -> list[FilterJob]:
    rng = np.random.default_rng(3000)
    jobs = []
    for i in range(n):
        H = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        W = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        theta = float(rng.choice([2.0, 5.0, 10.0]))
        sigma = float(rng.choice([10.0, 30.0, 80.0]))
        jobs.append(FilterJob(H, W, scaled_cells(H, W), 40.0, 10.0, 3000 + i,
                              theta=theta, sigma=sigma, eps=0.01))
    return jobs


def workload_stream(rate: float = 500.0, duration: float = 60.0, lo: int = 512,
                    hi: int = 4096, seed: int = 4000):
    """Poisson arrivals: list of (arrival_time_s, FilterJob)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        H = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        W = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        theta = float(rng.choice([2.0, 5.0, 10.0]))
        sigma = float(rng.choice([10.0, 30.0, 80.0]))
        K = int(rng.choice([4, 8, 16]))
        out.append((t, FilterJob(H, W, scaled_cells(H, W), 40.0, 10.0, seed + i,
                                 theta=theta, sigma=sigma, K=K)))
        i += 1
    return out
