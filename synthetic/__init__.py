"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the bench.

This module holds none of the decomposition's arithmetic: it only draws images and workload
parameters. The images stand in for the paper's greyscale MS COCO crops and BSDS500 / ellipse
images (Sec. 4.1, App. B), which are not available: piecewise-constant disks and axis-aligned
rectangles of random size and contrast on a zero background (TV eigenfunction-like
structures, Sec. 2.1), plus additive Gaussian noise.

Recipe (``make_image``): ``numpy.random.default_rng(seed)``; shapes painted in order (later
ones overwrite); each shape is a disk or a rectangle with probability 1/2; its centre is
uniform over the image; a disk has radius r ~ U(r_lo, r_hi) and covers the pixels with
``(i+.5-cy)^2 + (j+.5-cx)^2 <= r^2``; a rectangle has independent half-sides ~ U(r_lo, r_hi);
its value is a contrast ~ U(c_lo, 1); then i.i.d. N(0, sigma^2) noise is added. float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

INF = float("inf")

# Dyadic t-edges for the 6 bands of Sec. 4.1 ("combined dyadically"): {0,1,2,4,8,16,inf}.
DYADIC_EDGES = (0.0, 1.0, 2.0, 4.0, 8.0, 16.0, INF)


def make_image(H: int, W: int, n_shapes: int, r_range, c_range=(0.1, 1.0), sigma: float = 0.01,
               seed: int = 0) -> np.ndarray:
    """Piecewise-constant disks/rectangles + Gaussian noise, float32 (see module docstring).

    Each shape's pixel test is evaluated only inside its bounding box (plus one pixel); the
    test itself, and so the image, is the same as evaluating it everywhere.
    """
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W), dtype=np.float64)
    r_lo, r_hi = r_range
    c_lo, c_hi = c_range

    def box(c, h, n):
        lo = max(0, int(np.floor(c - h - 0.5)) - 1)
        hi = min(n, int(np.ceil(c + h - 0.5)) + 2)
        return lo, hi

    for _ in range(n_shapes):
        is_disk = rng.random() < 0.5
        cy = rng.uniform(0.0, H)
        cx = rng.uniform(0.0, W)
        c = rng.uniform(c_lo, c_hi)
        if is_disk:
            r = rng.uniform(r_lo, r_hi)
            i0, i1 = box(cy, r, H)
            j0, j1 = box(cx, r, W)
            ii = (np.arange(i0, i1, dtype=np.float64) + 0.5)[:, None]
            jj = (np.arange(j0, j1, dtype=np.float64) + 0.5)[None, :]
            mask = (ii - cy) ** 2 + (jj - cx) ** 2 <= r * r
        else:
            hy = rng.uniform(r_lo, r_hi)
            hx = rng.uniform(r_lo, r_hi)
            i0, i1 = box(cy, hy, H)
            j0, j1 = box(cx, hx, W)
            ii = (np.arange(i0, i1, dtype=np.float64) + 0.5)[:, None]
            jj = (np.arange(j0, j1, dtype=np.float64) + 0.5)[None, :]
            mask = (np.abs(ii - cy) <= hy) & (np.abs(jj - cx) <= hx)
        if i1 > i0 and j1 > j0:
            img[i0:i1, j0:j1][mask] = c
    if sigma > 0:
        img = img + rng.normal(0.0, sigma, size=(H, W))
    return img.astype(np.float32)


def disk_image(H: int, W: int, radius: float, height: float, cy=None, cx=None) -> np.ndarray:
    """One disk of the given radius and height centred in a zero background (float32)."""
    cy = H / 2.0 if cy is None else cy
    cx = W / 2.0 if cx is None else cx
    ii = (np.arange(H, dtype=np.float64) + 0.5)[:, None]
    jj = (np.arange(W, dtype=np.float64) + 0.5)[None, :]
    img = np.where((ii - cy) ** 2 + (jj - cx) ** 2 <= radius * radius, height, 0.0)
    return img.astype(np.float32)


@dataclass
class Job:
    """One decomposition: the image and its TV-flow schedule."""
    f: np.ndarray
    dt: float
    K: int
    n_inner: int
    edges: tuple
    seed: int = 0

    @property
    def px_iters(self) -> int:
        return int(self.f.size) * self.K * self.n_inner


@dataclass
class Workload:
    name: str
    jobs: list = field(default_factory=list)
    description: str = ""

    @property
    def px_iters(self) -> int:
        return sum(j.px_iters for j in self.jobs)


def config0(seed: int = 0) -> Workload:
    """64x64, 6 shapes r~U(3,16), c~U(0.1,1), sigma .01; K=20, dt=.5, 200 iters; 4 bands."""
    f = make_image(64, 64, 6, (3.0, 16.0), (0.1, 1.0), 0.01, seed)
    job = Job(f, 0.5, 20, 200, (0.0, 2.0, 5.0, 10.0, INF), seed)
    return Workload("config0_64x64_K20_it200", [job], "plain 64^2")


def config1(seed: int = 1000, H: int = 512, W: int = 512, K: int = 50, n_inner: int = 300,
            n_shapes: int = 40) -> Workload:
    """512x512, 40 shapes r~U(2,60), c~U(.05,1), sigma .02; K=50, dt=.5, 300 iters; 6 bands."""
    f = make_image(H, W, n_shapes, (2.0, 60.0), (0.05, 1.0), 0.02, seed)
    job = Job(f, 0.5, K, n_inner, DYADIC_EDGES, seed)
    return Workload(f"config1_{H}x{W}_K{K}_it{n_inner}", [job], "plain single image")


def m1024(seed: int = 5000) -> Workload:
    """1024x1024, config-1 generator with 160 shapes; K=50, dt=.5, 300 iters; 6 bands."""
    f = make_image(1024, 1024, 160, (2.0, 60.0), (0.05, 1.0), 0.02, seed)
    return Workload("m1024_1024x1024_K50_it300", [Job(f, 0.5, 50, 300, DYADIC_EDGES, seed)],
                    "1024^2 decomposition")


def config2(seed: int = 2000, n_images: int = 64, size_range=(128, 1024),
            K_range=(20, 60), n_inner: int = 300) -> Workload:
    """64 images, H,W ~ U{128..1024}; shapes scale with area; K~U{20..60}; dt~U{.25,.5,1}."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n_images):
        H = int(rng.integers(size_range[0], size_range[1] + 1))
        W = int(rng.integers(size_range[0], size_range[1] + 1))
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        dt = float(rng.choice([0.25, 0.5, 1.0]))
        n_shapes = max(1, int(round(40 * H * W / (512 * 512))))
        f = make_image(H, W, n_shapes, (2.0, 60.0), (0.05, 1.0), 0.02, seed * 100 + j)
        jobs.append(Job(f, dt, K, n_inner, DYADIC_EDGES, seed * 100 + j))
    return Workload(f"config2_batch{n_images}", jobs, "batched uneven sizes")


def config3(seed: int = 3000, H: int = 2048, W: int = 2048, K: int = 50,
            n_inner: int = 500) -> Workload:
    """2048x2048, 400 shapes r~U(2,200), sigma .02; K=50, dt=.5, 500 iters; 6 bands."""
    n_shapes = max(1, int(round(400 * H * W / (2048 * 2048))))
    f = make_image(H, W, n_shapes, (2.0, 200.0), (0.05, 1.0), 0.02, seed)
    return Workload(f"config3_{H}x{W}_K{K}_it{n_inner}",
                    [Job(f, 0.5, K, n_inner, DYADIC_EDGES, seed)], "precision study")


def serving_requests(n: int, rate_per_s: float, seed: int = 4000,
                     sizes=(256, 512, 1024, 2048), weights=(0.4, 0.3, 0.2, 0.1),
                     K_range=(20, 50), n_inner: int = 300):
    """Poisson arrivals for the serving workload: list of (arrival_s, Job)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for j in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        s = int(rng.choice(sizes, p=np.asarray(weights) / np.sum(weights)))
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        n_shapes = max(1, int(round(40 * s * s / (512 * 512))))
        f = make_image(s, s, n_shapes, (2.0, 60.0), (0.05, 1.0), 0.02, seed * 1000 + j)
        out.append((t, Job(f, 0.5, K, n_inner, DYADIC_EDGES, seed * 1000 + j)))
    return out


def band_index_ranges(dt: float, K: int, edges) -> list:
    """For each band m, the list of k in 1..K-1 with edges[m] <= k*dt < edges[m+1].

    Pure bookkeeping on the time grid t_k = k*dt (no image arithmetic): used by tests to
    state which phi_k each band collects.
    """
    out = []
    for m in range(len(edges) - 1):
        lo, hi = edges[m], edges[m + 1]
        out.append([k for k in range(1, K) if lo <= k * float(dt) < hi])
    return out


def finite_edges(edges) -> list:
    return [e for e in edges if math.isfinite(e)]
