"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the
CPU oracle's tests.

This module holds no arithmetic of the rounded-KLT method: it only draws images.
The paper measured on natural 8-bit grayscale photographs from a public image
bank (Sec. 4.1); those are not available here, so every workload uses
first-order Markov (AR(1)) fields, the signal model the paper builds the KLT for
(Sec. 2.1), drawn separably along rows and columns and quantised to uint8.

Recipe (one image, seed s, correlation rho, mean 128, std 40):
  w[y, x] ~ N(0, 1) i.i.d. from numpy's PCG64 generator seeded with s;
  along each row:    v[y, 0] = w[y, 0],  v[y, x] = rho*v[y, x-1] + sqrt(1-rho^2)*w[y, x];
  along each column: f[0, x] = v[0, x],  f[y, x] = rho*f[y-1, x] + sqrt(1-rho^2)*v[y, x];
  pixel = clip(floor(128 + 40*f + 0.5), 0, 255).
The field has unit variance and separable correlation rho^|dx| * rho^|dy|.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GRID_RHOS = (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 0.95)


def _ar1_along_axis0(w: np.ndarray, rho: float) -> np.ndarray:
    """out[0] = w[0]; out[k] = rho*out[k-1] + sqrt(1-rho^2)*w[k] (rows are contiguous)."""
    out = np.empty_like(w)
    c = math.sqrt(1.0 - rho * rho)
    out[0] = w[0]
    for k in range(1, w.shape[0]):
        np.multiply(out[k - 1], rho, out=out[k])
        out[k] += c * w[k]
    return out


def ar1_field(h: int, w: int, rho: float, seed: int) -> np.ndarray:
    """Unit-variance separable AR(1) field, float64, shape (h, w)."""
    g = np.random.Generator(np.random.PCG64(seed))
    white = g.standard_normal((h, w))
    # along each row (x): run the recursion on the transposed copy
    rows = np.ascontiguousarray(_ar1_along_axis0(np.ascontiguousarray(white.T), rho).T)
    # along each column (y)
    return _ar1_along_axis0(rows, rho)


def ar1_image(h: int, w: int, rho: float = 0.95, seed: int = 0,
              mean: float = 128.0, std: float = 40.0) -> np.ndarray:
    """uint8 image of shape (h, w) drawn from the recipe in the module docstring."""
    f = ar1_field(h, w, rho, seed)
    return np.clip(np.floor(mean + std * f + 0.5), 0, 255).astype(np.uint8)


def ar1_batch(n: int, h: int, w: int, rho: float = 0.95, base_seed: int = 0) -> np.ndarray:
    """n images (n, h, w) uint8; image i uses seed base_seed + i."""
    out = np.empty((n, h, w), dtype=np.uint8)
    for i in range(n):
        out[i] = ar1_image(h, w, rho, base_seed + i)
    return out


def uniform_image(h: int, w: int, seed: int) -> np.ndarray:
    """i.i.d. uniform bytes: the worst case for the integer range of the transform."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.integers(0, 256, size=(h, w), dtype=np.uint8)


def pattern_image(kind: str, h: int, w: int) -> np.ndarray:
    """Deterministic edge-case images: constant, extremes, checkerboards, impulse."""
    y, x = np.mgrid[0:h, 0:w]
    if kind == "zeros":
        return np.zeros((h, w), np.uint8)
    if kind == "full":
        return np.full((h, w), 255, np.uint8)
    if kind == "checker":
        return (((x + y) & 1) * 255).astype(np.uint8)
    if kind == "stripes":
        return ((x & 1) * 255).astype(np.uint8)
    if kind == "impulse":
        img = np.zeros((h, w), np.uint8)
        img[::7, ::5] = 255
        return img
    if kind == "ramp":
        return ((x * 7 + y * 3) % 256).astype(np.uint8)
    raise ValueError(kind)


# --------------------------------------------------------------------------
# Workload recipes (sizes and distributions of the benchmark configurations)
# --------------------------------------------------------------------------

def single_512() -> np.ndarray:
    """One 512x512 image, rho = 0.95, seed 0."""
    return ar1_image(512, 512, 0.95, 0)


def sweep_batch(n: int = 256, side: int = 512, base_seed: int = 1000):
    """r-sweep workload: n images of side x side, image rho ~ U(0.80, 0.98).

    Returns (images uint8 (n, side, side), rhos float64 (n,))."""
    g = np.random.Generator(np.random.PCG64(base_seed - 1))
    rhos = g.uniform(0.80, 0.98, size=n)
    imgs = np.empty((n, side, side), np.uint8)
    for i in range(n):
        imgs[i] = ar1_image(side, side, float(rhos[i]), base_seed + i)
    return imgs, rhos


def rank_seeds(base_seed: int, n_per_rank: int, rank: int) -> list:
    """Seeds of one rank's images when each process of a multi-GPU run takes its own
    images: rank r takes base + r*n .. base + r*n + n - 1, so ranks never share an
    image and rank 0 alone reproduces the single-GPU workload."""
    return [base_seed + rank * n_per_rank + i for i in range(n_per_rank)]


def roofline_batch(n: int = 16, side: int = 4096, base_seed: int = 2000) -> np.ndarray:
    """Bandwidth workload: n images of side x side, rho = 0.95."""
    return ar1_batch(n, side, side, 0.95, base_seed)


@dataclass
class MixedItem:
    h: int
    w: int
    rho: float
    r: int
    seed: int


def mixed_items(n: int = 2000, lo: int = 64, hi: int = 4096, step: int = 8,
                base_seed: int = 3000, rho_lo: float = 0.5, rho_hi: float = 0.98,
                r_max: int = 64) -> list:
    """Uneven-size batch: H, W iid uniform on {lo, lo+step, ..., hi};
    rho ~ U(rho_lo, rho_hi); r ~ U{1..r_max}; seed base_seed + i."""
    g = np.random.Generator(np.random.PCG64(base_seed - 1))
    sides = np.arange(lo, hi + 1, step)
    hs = g.choice(sides, size=n)
    ws = g.choice(sides, size=n)
    rhos = g.uniform(rho_lo, rho_hi, size=n)
    rs = g.integers(1, r_max + 1, size=n)
    return [MixedItem(int(hs[i]), int(ws[i]), float(rhos[i]), int(rs[i]), base_seed + i)
            for i in range(n)]


def nearest_grid_rho(rho: float, grid=GRID_RHOS) -> float:
    """Nearest grid value; an exact tie goes to the lower value."""
    best = grid[0]
    for g_ in grid:
        if abs(g_ - rho) < abs(best - rho):
            best = g_
    return best


def lognormal_side(g: np.random.Generator, median: float = 768.0, sigma: float = 0.5,
                   lo: int = 64, hi: int = 4096, step: int = 8) -> int:
    """Side length: lognormal(median, sigma), rounded to the nearest multiple of
    step (ties up), clipped to [lo, hi]."""
    v = median * math.exp(sigma * g.standard_normal())
    m = int(math.floor(v / step + 0.5)) * step
    return int(min(max(m, lo), hi))


def serving_requests(rate_hz: float, duration_s: float, seed: int = 5000,
                     rhos=(0.5, 0.8, 0.9, 0.95), r_max: int = 64):
    """Poisson request stream: list of (arrival_s, h, w, rho, r, seed)."""
    g = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    i = 0
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        h = lognormal_side(g)
        w = lognormal_side(g)
        rho = float(rhos[int(g.integers(0, len(rhos)))])
        r = int(g.integers(1, r_max + 1))
        out.append((t, h, w, rho, r, seed + 1 + i))
        i += 1
    return out


# --------------------------------------------------------------------------
# Large pools by cropping: a window of an AR(1) field is itself an AR(1) field
# with the same rho, so many distinct images of any size come from a few large
# base fields (one per rho) without drawing each one from scratch.
# --------------------------------------------------------------------------

def base_fields(rhos, side: int = 4096, base_seed: int = 6000) -> dict:
    """{rho: uint8 side x side AR(1) image}, seed base_seed + index of rho."""
    return {float(rho): ar1_image(side, side, float(rho), base_seed + k) for k, rho in enumerate(rhos)}


def crop(base: np.ndarray, h: int, w: int, seed: int) -> np.ndarray:
    """h x w window of `base` at an offset drawn from PCG64(seed) (requires h, w <= side)."""
    g = np.random.Generator(np.random.PCG64(seed))
    y = int(g.integers(0, base.shape[0] - h + 1))
    x = int(g.integers(0, base.shape[1] - w + 1))
    return base[y:y + h, x:x + w]


def mixed_batch(items: list, bases: dict) -> list:
    """Images for mixed_items(): each a crop of the base field whose rho is the
    grid value nearest to the item's rho."""
    return [crop(bases[nearest_grid_rho(it.rho, tuple(bases))], it.h, it.w, it.seed) for it in items]


def serving_pool(n: int, bases: dict, median: float = 768.0, sigma: float = 0.5, seed: int = 5100) -> list:
    """n request images with lognormal sides (median, sigma; multiples of 8 in
    [64, 4096]) cropped from the base fields, rho cycling over the bases."""
    g = np.random.Generator(np.random.PCG64(seed))
    keys = list(bases)
    out = []
    for i in range(n):
        h = lognormal_side(g, median, sigma)
        w = lognormal_side(g, median, sigma)
        out.append(crop(bases[keys[i % len(keys)]], h, w, seed + 1 + i))
    return out
