"""Seeded synthetic inputs: ellipse phantoms, detector noise, workload shapes.

This module holds none of the reconstruction method's arithmetic.  It draws
random numbers and lays out workloads; the sinogram itself is produced by a
projector the caller passes in (the CUDA projector for the product path, the
FP64 oracle in tests), so that each side builds its data with its own ``A``.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser constants
of Vigna's public-domain ``splitmix64``), used as a counter-based generator:
draw k of stream (seed, tag) is ``mix(key(seed, tag) + (k+1) * golden)``.
Normals use the Box-Muller transform.

The paper (Sec. 4) does not describe its phantom; these seeded ellipse
phantoms, with the shapes of its workloads, stand in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _key(seed: int, tag: str) -> np.uint64:
    h = seed & _MASK
    for ch in tag.encode():
        h = (h * 0x100000001B3 + ch) & _MASK      # FNV-style fold of the tag
    return _mix(np.array([h], dtype=np.uint64))[0]


def uniform(seed: int, tag: str, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``count`` draws in [lo, hi) from stream (seed, tag)."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(seed, tag) + k * _GOLDEN
    u = (_mix(z) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, tag: str, count: int) -> np.ndarray:
    """``count`` standard normals from stream (seed, tag), Box-Muller."""
    m = (count + 1) // 2
    u = uniform(seed, tag, 2 * m)
    u1 = 1.0 - u[0::2]                      # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * math.pi * u2)
    z[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return z[:count]


def ellipse_phantom(n: int, n_ellipses: int, seed: int) -> np.ndarray:
    """N x N phantom: sum of ``n_ellipses`` random ellipses, clipped at 0.

    Per ellipse, in draw order: centre cx, cy ~ U[-0.8, 0.8], semi-axes
    ax, ay ~ U[0.05, 0.5], rotation phi ~ U[0, pi), density rho ~ U[-0.5, 1],
    in coordinates normalised to the image half-width (u = xc/(N/2),
    v = yc/(N/2)); each ellipse is point-sampled at the pixel centres.
    """
    p = uniform(seed, "ellipses", 6 * n_ellipses).reshape(n_ellipses, 6)
    half = 0.5 * n
    idx = np.arange(n) - 0.5 * (n - 1)
    v, u = np.meshgrid(idx / half, idx / half, indexing="ij")   # v: rows, u: columns
    img = np.zeros((n, n))
    for e in range(n_ellipses):
        cx = -0.8 + 1.6 * p[e, 0]
        cy = -0.8 + 1.6 * p[e, 1]
        ax = 0.05 + 0.45 * p[e, 2]
        ay = 0.05 + 0.45 * p[e, 3]
        phi = math.pi * p[e, 4]
        rho = -0.5 + 1.5 * p[e, 5]
        du, dv = u - cx, v - cy
        cu = du * math.cos(phi) + dv * math.sin(phi)
        cv = -du * math.sin(phi) + dv * math.cos(phi)
        img += rho * ((cu / ax) ** 2 + (cv / ay) ** 2 <= 1.0)
    return np.maximum(img, 0.0)


def bins_for(n: int) -> int:
    """Detector bins covering the image diagonal: ceil(sqrt(2) * N)."""
    return int(math.ceil(math.sqrt(2.0) * n))


@dataclass
class Workload:
    """One reconstruction problem's shape and noise recipe."""
    name: str
    n: int
    n_angles: int
    n_bins: int
    n_ellipses: int
    noise_frac: float          # sigma = noise_frac * max(A x_true)
    eps_factor: float          # eps = eps_factor * L * sigma^2 / 2
    max_iter: int = 100
    notes: str = ""

    @property
    def J(self) -> int:
        return self.n * self.n

    @property
    def L(self) -> int:
        return self.n_angles * self.n_bins


# Workload shapes (each a synthetic stand-in for the paper's unnamed phantom).
SMALL_FP64 = Workload("ellipse64_a90_b95", 64, 90, 95, 10, 0.01, 1.05, 100,
                      "64x64, 10 ellipses, 90 angles x 95 bins, 1% noise")
SINGLE_512 = Workload("ellipse512_a720_b725", 512, 720, 725, 20, 0.005, 1.05, 100,
                      "512x512, 20 ellipses, 720 angles x 725 bins, 0.5% noise")
MIXED_1024 = Workload("ellipse1024_a1440_b1449", 1024, 1440, 1449, 40, 0.005, 1.05, 100,
                      "1024x1024, 40 ellipses, 1440 angles x 1449 bins, 0.5% noise")
PAPER_512 = Workload("paper512_a256_b512", 512, 256, 512, 20, 0.05, 2.0, 100,
                     "the paper's Sec. 4 shape: 512x512, 256 angles x 512 rays")

BATCH_SIZES = (128, 192, 256, 384, 512, 768)
BATCH_ANGLES = (60, 120, 180, 360, 720)


def batch_workloads(count: int, seed: int) -> list[Workload]:
    """Uneven batch: N ~ U{128,...,768}, angles ~ U{60,...,720}, 1% noise."""
    u = uniform(seed, "batch", 2 * count).reshape(count, 2)
    out = []
    for q in range(count):
        n = BATCH_SIZES[int(u[q, 0] * len(BATCH_SIZES))]
        na = BATCH_ANGLES[int(u[q, 1] * len(BATCH_ANGLES))]
        out.append(Workload(f"batch{q}_n{n}_a{na}", n, na, bins_for(n), 10, 0.01, 1.05, 100))
    return out


def serving_workloads(count: int, seed: int, n_min: int = 128, n_max: int = 1024,
                      a_min: int = 30, a_max: int = 180) -> list[Workload]:
    """Few-view request stream: N ~ U{n_min..n_max step 64}, angles ~ U{a_min..a_max},
    eps factor ~ U[1.02, 1.2], 1% noise."""
    u = uniform(seed, "serving", 3 * count).reshape(count, 3)
    sizes = list(range(n_min, n_max + 1, 64))
    out = []
    for q in range(count):
        n = sizes[int(u[q, 0] * len(sizes))]
        na = a_min + int(u[q, 1] * (a_max - a_min + 1))
        ef = 1.02 + 0.18 * u[q, 2]
        out.append(Workload(f"req{q}_n{n}_a{na}", n, na, bins_for(n), 10, 0.01, ef, 100))
    return out


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with ``rate`` requests/s."""
    u = uniform(seed, "arrivals", count)
    gaps = -np.log(1.0 - u) / rate
    return np.cumsum(gaps)


@dataclass
class Problem:
    work: Workload
    seed: int
    x_true: np.ndarray
    y: np.ndarray
    sigma: float
    eps: float


def make_problem(work: Workload, seed: int,
                 project: Callable[[np.ndarray, int, int], np.ndarray]) -> Problem:
    """Phantom, then noisy data y = A x_true + sigma * n with the caller's ``A``.

    ``project(x, n_angles, n_bins)`` returns the clean sinogram as an array of
    shape (n_angles, n_bins).
    """
    x_true = ellipse_phantom(work.n, work.n_ellipses, seed)
    clean = np.asarray(project(x_true, work.n_angles, work.n_bins), dtype=np.float64)
    sigma = work.noise_frac * float(np.max(clean))
    noise = normal(seed, "noise", work.L).reshape(work.n_angles, work.n_bins)
    y = clean + sigma * noise
    eps = work.eps_factor * work.L * sigma * sigma / 2.0
    return Problem(work, seed, x_true, y, sigma, eps)
