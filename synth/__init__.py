"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *generates inputs*: phase masks (uint8, 1 = inclusion phase 1,
0 = matrix phase 2) and lists of inclusion conductivities.  It contains none of
the solver's arithmetic (no Fourier transform, no Green operator, no scheme),
so that the FP64 oracle and the CUDA path can both draw the same inputs without
sharing any code of the method itself.

Array convention: a 2-D mask has shape (n_y, n_x) and a 3-D mask has shape
(n_z, n_y, n_x); x is the fastest-varying (last) axis.

Workloads follow the paper's model example (a periodic square array of squares
at 25 % volume fraction, section "The numerical example of Moulinec and
Suquet") and its 3-D analogue, plus the random microstructures used for the
batched sweep and the gradient check.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "square_array_mask",
    "laminate_mask",
    "random_mask",
    "rsa_disk_mask",
    "bernoulli_majority_mask",
    "complex_sigma_ray",
    "SIGMA1_SWEEP_2D",
    "SIGMA1_SWEEP_3D",
]

# Inclusion conductivities of the 2-D and 3-D square/cubic-array workloads.
SIGMA1_SWEEP_2D = (0.01, 0.1, 10.0, 100.0, 1.0e4)
SIGMA1_SWEEP_3D = (5.0, 50.0, 500.0)


def square_array_mask(n: int, d: int = 2) -> np.ndarray:
    """Centred square (d=2) or cube (d=3) of side n/2 in a periodic cell of n^d voxels.

    The inclusion occupies indices [n/4, 3n/4) on every axis, so its volume
    fraction is exactly 1/4 in 2-D and 1/8 in 3-D.  n must be divisible by 4.
    This is the paper's square array of squares at 25 % volume fraction.
    """
    if n % 4 != 0:
        raise ValueError("square_array_mask needs n divisible by 4")
    if d not in (2, 3):
        raise ValueError("d must be 2 or 3")
    line = np.zeros(n, dtype=np.uint8)
    line[n // 4 : 3 * n // 4] = 1
    if d == 2:
        return np.ascontiguousarray(line[:, None] & line[None, :])
    return np.ascontiguousarray(line[:, None, None] & line[None, :, None] & line[None, None, :])


def laminate_mask(shape, width: int, axis: int) -> np.ndarray:
    """Layers of phase 1 of thickness `width` alternating with phase 2 layers of
    the same thickness, stacked along array axis `axis` (0 = slowest)."""
    shape = tuple(int(s) for s in shape)
    n = shape[axis]
    if n % (2 * width) != 0:
        raise ValueError("laminate needs the axis length divisible by 2*width")
    idx = np.arange(n)
    layer = ((idx // width) % 2 == 0).astype(np.uint8)
    bshape = [1] * len(shape)
    bshape[axis] = n
    return np.ascontiguousarray(np.broadcast_to(layer.reshape(bshape), shape).astype(np.uint8))


def random_mask(shape, p: float, seed: int) -> np.ndarray:
    """Independent Bernoulli(p) inclusion voxels."""
    rng = np.random.default_rng(seed)
    return (rng.random(tuple(shape)) < p).astype(np.uint8)


def rsa_disk_mask(n: int, seed: int, r_range=(0.03, 0.06), gap: float = 0.02,
                  f_range=(0.25, 0.35), max_rejects: int = 1_000_000) -> tuple[np.ndarray, dict]:
    """Random sequential addition of non-overlapping disks in the periodic unit square.

    Radii are uniform in r_range (in units of the cell side L=1), every pair of
    disks keeps an edge-to-edge gap of at least `gap` (periodic minimum-image
    distance), and disks are added until the covered area reaches a target
    fraction drawn uniformly from f_range.  After `max_rejects` consecutive
    rejections the attempt restarts with the next sub-seed.  A voxel belongs to
    phase 1 when its centre lies inside a disk.  Returns (mask, info).
    """
    sub = 0
    while True:
        rng = np.random.default_rng([seed, sub])
        target = rng.uniform(*f_range)
        cx, cy, rad = [], [], []
        area = 0.0
        rejects = 0
        ok = True
        while area < target:
            r = rng.uniform(*r_range)
            x, y = rng.random(2)
            if cx:
                dx = np.abs(np.asarray(cx) - x)
                dy = np.abs(np.asarray(cy) - y)
                dx = np.minimum(dx, 1.0 - dx)
                dy = np.minimum(dy, 1.0 - dy)
                dist = np.sqrt(dx * dx + dy * dy)
                if np.any(dist < np.asarray(rad) + r + gap):
                    rejects += 1
                    if rejects >= max_rejects:
                        ok = False
                        break
                    continue
            rejects = 0
            cx.append(x)
            cy.append(y)
            rad.append(r)
            area += math.pi * r * r
        if ok:
            break
        sub += 1
    c = (np.arange(n) + 0.5) / n
    X = c[None, :]
    Y = c[:, None]
    mask = np.zeros((n, n), dtype=bool)
    for x, y, r in zip(cx, cy, rad):
        dx = np.abs(X - x)
        dy = np.abs(Y - y)
        dx = np.minimum(dx, 1.0 - dx)
        dy = np.minimum(dy, 1.0 - dy)
        mask |= dx * dx + dy * dy < r * r
    info = {"disks": len(rad), "target_fraction": float(target), "area_fraction": float(area),
            "voxel_fraction": float(mask.mean()), "sub_seed": sub}
    return mask.astype(np.uint8), info


def bernoulli_majority_mask(n: int, p: float = 0.2, seed: int = 5, threshold: int = 14) -> np.ndarray:
    """3-D Bernoulli(p) voxels smoothed by one periodic 3x3x3 majority filter.

    A voxel is kept in phase 1 when at least `threshold` of the 27 voxels of
    its periodic 3x3x3 neighbourhood (itself included) are phase 1.
    """
    rng = np.random.default_rng(seed)
    b = (rng.random((n, n, n)) < p).astype(np.int16)
    count = np.zeros_like(b)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                count += np.roll(b, (dz, dy, dx), axis=(0, 1, 2))
    return (count >= threshold).astype(np.uint8)


def complex_sigma_ray(count: int = 512, seed: int = 1000, log10_r=(-2.0, 2.0),
                      theta=(0.05, math.pi - 0.05)) -> np.ndarray:
    """Complex inclusion conductivities r*exp(i*theta), log10 r and theta uniform."""
    rng = np.random.default_rng(seed)
    r = 10.0 ** rng.uniform(*log10_r, size=count)
    th = rng.uniform(*theta, size=count)
    return r * np.exp(1j * th)
