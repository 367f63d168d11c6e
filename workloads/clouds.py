"""Seeded synthetic point clouds with the geometry of the paper's workloads.

The paper's 3-D model (an image-type hologram scene of about 10^5 points,
Sec. 2) is not available, so two stand-ins are generated:

* ``uniform_cloud`` — x, y uniform integer pixels, z uniform in [zmin, zmax];
* ``heightfield_cloud`` — points on a smooth surface: distinct pixels drawn
  uniformly without replacement, z taken from a sum of 32 random Gaussian
  bumps rescaled to span [zmin, zmax].

Amplitudes are a = 1 - U[0, 1), i.e. uniform in (0, 1].  Every draw comes
from one SplitMix64 stream per cloud, at fixed offsets, so a cloud is a pure
function of (seed, sizes).  Points are returned as a dict of numpy arrays:
x, y (int32 pixel indices), z (float64 metres) and a (float32).
"""
from __future__ import annotations

import numpy as np

from .splitmix import splitmix64, uniform01

_NG = 32  # Gaussian bumps in a height field


def _ints(seed: int, n: int, hi: int, start: int) -> np.ndarray:
    return np.floor(uniform01(seed, n, start) * hi).astype(np.int64)


def uniform_cloud(seed: int, N: int, Nh: int, zmin: float, zmax: float) -> dict:
    x = _ints(seed, N, Nh, 0).astype(np.int32)
    y = _ints(seed, N, Nh, N).astype(np.int32)
    z = zmin + uniform01(seed, N, 2 * N) * (zmax - zmin)
    a = (1.0 - uniform01(seed, N, 3 * N)).astype(np.float32)
    return {"x": x, "y": y, "z": z, "a": a}


def _distinct_pixels(seed: int, N: int, Nh: int, start: int) -> np.ndarray:
    total = Nh * Nh
    if N > total:
        raise ValueError("more points than pixels")
    got = np.empty(0, np.int64)
    drawn = 0
    batch = max(16, int(N * 1.05) + 64)
    while got.size < N:
        cand = _ints(seed, batch, total, start + drawn)
        drawn += batch
        allc = np.concatenate([got, cand])
        _, first = np.unique(allc, return_index=True)
        got = allc[np.sort(first)]
    return got[:N]


def heightfield_cloud(seed: int, N: int, Nh: int, zmin: float, zmax: float) -> dict:
    g = uniform01(seed, 4 * _NG, 0).reshape(4, _NG)
    mx, my = g[0] * Nh, g[1] * Nh
    sig = Nh / 32.0 + g[2] * (Nh / 4.0 - Nh / 32.0)
    amp = 2.0 * g[3] - 1.0
    lin = _distinct_pixels(seed, N, Nh, 1024)
    x = (lin % Nh).astype(np.int32)
    y = (lin // Nh).astype(np.int32)
    xf, yf = x.astype(np.float64), y.astype(np.float64)
    h = np.zeros(N, np.float64)
    for k in range(_NG):
        h += amp[k] * np.exp(-((xf - mx[k]) ** 2 + (yf - my[k]) ** 2) / (2.0 * sig[k] ** 2))
    lo, hi = (h.min(), h.max()) if N else (0.0, 0.0)
    t = (h - lo) / (hi - lo) if hi > lo else np.zeros_like(h)
    z = np.clip(zmin + t * (zmax - zmin), zmin, zmax)
    a = (1.0 - uniform01(seed ^ 0x5A5A5A5A, N, 0)).astype(np.float32)
    return {"x": x, "y": y, "z": z, "a": a}


def aligned(points: dict, step: int) -> dict:
    """A copy with x and y rounded down to multiples of ``step``."""
    out = dict(points)
    out["x"] = (points["x"] // step * step).astype(np.int32)
    out["y"] = (points["y"] // step * step).astype(np.int32)
    return out
