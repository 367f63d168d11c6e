"""Shared helpers for the tests (layout conversions written from the ABI's
documented layouts, tensor plumbing).  No arithmetic of the method here."""
from __future__ import annotations

import numpy as np


def slot_table(L: int):
    """(level, band, ix, iy) of every in-tile slot: slot = (band << 2m) + (iy << m) + ix,
    m = L - level, band 0 only at slot 0 (include/wasabi.h)."""
    n = 1 << (2 * L)
    lev = np.empty(n, np.int64)
    band = np.empty(n, np.int64)
    ix = np.empty(n, np.int64)
    iy = np.empty(n, np.int64)
    lev[0], band[0], ix[0], iy[0] = L, 0, 0, 0
    for l in range(1, L + 1):
        m = L - l
        for b in (1, 2, 3):
            for qy in range(1 << m):
                for qx in range(1 << m):
                    s = (b << (2 * m)) + (qy << m) + qx
                    lev[s], band[s], ix[s], iy[s] = l, b, qx, qy
    return lev, band, ix, iy


def tile_major_to_mallat(wbuf: np.ndarray, w: int, h: int, L: int) -> np.ndarray:
    """Permute a tile-major wavelet buffer into the whole-image Mallat layout."""
    lev, band, ix, iy = slot_table(L)
    TSL = 1 << (2 * L)
    ntx, nty = w >> L, h >> L
    buf = wbuf.reshape(nty, ntx, TSL)
    TY, TX = np.meshgrid(np.arange(nty), np.arange(ntx), indexing="ij")
    m = L - lev
    P = (TX[..., None] << m) + ix
    Q = (TY[..., None] << m) + iy
    Sx, Sy = w >> lev, h >> lev
    col = P + np.where((band == 1) | (band == 3), Sx, 0)
    row = Q + np.where((band == 2) | (band == 3), Sy, 0)
    out = np.zeros((h, w), wbuf.dtype)
    out[row, col] = buf
    return out


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))
