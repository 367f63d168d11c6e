"""Element-wise error bounds for comparing the GPU hologram with the oracle.

Both sides compute Eq. (2) in FP32, but differently: the oracle adds a_j c_k
into an FP32 buffer point by point; the GPU forms a_j c_k in FP32, scales it
by a power of two 2^sh chosen per super-tile, rounds it to an integer and
adds integers exactly.  A pixel of the two results may therefore differ by at
most the sum, over the wavelet cells that build it, of

* the fixed-point rounding: half a quantum 2^-sh per contribution;
* FP32 rounding of the products and of the oracle's running sums: at most
  (n + 2) units of 2^-24 of sum |a_j c_k| for a cell with n contributions;

carried through the inverse transform with absolute values (each level adds
the four children's bounds and halves them, like the orthonormal inverse
Haar), plus the rounding of the inverse itself on both sides.

The quantum is bounded without reading the kernel's choice: the scale keeps
(candidate points within reach) x max|a| x max|c| below 2^31, so
2^-sh <= 2 (candidates) max|a| max|c| / 2e9 (x2 for the logarithm's rounding),
and the candidates of any super-tile (at most 256 pixels wide) that holds a
pixel lie within 512 + reach pixels of it.  The bound is loose by that
factor only; a dropped, duplicated or misplaced coefficient of any
point with a_j |c_k| above it still fails the check.

This module holds error analysis, not the method: it calls the oracle's
superposition on a magnitude-valued and a count-valued copy of its LUT.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

U32 = 2.0 ** -24
BLOCK = 64  # pixels per side of the blocks the quantum bound is taken over


def _abs_inverse(a: np.ndarray, L: int) -> np.ndarray:
    """Propagate non-negative per-coefficient bounds through the inverse Haar
    transform of a Mallat-layout buffer: every output of a level gets half
    the sum of its four inputs."""
    a = np.array(a, np.float64)
    n = a.shape[0]
    for lev in range(L, 0, -1):
        S = n >> lev
        s = a[:S, :S]
        t = (s + a[:S, S:2 * S] + a[S:2 * S, :S] + a[S:2 * S, S:2 * S]) * 0.5
        a[:2 * S, :2 * S] = np.kron(t, np.ones((2, 2)))
    return a


def _point_box_counts(pts: dict, Nh: int) -> np.ndarray:
    """2-D prefix sums of point counts over BLOCK x BLOCK blocks (points
    outside the hologram clamp to its border blocks, which only loosens)."""
    nb = (Nh + BLOCK - 1) // BLOCK
    bx = np.clip(pts["x"].astype(np.int64) // BLOCK, 0, nb - 1)
    by = np.clip(pts["y"].astype(np.int64) // BLOCK, 0, nb - 1)
    h = np.zeros((nb, nb), np.int64)
    np.add.at(h, (by, bx), 1)
    c = np.zeros((nb + 1, nb + 1), np.int64)
    c[1:, 1:] = h.cumsum(0).cumsum(1)
    return c


def _quantum_bound(counts, Nh: int, x0: int, y0: int, Ns: int, reach: int, amax: float, cmax: float):
    """Upper bound of the fixed-point quantum per BLOCK x BLOCK block of the
    window [x0, x0 + Ns) x [y0, y0 + Ns)."""
    nb = counts.shape[0] - 1
    nbw = Ns // BLOCK
    q = np.empty((nbw, nbw))
    m = 512 + reach
    for j in range(nbw):
        for i in range(nbw):
            px0, py0 = x0 + i * BLOCK, y0 + j * BLOCK
            lo_x = max(0, (px0 - m) // BLOCK)
            hi_x = min(nb, (px0 + BLOCK + m + BLOCK - 1) // BLOCK)
            lo_y = max(0, (py0 - m) // BLOCK)
            hi_y = min(nb, (py0 + BLOCK + m + BLOCK - 1) // BLOCK)
            tot = counts[hi_y, hi_x] - counts[lo_y, hi_x] - counts[hi_y, lo_x] + counts[lo_y, lo_x]
            q[j, i] = max(2.0 ** -30, 4.0 * float(tot) * amax * cmax / 2.0e9)
    return np.kron(q, np.ones((BLOCK, BLOCK)))


class FieldBound:
    """Per-pixel bound of |u_gpu - u_oracle| on sampled sub-holograms of one
    hologram (the oracle LUT, points and side fixed at construction)."""

    def __init__(self, orc, olut, pts: dict, Nh: int, rule: int = 0):
        self.orc = orc
        self.L = olut.L
        self.Nh = Nh
        self.rule = rule
        self.pts_abs = dict(pts, a=np.abs(pts["a"]).astype(np.float32))
        self.pts_one = dict(pts, a=np.ones_like(pts["a"], np.float32))
        v = olut.val
        mag = np.abs(v.astype(np.complex128)).astype(np.float32)
        self.lut_abs = replace(olut, val=mag.astype(np.complex64))
        self.lut_one = replace(olut, val=np.ones(v.shape, np.complex64))
        self.reach = olut.W // 2 + (2 << olut.L)
        self.amax = float(np.abs(pts["a"]).max()) if pts["a"].size else 0.0
        self.cmax = float(np.max(np.maximum(np.abs(v.real), np.abs(v.imag)))) if v.size else 0.0
        self.counts = _point_box_counts(pts, Nh)

    def _parts(self, Ns: int, s: int, t: int):
        ox, oy = s * Ns, t * Ns
        mabs = self.orc.superpose(self.lut_abs, self.pts_abs, Ns, ox=ox, oy=oy, rule=self.rule).real
        ncnt = self.orc.superpose(self.lut_one, self.pts_one, Ns, ox=ox, oy=oy, rule=self.rule).real
        q = _quantum_bound(self.counts, self.Nh, ox, oy, Ns, self.reach, self.amax, self.cmax)
        return mabs.astype(np.float64), np.rint(ncnt.astype(np.float64)), q

    def coeffs(self, Ns: int, s: int, t: int) -> np.ndarray:
        """Bound per wavelet coefficient (Mallat layout) of sub-hologram
        (s, t): the quantum of the block under the coefficient's footprint."""
        mabs, ncnt, q = self._parts(Ns, s, t)
        qc = np.empty_like(q)
        n = Ns
        qc[:n >> self.L, :n >> self.L] = q[::1 << self.L, ::1 << self.L]
        for lev in range(1, self.L + 1):
            S = n >> lev
            ql = q[::1 << lev, ::1 << lev]
            qc[:S, S:2 * S] = ql
            qc[S:2 * S, :S] = ql
            qc[S:2 * S, S:2 * S] = ql
        return ncnt * (0.5 * qc) + (ncnt + 3.0) * mabs * U32

    def window(self, Ns: int, s: int, t: int) -> np.ndarray:
        """Bound for sub-hologram (s, t) of side Ns (a multiple of BLOCK)."""
        mabs, ncnt, q = self._parts(Ns, s, t)
        # q is constant over each block and every coefficient's footprint
        # (at most 2^L <= BLOCK pixels) lies in one block, so the quantum
        # term can be propagated as counts and scaled afterwards.
        b_quant = _abs_inverse(ncnt, self.L) * (0.5 * q)
        b_round = _abs_inverse((ncnt + 2.0) * mabs, self.L) * U32
        b_inv = _abs_inverse(mabs, self.L) * (6.0 * self.L * U32)
        return b_quant + b_round + b_inv


def check_field(got: np.ndarray, ref: np.ndarray, bound: np.ndarray, factor: float = 2.0) -> int:
    """Assert |got - ref| <= factor * bound for the real and imaginary parts
    of every pixel; returns the number of pixels checked."""
    g = np.asarray(got, np.complex128)
    r = np.asarray(ref, np.complex128)
    for part in (np.real, np.imag):
        err = np.abs(part(g) - part(r))
        bad = err > factor * bound
        assert not bad.any(), (f"{int(bad.sum())} pixels beyond the element-wise bound; worst "
                               f"{float((err / np.maximum(bound, 1e-300)).max()):.3g} x bound")
    return g.size


def check_bits(bits_window: np.ndarray, ref: np.ndarray, bound: np.ndarray, factor: float = 2.0) -> int:
    """Binarised pixels (bool, row-major window) against Re(ref) > 0: a pixel
    may differ only where |Re ref| is within factor * bound of zero.
    Returns the number of differing pixels."""
    want = np.real(ref) > 0
    diff = bits_window != want
    if diff.any():
        margin = np.abs(np.real(ref))[diff]
        assert np.all(margin <= factor * bound[diff]), (
            f"{int(diff.sum())} flipped bits, {int((margin > factor * bound[diff]).sum())} "
            f"beyond the element-wise bound")
    return int(diff.sum())
