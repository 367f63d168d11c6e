"""Pins of the oracle's coiflet transform (reading R14: order 1, periodic
filter banks) and of WASABI with it: the taps solve the defining equations,
the transform is orthonormal (perfect reconstruction, Parseval), it has the
vanishing moments that define a coiflet (which fixes the tap centring), and
with every coefficient kept and points on the 2^L grid WASABI equals Eq. (1)."""
import numpy as np
import pytest

LAM, PITCH = 633e-9, 1e-6


def test_taps_solve_the_coiflet_equations(orc):
    h, g = orc.coif1_taps()
    k = np.arange(-2, 4)
    assert abs(h.sum() - np.sqrt(2)) <= 1e-15
    assert abs(h @ h - 1) <= 1e-15
    assert abs(h[:-2] @ h[2:]) <= 1e-15 and abs(h[:-4] @ h[4:]) <= 1e-15
    assert abs(((-1.0) ** k * k) @ h) <= 1e-15   # second vanishing wavelet moment
    assert abs(((-1.0) ** k) @ h) <= 1e-15       # first (zeroth moment)
    assert abs(k @ h) <= 1e-15                   # vanishing first scaling moment
    assert np.allclose(g, [(-1.0) ** kk * h[(1 - kk) + 2] for kk in k], atol=0)
    assert h.argmax() == 2                       # the root whose largest tap is h_0


@pytest.mark.parametrize("n,L", [(64, 3), (8, 3), (32, 1)])
def test_perfect_reconstruction_and_parseval(orc, n, L):
    rng = np.random.default_rng(n + L)
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    c = orc.wavelet_fwd(a, L, "coif1")
    assert abs(np.sum(np.abs(c) ** 2) - np.sum(np.abs(a) ** 2)) <= 1e-12 * np.sum(np.abs(a) ** 2)
    assert np.max(np.abs(orc.wavelet_inv(c, L, "coif1") - a)) <= 1e-13
    assert np.max(np.abs(c - orc.wavelet_fwd(a, L, "haar"))) > 1e-3  # not the Haar transform


def test_vanishing_moments_fix_the_centring(orc):
    """A ramp along x, constant along y: away from the periodic wrap the
    x-high bands vanish (two wavelet moments), the y-high bands vanish
    everywhere, and the scaling coefficients are s[q][m] = 4 m (the first
    scaling moment vanishes about k = 0, so the ramp is sampled at 2m)."""
    n = 32
    a = np.tile(np.arange(n, dtype=np.float64), (n, 1)).astype(np.complex128)
    c = orc.wavelet_fwd(a, 1, "coif1")
    h = n // 2
    inner = slice(1, h - 2)   # level-1 outputs whose taps 2m-2 .. 2m+3 do not wrap
    assert np.max(np.abs(c[:h, h:][:, inner])) <= 1e-12   # LH: high along x
    assert np.max(np.abs(c[h:, :])) <= 1e-12              # HL, HH: high along y
    m = np.arange(h)[inner]
    assert np.max(np.abs(c[:h, :h][:, inner] - 4.0 * m)) <= 1e-12


def test_keep_all_aligned_points_equal_eq1(orc):
    """Every coefficient kept, points on the 2^L grid and the PSFs (plus the
    filters' spread over L levels) inside both the window and the hologram:
    the coiflet WASABI hologram is the Eq. (1) sum (FP64)."""
    L, W, N = 3, 160, 256
    zd = np.array([60e-6, 95e-6])
    olut = orc.build_lut(LAM, PITCH, zd, W, L, 1.0, dtype="f64", wavelet="coif1")
    rng = np.random.default_rng(4)
    n = 6
    x = (W // 2 + 8 * rng.integers(3, 12, n)).astype(np.int32) - 8 * 4 + 8
    y = (W // 2 + 8 * rng.integers(3, 12, n)).astype(np.int32) - 8 * 4 + 8
    d = rng.integers(0, 2, n).astype(np.uint32)
    a = rng.uniform(0.2, 1.0, n).astype(np.float32)
    pts = {"x": x, "y": y, "a": a, "d": d}
    u = orc.hologram(olut, pts, N)
    ref = orc.cgh_direct(LAM, PITCH, x, y, a, zd[d], 0, 0, N, N, aperture=True)
    assert np.max(np.abs(u - ref)) <= 1e-12
    # With Haar the same holds: the two transforms agree on this pin.
    hlut = orc.build_lut(LAM, PITCH, zd, W, L, 1.0, dtype="f64")
    assert np.max(np.abs(orc.hologram(hlut, pts, N) - ref)) <= 1e-12
