"""Pins for the oracle's phase arithmetic (reading R8) and PSF (Sec. 1, step 1)."""
import numpy as np


def test_sincos2pi_matches_libm(orc):
    # Dense sweep plus every quadrant boundary and its neighbours.
    g = np.linspace(0.0, 1.0, 200_001, dtype=np.float64).astype(np.float32)
    edges = np.array([0.0, 0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 1.0], np.float32)
    g = np.concatenate([g, edges, np.nextafter(edges, np.float32(2)),
                        np.nextafter(edges, np.float32(-1))])
    g = g[(g >= 0) & (g <= 1)]
    c, s = orc.sincos2pi_f32(g)
    ang = 2.0 * np.pi * g.astype(np.float64)
    assert np.max(np.abs(c - np.cos(ang))) < 4e-7
    assert np.max(np.abs(s - np.sin(ang))) < 4e-7


def test_sincos2pi_exact_points(orc):
    g = np.array([0.0, 0.25, 0.5, 0.75, 1.0], np.float32)
    c, s = orc.sincos2pi_f32(g)
    assert list(c) == [1.0, 0.0, -1.0, 0.0, 1.0]
    assert list(s) == [0.0, 1.0, 0.0, -1.0, 0.0]


def test_psf_f32_close_to_definition(orc):
    lam, p, z, W = 633e-9, 1e-6, 0.37e-3, 512
    a = orc.psf_f32(lam, p, z, W)
    b = orc.psf_f64(lam, p, z, W)
    assert np.max(np.abs(a.astype(np.complex128) - b)) < 1e-6
    # Support is exactly the open disk of reading R1 and |u| = 1 inside it.
    R = orc.support_radius(lam, p, z)
    v, u = np.mgrid[0:W, 0:W]
    n = (u - W // 2) ** 2 + (v - W // 2) ** 2
    inside = n < R * R
    assert np.all(b[~inside] == 0)
    assert np.allclose(np.abs(b[inside]), 1.0, atol=1e-14)


def test_psf_centre_phase_is_z_over_lambda(orc):
    # At the centre pixel r = z, so u = exp(i 2 pi z / lambda) (Eq. (1)).
    lam, p, z, W = 532e-9, 1e-6, 0.61e-3, 256
    b = orc.psf_f64(lam, p, z, W)
    frac = (z / lam) % 1.0
    assert abs(b[W // 2, W // 2] - np.exp(2j * np.pi * frac)) < 1e-12


def test_psf_radial_symmetry(orc):
    lam, p, z, W = 633e-9, 1e-6, 0.2e-3, 256
    b = orc.psf_f32(lam, p, z, W)
    c = W // 2
    core = b[1:, 1:]            # du, dv in [-W/2+1, W/2-1]: symmetric square
    assert np.array_equal(core, core[::-1, :])
    assert np.array_equal(core, core[:, ::-1])
    assert np.array_equal(core, core.T)
    assert b[c, c] != 0
