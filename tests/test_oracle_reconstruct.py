"""Pins of the oracle's numerical reconstruction (reading R13: the angular
spectrum method): closed-form propagation of plane waves (including the
evanescent cut), composition of distances, and refocusing of a point's
Eq. (1) field at d = -z (which fixes the sign convention)."""
import numpy as np
import pytest

LAM, PITCH = 633e-9, 1e-6


@pytest.mark.parametrize("mx,my,d", [(3, -5, 2e-3), (-60, 17, -0.7e-3), (0, 0, 1e-3)])
def test_plane_wave_propagates_by_its_closed_form(orc, mx, my, d):
    h, w = 96, 128
    x = np.arange(w)[None, :] * PITCH
    y = np.arange(h)[:, None] * PITCH
    fx, fy = mx / (w * PITCH), my / (h * PITCH)
    u0 = np.exp(2j * np.pi * (fx * x + fy * y))
    kz = np.sqrt(1 / LAM ** 2 - fx ** 2 - fy ** 2)
    want = u0 * np.exp(2j * np.pi * d * kz)
    assert np.max(np.abs(orc.reconstruct(u0, LAM, PITCH, d) - want)) <= 1e-9


def test_evanescent_frequencies_are_dropped(orc):
    pitch = 0.2e-6  # grid frequencies up to 2.5 / um > 1 / lambda
    h, w = 32, 64
    x = np.arange(w)[None, :] * pitch
    fx = 25 / (w * pitch)  # 1.95 / um > 1 / lambda = 1.58 / um
    u0 = np.exp(2j * np.pi * fx * x) * np.ones((h, 1))
    assert np.max(np.abs(orc.reconstruct(u0, LAM, pitch, 1e-6))) <= 1e-12
    fx2 = 12 / (w * pitch)  # 0.94 / um: propagates, modulus kept
    u2 = np.exp(2j * np.pi * fx2 * x) * np.ones((h, 1))
    assert np.allclose(np.abs(orc.reconstruct(u2, LAM, pitch, 1e-6)), 1.0, atol=1e-12)


def test_distances_compose(orc):
    rng = np.random.default_rng(3)
    u0 = rng.normal(size=(64, 80)) + 1j * rng.normal(size=(64, 80))
    a = orc.reconstruct(orc.reconstruct(u0, LAM, PITCH, 0.3e-3), LAM, PITCH, -1.1e-3)
    b = orc.reconstruct(u0, LAM, PITCH, -0.8e-3)
    assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(u0))


@pytest.mark.parametrize("z", [0.4e-3, -0.4e-3])
def test_a_point_refocuses_at_minus_z(orc, z):
    n = 256
    px, py = 131, 120
    u0 = orc.cgh_direct(LAM, PITCH, [px], [py], [1.0], [z], 0, 0, n, n, aperture=True)
    good = np.abs(orc.reconstruct(u0, LAM, PITCH, -z)) ** 2
    bad = np.abs(orc.reconstruct(u0, LAM, PITCH, z)) ** 2
    assert np.unravel_index(np.argmax(good), good.shape) == (py, px)
    assert good[py, px] > 20 * bad.max()
    # The focused spot holds most of the energy within a few pixels.
    assert good[py - 2:py + 3, px - 2:px + 3].sum() > 0.5 * good.sum()
