"""Pins for readings R1-R3 (Sec. 1, step 1; Sec. 2)."""
import numpy as np
import pytest


@pytest.mark.parametrize("lam", [532e-9, 633e-9])
@pytest.mark.parametrize("z", [0.1e-3, 0.55e-3, 1.0e-3])
def test_radius_is_nyquist_limit_of_chirp(orc, lam, z):
    """R1 pin from the physics of Eq. (1): the local spatial frequency of
    exp(i 2 pi r / lambda) at the support edge equals the sampling limit
    1 / (2 p).  Measured by a central difference of r(rho) / lambda."""
    p = 1e-6
    R = orc.support_radius(lam, p, z)
    rho = R * p
    h = 1e-9
    r = lambda q: np.sqrt(q * q + z * z)
    freq = (r(rho + h) - r(rho - h)) / (2 * h * lam)
    assert abs(freq - 1.0 / (2 * p)) / (1.0 / (2 * p)) < 1e-6


def test_radius_per_mm_values(orc):
    # 633 nm: 333.65 px/mm; 532 nm: 275.94 px/mm at 1 um pitch.
    assert abs(orc.support_radius(633e-9, 1e-6, 1e-3) - 333.652) < 1e-3
    assert abs(orc.support_radius(532e-9, 1e-6, 1e-3) - 275.941) < 1e-3


def test_keep_target_is_fraction_of_disk_area(orc):
    """R3 pin: gamma * pi R^2 is gamma times the pixel count of the disk,
    up to the lattice-count boundary term (Gauss circle problem)."""
    for R in [34.5, 101.9, 242.3, 332.48]:
        r = int(np.ceil(R))
        v, u = np.mgrid[-r:r + 1, -r:r + 1]
        count = int(np.sum(u * u + v * v < R * R))
        for gamma in [0.01, 0.02, 0.05]:
            t = orc.keep_target(gamma, R)
            assert abs(t - gamma * count) <= gamma * 4 * R + 2


def test_keep_target_known_values(orc):
    zd = orc.depth_grid(0.1e-3, 1.0e-3, 128)
    R = orc.support_radius(633e-9, 1e-6, zd[127])
    assert abs(R - 332.48) < 0.01
    assert orc.keep_target(0.01, R) == 3473
    zd = orc.depth_grid(0.2e-3, 0.9e-3, 16)
    nr = [orc.keep_target(0.05, orc.support_radius(532e-9, 1e-6, z)) for z in zd]
    assert nr[0] == 589 and nr[-1] == 9223


def test_depth_grid_paper_spacing(orc):
    """Sec. 2: 30 mm of depth over N_z = 29 planes gives dz = 30/29 mm."""
    zd = orc.depth_grid(-15e-3, 15e-3, 29)
    assert np.allclose(np.diff(zd), 30e-3 / 29, rtol=0, atol=1e-15)
    assert abs(np.diff(zd)[0] - 1.03e-3) < 0.01e-3


def test_quantize_puts_points_in_their_bin(orc):
    rng = np.random.default_rng(0)
    zmin, zmax, D = 0.3e-3, 1.0e-3, 64
    z = np.concatenate([rng.uniform(zmin, zmax, 10000), [zmin, zmax]])
    d, bad = orc.quantize(z, zmin, zmax, D)
    assert bad == 0
    zd = orc.depth_grid(zmin, zmax, D)
    dz = (zmax - zmin) / D
    assert np.all(np.abs(z - zd[d]) <= dz / 2 * (1 + 1e-9))
    assert d.min() == 0 and d.max() == D - 1


def test_quantize_flags_out_of_range(orc):
    d, bad = orc.quantize(np.array([0.1e-3, 0.5e-3, 2e-3, np.nan]), 0.3e-3, 1.0e-3, 8)
    assert bad == 3
    assert list(d) == [8, 2, 8, 8]
