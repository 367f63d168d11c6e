"""Pins of the oracle's reference wave and reference binarisation (reading
R12, Sec. 2: a spherical reference wave from (x_r, y_r, z_r); the binary
hologram is the sign of the interference term).

The reference wave is checked against the oracle's Eq. (1) with a single
unit point at the source (an independent code path, pinned by brute force
elsewhere), the bits against the interference intensity |u + R|^2 written
with complex arithmetic, and the sign convention and fractional source
positions against exact symmetries."""
import numpy as np
import pytest

LAM, PITCH = 633e-9, 1e-6


@pytest.mark.parametrize("zr", [0.4, -0.4, 2e-3, -7e-4])
def test_reference_wave_is_the_field_of_a_unit_point_source(orc, zr):
    # The source at an integer pixel, here outside the region (as in the
    # paper's setup: 30 mm off axis, 400 mm behind the plane) and inside it.
    for xr, yr, ox, oy in [(3, -900, 0, 0), (20, 9, 0, 0), (-40, 70, 16, 48)]:
        R = orc.reference_wave(LAM, PITCH, float(xr), float(yr), zr, 48, 24, ox, oy)
        eq1 = orc.cgh_direct(LAM, PITCH, [xr], [yr], [1.0], [zr], ox, oy, 48, 24, aperture=False)
        assert np.max(np.abs(R - eq1)) <= 1e-8, (xr, yr, zr)


def test_bits_are_the_sign_of_the_interference_term(orc):
    rng = np.random.default_rng(5)
    h, w = 40, 56
    u = rng.normal(size=(h, w)) + 1j * rng.normal(size=(h, w))
    # R from Eq. (1) for a source at an integer pixel; from the oracle's own
    # reference wave (pinned above and below) for a fractional one.
    cases = [(-0.4, 10.0, -30000.0, orc.cgh_direct(LAM, PITCH, [10], [-30000], [1.0], [-0.4], 0, 0, w, h,
                                                    aperture=False)),
             (0.01, 27.25, 11.5, orc.reference_wave(LAM, PITCH, 27.25, 11.5, 0.01, w, h))]
    for zr, xr, yr, R in cases:
        inter = np.abs(u + R) ** 2 - np.abs(u) ** 2 - np.abs(R) ** 2  # = 2 Re(u conj R)
        bits, val = orc.binarize_ref(u, LAM, PITCH, xr, yr, zr)
        assert np.allclose(2.0 * val, inter, atol=1e-9)
        mine = np.unpackbits(bits, bitorder="little")[: h * w].reshape(h, w).astype(bool)
        sure = np.abs(inter) > 1e-9
        assert np.array_equal(mine[sure], (inter > 0)[sure])
        assert sure.mean() > 0.99


def test_source_behind_the_plane_is_the_conjugate(orc):
    """R_{-z} = conj(R_z), so binarising u against the source at -z gives the
    bits of conj(u) against +z, value for value."""
    rng = np.random.default_rng(9)
    u = rng.normal(size=(24, 32)) + 1j * rng.normal(size=(24, 32))
    b1, v1 = orc.binarize_ref(u, LAM, PITCH, 3.5, -120.0, -0.25, 8, 16)
    b2, v2 = orc.binarize_ref(np.conj(u), LAM, PITCH, 3.5, -120.0, 0.25, 8, 16)
    assert np.array_equal(v1, v2) and np.array_equal(b1, b2)
    R1 = orc.reference_wave(LAM, PITCH, 3.5, -120.0, -0.25, 32, 24, 8, 16)
    R2 = orc.reference_wave(LAM, PITCH, 3.5, -120.0, 0.25, 32, 24, 8, 16)
    assert np.array_equal(R1, np.conj(R2))


def test_fractional_source_position_is_symmetric(orc):
    """A source at x_r = 20.5 sits between pixel columns 20 and 21: column
    20 - k mirrors column 21 + k (likewise for y), to rounding."""
    R = orc.reference_wave(LAM, PITCH, 20.5, 11.5, 3e-3, 42, 24)
    assert np.max(np.abs(R[:, 20::-1] - R[:, 21:42])) <= 1e-9
    assert np.max(np.abs(R[11::-1, :] - R[12:24, :])) <= 1e-9
    # Off by a whole pixel the symmetry breaks (the position is not rounded).
    assert np.max(np.abs(R[:, 19::-1] - R[:, 21:41])) > 1e-3
