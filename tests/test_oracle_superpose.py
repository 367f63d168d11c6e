"""Pins for the oracle's superposition (Eq. (2), reading R6), inverse (Sec. 1,
step 3), sub-hologram driver (Sec. 1, large-scale steps 2-4) and Eq. (1)."""
import numpy as np
import pytest

from workloads import aligned, uniform_cloud

LAM, PITCH = 633e-9, 1e-6
ZMIN, ZMAX, D = 20e-6, 90e-6, 4       # R <= 30 px: fits a 64-px window
W, L, NH = 64, 3, 128


def _setup(orc, N, seed=11, step=8, dtype="f64", gamma=1.0, Nh=NH):
    pts = aligned(uniform_cloud(seed, N, Nh, ZMIN, ZMAX), step) if step else \
        uniform_cloud(seed, N, Nh, ZMIN, ZMAX)
    zd = orc.depth_grid(ZMIN, ZMAX, D)
    pts["d"], bad = orc.quantize(pts["z"], ZMIN, ZMAX, D)
    assert bad == 0
    lut = orc.build_lut(LAM, PITCH, zd, W, L, gamma, dtype=dtype)
    return pts, zd, lut


def _eq1(orc, pts, zd, Nh, aperture=True):
    return orc.cgh_direct(LAM, PITCH, pts["x"], pts["y"], pts["a"], zd[pts["d"]],
                          0, 0, Nh, Nh, aperture)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def test_keep_all_reproduces_direct_sum_fp64(orc):
    """gamma >= 1 with points on the 2^L grid: WASABI equals the apertured
    Eq. (1) superposition (spec acceptance pin), edges included."""
    pts, zd, lut = _setup(orc, 40)
    pts["x"][:4] = [0, NH - 8, 8, NH - 16]
    pts["y"][:4] = [NH - 8, 0, 64, 120]
    u = orc.hologram(lut, pts, NH)
    ref = _eq1(orc, pts, zd, NH)
    assert np.max(np.abs(u - ref)) < 1e-12 * np.max(np.abs(ref))


def test_keep_all_reproduces_direct_sum_fp32(orc):
    pts, zd, lut = _setup(orc, 40, dtype="f32")
    u = orc.hologram(lut, pts, NH)
    assert u.dtype == np.complex64
    assert _rel(u.astype(np.complex128), _eq1(orc, pts, zd, NH)) < 1e-6


def test_single_point_closed_form(orc):
    pts, zd, lut = _setup(orc, 1)
    pts["x"][:] = 64
    pts["y"][:] = 56
    u = orc.hologram(lut, pts, NH)
    a, z = float(pts["a"][0]), zd[pts["d"][0]]
    assert abs(u[56, 64] - a * np.exp(2j * np.pi * ((z / LAM) % 1.0))) < 1e-12
    R = orc.support_radius(LAM, PITCH, z)
    yy, xx = np.mgrid[0:NH, 0:NH]
    inside = (xx - 64) ** 2 + (yy - 56) ** 2 < R * R
    assert np.allclose(np.abs(u[inside]), a, atol=1e-12)
    assert np.max(np.abs(u[~inside])) < 1e-12


@pytest.mark.parametrize("gamma", [0.05, 0.2, 0.6])
def test_parseval_error_law(orc, gamma):
    """One aligned point whose window lies inside the hologram: the squared
    error against Eq. (1) equals a^2 times the energy of the dropped
    coefficients, i.e. a^2 (pixels in the disk - sum over kept |c|^2)."""
    pts, zd, lut = _setup(orc, 1, gamma=gamma)
    pts["x"][:] = 64
    pts["y"][:] = 64
    d = int(pts["d"][0])
    a = float(pts["a"][0])
    u = orc.hologram(lut, pts, NH)
    ref = _eq1(orc, pts, zd, NH)
    R = orc.support_radius(LAM, PITCH, zd[d])
    v, uu = np.mgrid[0:W, 0:W]
    ndisk = np.sum((uu - W // 2) ** 2 + (v - W // 2) ** 2 < R * R)
    _, val = lut.depth(d)
    dropped = ndisk - np.sum(np.abs(val) ** 2)
    err2 = np.sum(np.abs(u - ref) ** 2)
    assert dropped > 0
    assert abs(err2 - a * a * dropped) < 1e-9 * max(1.0, a * a * ndisk)


def test_error_monotone_in_gamma(orc):
    errs = []
    for gamma in [0.02, 0.05, 0.1, 0.3, 1.0]:
        pts, zd, lut = _setup(orc, 1, gamma=gamma)
        pts["x"][:] = 64
        pts["y"][:] = 64
        errs.append(_rel(orc.hologram(lut, pts, NH), _eq1(orc, pts, zd, NH)))
    assert all(b <= a + 1e-15 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-12


def test_linearity(orc):
    pts, zd, lut = _setup(orc, 30, step=0, gamma=0.3)
    A = {k: v[:13] for k, v in pts.items()}
    B = {k: v[13:] for k, v in pts.items()}
    u = orc.hologram(lut, pts, NH)
    assert np.max(np.abs(u - (orc.hologram(lut, A, NH) + orc.hologram(lut, B, NH)))) < 1e-12


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_subholograms_tile_the_full_hologram(orc, dtype):
    """Sec. 1, large-scale steps 2-4: every sub-hologram equals the crop of
    the whole-buffer result, bit for bit."""
    Nw, Ns = 256, 64
    pts, zd, lut = _setup(orc, 60, step=0, dtype=dtype, gamma=0.2, Nh=Nw)
    full = orc.hologram(lut, pts, Nw)
    for t in range(Nw // Ns):
        for s in range(Nw // Ns):
            sub = orc.subhologram(lut, pts, Ns, s, t)
            assert np.array_equal(sub, full[t * Ns:(t + 1) * Ns, s * Ns:(s + 1) * Ns])


def test_rules_agree_on_aligned_points(orc):
    pts, zd, lut = _setup(orc, 20, gamma=0.3, dtype="f32")
    assert np.array_equal(orc.hologram(lut, pts, NH, rule=0), orc.hologram(lut, pts, NH, rule=1))


def test_floor_rule_ignores_sub_tile_offsets_at_level_L(orc):
    """With L = 1 the floor rule maps x = 2m and x = 2m + 1 to the same
    coefficient positions, so the two holograms are identical."""
    zd = orc.depth_grid(ZMIN, ZMAX, D)
    lut = orc.build_lut(LAM, PITCH, zd, W, 1, 0.3, dtype="f32")
    p0 = {"x": np.array([40], np.int32), "y": np.array([50], np.int32),
          "a": np.array([0.7], np.float32), "d": np.array([2], np.uint32)}
    p1 = dict(p0, x=np.array([41], np.int32), y=np.array([51], np.int32))
    assert np.array_equal(orc.hologram(lut, p0, NH), orc.hologram(lut, p1, NH))
    assert not np.array_equal(orc.hologram(lut, p0, NH, rule=1),
                              orc.hologram(lut, p1, NH, rule=1))


def test_unaligned_error_is_reported(orc):
    pts, zd, lut = _setup(orc, 40, step=0, gamma=1.0)
    for rule in (0, 1):
        e = _rel(orc.hologram(lut, pts, NH, rule=rule), _eq1(orc, pts, zd, NH))
        assert 0 < e < 2.0


def test_bad_depth_rejected(orc):
    pts, zd, lut = _setup(orc, 3)
    pts["d"][1] = D
    with pytest.raises(ValueError):
        orc.hologram(lut, pts, NH)


def test_window_too_small_rejected(orc):
    zd = orc.depth_grid(ZMIN, 200e-6, D)
    with pytest.raises(ValueError):
        orc.build_lut(LAM, PITCH, zd, W, L, 0.1)


# ------------------------------------------------------------- Eq. (1) pins

def test_direct_single_point_closed_form(orc):
    x, y, a, z = [37], [21], [0.5], [0.7e-3]
    w = h = 96
    u = orc.cgh_direct(LAM, PITCH, x, y, a, z, 0, 0, w, h, True)
    R = orc.support_radius(LAM, PITCH, z[0])
    yy, xx = np.mgrid[0:h, 0:w]
    inside = (xx - 37) ** 2 + (yy - 21) ** 2 < R * R
    assert np.allclose(np.abs(u[inside]), 0.5, atol=1e-14)
    assert not np.any(u[~inside])
    assert abs(u[21, 37] - 0.5 * np.exp(2j * np.pi * ((z[0] / LAM) % 1))) < 1e-13
    ub = orc.cgh_direct(LAM, PITCH, x, y, a, z, 0, 0, w, h, False)
    assert np.allclose(np.abs(ub), 0.5, atol=1e-14)


def test_direct_eightfold_symmetry(orc):
    c = 40
    u = orc.cgh_direct(LAM, PITCH, [c], [c], [1.0], [0.3e-3], 0, 0, 81, 81, True)
    core = u[:81, :81]
    assert np.array_equal(core, core[::-1, :])
    assert np.array_equal(core, core[:, ::-1])
    assert np.array_equal(core, core.T)


def test_direct_region_and_additivity(orc):
    rng = np.random.default_rng(3)
    x = rng.integers(0, 64, 9)
    y = rng.integers(0, 64, 9)
    a = rng.uniform(0.1, 1, 9)
    z = rng.uniform(0.1e-3, 0.3e-3, 9)
    full = orc.cgh_direct(LAM, PITCH, x, y, a, z, 0, 0, 64, 64)
    part = orc.cgh_direct(LAM, PITCH, x, y, a, z, 16, 8, 20, 30)
    assert np.array_equal(part, full[8:38, 16:36])
    s = orc.cgh_direct(LAM, PITCH, x[:4], y[:4], a[:4], z[:4], 0, 0, 64, 64) + \
        orc.cgh_direct(LAM, PITCH, x[4:], y[4:], a[4:], z[4:], 0, 0, 64, 64)
    assert np.max(np.abs(s - full)) < 1e-12


def test_binarize_bit_order(orc):
    u = np.array([[1, -1, 0, 2, -3, 4, 5, -6, 7, 0, 0, 0, 0, 0, 0, 1]], np.complex64)
    bits = orc.binarize(u)
    # x = 0, 3, 5, 6 set in byte 0; x = 8 and 15 in byte 1.
    assert list(bits) == [0b01101001, 0b10000001]


# ---- R11: image-type holograms (points on both sides of the plane) --------

def test_lut_behind_the_plane_is_the_conjugate(orc):
    """A depth -z keeps the same coefficients as +z with conjugate values
    (the PSF of a point behind the plane converges on it), FP32 and FP64."""
    zd = np.array([-70e-6, -33e-6, 33e-6, 70e-6])
    for dtype in ("f32", "f64"):
        lut = orc.build_lut(LAM, PITCH, zd, W, L, 0.3, dtype=dtype)
        for dn, dp in ((0, 3), (1, 2)):
            i_n, v_n = lut.depth(dn)
            i_p, v_p = lut.depth(dp)
            assert np.array_equal(i_n, i_p)
            assert np.array_equal(v_n, np.conj(v_p))


def test_hologram_behind_the_plane_is_the_conjugate(orc):
    pts = uniform_cloud(3, 30, NH, ZMIN, ZMAX)
    zp = orc.depth_grid(ZMIN, ZMAX, D)
    zd = np.concatenate([-zp[::-1], zp])  # depth D - 1 - d is exactly -(depth D + d)
    d, _ = orc.quantize(pts["z"], ZMIN, ZMAX, D)
    d_pos, d_neg = (D + d).astype(np.uint32), (D - 1 - d).astype(np.uint32)
    assert np.array_equal(zd[d_neg], -zd[d_pos])
    for dtype in ("f32", "f64"):
        lut = orc.build_lut(LAM, PITCH, zd, W, L, 0.4, dtype=dtype)
        up = orc.hologram(lut, dict(pts, d=d_pos), NH)
        un = orc.hologram(lut, dict(pts, d=d_neg), NH)
        assert np.array_equal(un, np.conj(up))
    ep = orc.cgh_direct(LAM, PITCH, pts["x"], pts["y"], pts["a"], zd[d_pos], 0, 0, NH, NH, True)
    en = orc.cgh_direct(LAM, PITCH, pts["x"], pts["y"], pts["a"], zd[d_neg], 0, 0, NH, NH, True)
    assert np.array_equal(en, np.conj(ep))


def test_point_on_the_plane_is_a_delta(orc):
    """z = 0: the support is the centre pixel, every coefficient of the delta
    is kept, and on the 2^L grid the hologram is a_j at (x_j, y_j) exactly
    (Eq. (1) gives the same)."""
    g = np.random.default_rng(4)
    n = 20
    pts = {"x": (g.integers(0, NH // 8, n) * 8).astype(np.int32), "y": (g.integers(0, NH // 8, n) * 8).astype(np.int32),
           "a": (1.0 - g.random(n)).astype(np.float32), "d": np.zeros(n, np.uint32)}
    lut = orc.build_lut(LAM, PITCH, np.array([0.0]), W, L, 0.01, dtype="f64")
    assert lut.nr[0] == 3 * L + 1
    u = orc.hologram(lut, pts, NH)
    want = np.zeros((NH, NH), np.complex128)
    np.add.at(want, (pts["y"], pts["x"]), pts["a"].astype(np.float64))
    assert np.max(np.abs(u - want)) < 1e-12
    e = orc.cgh_direct(LAM, PITCH, pts["x"], pts["y"], pts["a"], np.zeros(n), 0, 0, NH, NH, True)
    assert np.max(np.abs(e - want)) < 1e-12


def test_keep_all_exact_on_both_sides_of_the_plane(orc):
    pts = aligned(uniform_cloud(9, 30, NH, -ZMAX, ZMAX), 8)
    zd = orc.depth_grid(-ZMAX, ZMAX, 2 * D)
    pts["d"], bad = orc.quantize(pts["z"], -ZMAX, ZMAX, 2 * D)
    assert bad == 0 and np.any(zd[pts["d"]] < 0) and np.any(zd[pts["d"]] > 0)
    lut = orc.build_lut(LAM, PITCH, zd, W, L, 1.0, dtype="f64")
    assert _rel(orc.hologram(lut, pts, NH), _eq1(orc, pts, zd, NH)) < 1e-12
