"""GPU point preparation, superposition (Eq. (2)) and hologram against the
oracle.  Fields: rel-L2 <= 1e-5 (FP32, norms in FP64); depth indices and
bits: exact (bits may differ only where |Re u| is within rounding of 0)."""
import os

import numpy as np
import pytest
import torch

from tests._bounds import FieldBound, check_bits, check_field
from tests._helpers import rel_l2, tile_major_to_mallat
from workloads import CONFIGS, aligned, uniform_cloud

pytestmark = pytest.mark.gpu
TOL = 1e-5
NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


def _dev_points(w, pts, zmin, zmax, D):
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in pts.items() if k in "xyza"}
    return w.quantize_points(t["x"], t["y"], t["z"], t["a"], zmin, zmax, D)


@pytest.fixture(scope="module")
def c1(w, orc):
    c = CONFIGS["C1"]
    pts = c.points()
    zd = orc.depth_grid(c.zmin, c.zmax, c.D)
    pts["d"], bad = orc.quantize(pts["z"], c.zmin, c.zmax, c.D)
    assert bad == 0
    olut = orc.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma, threads=NPROC)
    lut = w.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma)
    return c, pts, zd, olut, lut


def test_quantize_bit_exact(w, orc, c1):
    c, pts, _, _, _ = c1
    p = _dev_points(w, pts, c.zmin, c.zmax, c.D).cpu().numpy()
    assert np.array_equal(p[:, 3].view(np.uint32), pts["d"])
    assert np.array_equal(p[:, 0], pts["x"]) and np.array_equal(p[:, 2].view(np.float32), pts["a"])
    w.sync_status()


def test_quantize_flags_out_of_range(w, orc):
    z = np.array([0.5e-3, 2e-3, 0.1e-3])
    pts = {"x": np.zeros(3, np.int32), "y": np.zeros(3, np.int32), "z": z, "a": np.ones(3, np.float32)}
    p = _dev_points(w, pts, 0.3e-3, 1.0e-3, 8).cpu().numpy()
    d_ref, _ = orc.quantize(z, 0.3e-3, 1.0e-3, 8)
    assert np.array_equal(p[:, 3].view(np.uint32), d_ref)
    with pytest.raises(w.WasabiError, match="RANGE"):
        w.sync_status()
    w.sync_status()  # cleared


@pytest.mark.parametrize("rule", [0, 1])
def test_c1_wavelet_buffer_and_field(w, orc, c1, rule):
    c, pts, zd, olut, lut = c1
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    wbuf = w.superpose(lut, p, c.Nh, c.Nh, rule=rule)
    u = w.inverse_haar(wbuf, c.Nh, c.Nh, c.L).cpu().numpy()
    w.sync_status()
    psi = orc.superpose(olut, pts, c.Nh, rule=rule)
    got = tile_major_to_mallat(wbuf.cpu().numpy(), c.Nh, c.Nh, c.L)
    assert rel_l2(got, psi) <= TOL
    fb = FieldBound(orc, olut, pts, c.Nh, rule=rule)
    check_field(got, psi, fb.coeffs(c.Nh, 0, 0))
    ref = orc.haar_inv(psi, c.L)
    assert rel_l2(u, ref) <= TOL
    check_field(u, ref, fb.window(c.Nh, 0, 0))


def test_c1_wasabi_vs_eq1_reported(w, orc, c1):
    """The approximation error of WASABI against Eq. (1) (reported, not
    bounded: the paper prints no error figure)."""
    c, pts, zd, olut, lut = c1
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    u = w.hologram(lut, p, c.Nh, c.Nh).cpu().numpy()
    ref = orc.cgh_direct(c.lam, c.pitch, pts["x"], pts["y"], pts["a"], zd[pts["d"]], 0, 0,
                         c.Nh, c.Nh, True, threads=NPROC)
    e = rel_l2(u, ref)
    print(f"C1 WASABI vs Eq.(1) rel-L2 = {e:.4f}")
    assert 0 < e < 2


def test_keep_all_equals_direct_sum(w, orc):
    """keep_ratio >= 1 with points on the 2^L grid reproduces the apertured
    Eq. (1) sum (spec pin), here on the GPU."""
    lam, pitch, zmin, zmax, D, W, L, Nh = 633e-9, 1e-6, 20e-6, 90e-6, 4, 64, 3, 256
    pts = aligned(uniform_cloud(4, 60, Nh, zmin, zmax), 8)
    zd = orc.depth_grid(zmin, zmax, D)
    pts["d"], _ = orc.quantize(pts["z"], zmin, zmax, D)
    lut = w.build_lut(lam, pitch, zd, W, L, 1.0)
    u = w.hologram(lut, w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"]), Nh, Nh).cpu().numpy()
    ref = orc.cgh_direct(lam, pitch, pts["x"], pts["y"], pts["a"], zd[pts["d"]], 0, 0, Nh, Nh, True)
    assert rel_l2(u, ref) <= 1e-6


def _oracle_case(orc, seed, N, Nh, L, W, gamma, xr=None):
    lam, pitch, zmin, zmax, D = 633e-9, 1e-6, 20e-6, 150e-6, 6
    pts = uniform_cloud(seed, N, Nh, zmin, zmax)
    if xr is not None:
        r = np.random.default_rng(seed)
        pts["x"] = r.integers(xr[0], xr[1], N).astype(np.int32)
        pts["y"] = r.integers(xr[0], xr[1], N).astype(np.int32)
    zd = orc.depth_grid(zmin, zmax, D)
    pts["d"], _ = orc.quantize(pts["z"], zmin, zmax, D)
    olut = orc.build_lut(lam, pitch, zd, W, L, gamma)
    return lam, pitch, zd, pts, olut


@pytest.mark.parametrize("L,W,Nh,T,threads", [
    (2, 128, 200, 64, 256), (3, 128, 1000, 128, 1024), (4, 128, 528, 64, 512),
    (5, 128, 512, 128, 1024), (4, 256, 256, 128, 1024), (1, 128, 130, 32, 128)])
def test_sizes_levels_and_tiles(w, orc, monkeypatch, L, W, Nh, T, threads):
    """Ragged hologram sides (not multiples of the super-tile), every level
    count, super-tile sizes and block sizes, points inside and far outside."""
    monkeypatch.setenv("WASABI_SUPERPOSE_T", str(T))
    monkeypatch.setenv("WASABI_SUPERPOSE_THREADS", str(threads))
    lam, pitch, zd, pts, olut = _oracle_case(orc, L + Nh, 150, Nh, L, W, 0.2, xr=(-200, Nh + 200))
    lut = w.build_lut(lam, pitch, zd, W, L, 0.2)
    for rule in (0, 1):
        wbuf = w.superpose(lut, w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"]), Nh, Nh, rule=rule)
        w.sync_status()
        psi = orc.superpose(olut, pts, Nh, rule=rule)
        assert rel_l2(tile_major_to_mallat(wbuf.cpu().numpy(), Nh, Nh, L), psi) <= TOL


def test_empty_point_set_gives_zero_buffer(w, orc):
    lam, pitch, zd, pts, olut = _oracle_case(orc, 1, 5, 256, 4, 128, 0.2)
    lut = w.build_lut(lam, pitch, zd, 128, 4, 0.2)
    wbuf = torch.full((256 * 256,), 7.0 + 1j, dtype=torch.complex64, device="cuda")
    w.superpose(lut, torch.empty((0, 4), dtype=torch.int32, device="cuda"), 256, 256, wbuf=wbuf)
    w.sync_status()
    assert not wbuf.abs().max().item()


def test_rectangular_is_crop_of_square(w, orc):
    lam, pitch, zd, pts, olut = _oracle_case(orc, 5, 200, 512, 4, 128, 0.3)
    lut = w.build_lut(lam, pitch, zd, 128, 4, 0.3)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    full = w.hologram(lut, p, 512, 512).cpu().numpy()
    rect = w.hologram(lut, p, 320, 176).cpu().numpy()
    ref = orc.hologram(olut, pts, 512)
    assert rel_l2(full, ref) <= TOL
    assert rel_l2(rect, full[:176, :320]) <= TOL


def test_bad_depth_reports_range_and_is_skipped(w, orc):
    lam, pitch, zd, pts, olut = _oracle_case(orc, 8, 40, 256, 4, 128, 0.2)
    lut = w.build_lut(lam, pitch, zd, 128, 4, 0.2)
    d = pts["d"].copy()
    d[3] = 99
    wbuf = w.superpose(lut, w.pack_points(pts["x"], pts["y"], pts["a"], d), 256, 256)
    with pytest.raises(w.WasabiError, match="RANGE"):
        w.sync_status()
    keep = np.arange(40) != 3
    sub = {k: v[keep] for k, v in pts.items()}
    psi = orc.superpose(olut, sub, 256)
    assert rel_l2(tile_major_to_mallat(wbuf.cpu().numpy(), 256, 256, 4), psi) <= TOL


def test_reduced_precision_forms(w, orc):
    """C4 forms on a small case: error against the FP64 oracle is reported
    per dtype; FP16 must stay close to FP32."""
    lam, pitch, zd, pts, _ = _oracle_case(orc, 12, 300, 512, 4, 256, 0.05)
    o64 = orc.build_lut(lam, pitch, zd, 256, 4, 0.05, dtype="f64", select_fp32=True)
    ref = orc.hologram(o64, pts, 512)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    errs = {}
    for dt in ("f32", "f16s", "bf16s"):
        lut = w.build_lut(lam, pitch, zd, 256, 4, 0.05, dtype=dt)
        errs[dt] = rel_l2(w.hologram(lut, p, 512, 512).cpu().numpy(), ref)
    print("rel-L2 vs FP64 oracle:", errs)
    assert errs["f32"] <= 1e-5
    assert errs["f16s"] <= 1e-3
    assert errs["bf16s"] <= 1e-2


def test_fixed_point_is_deterministic_and_matches_float(w, orc, monkeypatch, c1):
    """The exact fixed-point accumulator gives bit-identical buffers run to
    run, and agrees with the FP32-atomic accumulator and the oracle."""
    c, pts, zd, olut, lut = c1
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    a1 = w.superpose(lut, p, c.Nh, c.Nh).cpu().numpy()
    a2 = w.superpose(lut, p, c.Nh, c.Nh).cpu().numpy()
    assert np.array_equal(a1, a2)
    monkeypatch.setenv("WASABI_ACC_FLOAT", "1")
    f1 = w.superpose(lut, p, c.Nh, c.Nh).cpu().numpy()
    w.sync_status()
    psi = orc.superpose(olut, pts, c.Nh)
    assert rel_l2(tile_major_to_mallat(f1, c.Nh, c.Nh, c.L), psi) <= TOL
    assert rel_l2(a1, f1) <= TOL


@pytest.mark.parametrize("want,T,rcap", [("bits", 256, 0), ("both", 192, 0), ("bits", 256, 1024)])
def test_widest_tiles_many_candidate_batches(w, orc, monkeypatch, want, T, rcap):
    """The benchmark's launch configurations on a hologram small enough for
    the whole-field oracle: 1,024-thread CTAs on 256-pixel super-tiles with
    real-part accumulation (bits alone) and on 192-pixel super-tiles with
    complex accumulation, C3's optics and LUT shape (633 nm, W = 1024, L = 4,
    keep 1%, z in [0.1, 1.0] mm), and enough points within reach of every
    super-tile that its coefficient visits need several rounds of passes (a
    round holds at most the launch's pass capacity; rcap = 1,024 forces many
    rounds and candidate batches of 256).  Element-wise bounds on every
    pixel."""
    monkeypatch.setenv("WASABI_SUPERPOSE_T", str(T))
    monkeypatch.setenv("WASABI_SUPERPOSE_THREADS", "1024")
    if rcap:
        monkeypatch.setenv("WASABI_RANGE_CAP", str(rcap))
    lam, pitch, zmin, zmax, D, W, L, gamma, Nh, N = 633e-9, 1e-6, 0.1e-3, 1.0e-3, 16, 1024, 4, 0.01, 1024, 1800
    pts = uniform_cloud(77, N, Nh, zmin, zmax)
    r = np.random.default_rng(77)
    pts["x"] = r.integers(-300, Nh + 300, N).astype(np.int32)
    pts["y"] = r.integers(-300, Nh + 300, N).astype(np.int32)
    zd = orc.depth_grid(zmin, zmax, D)
    pts["d"], _ = orc.quantize(pts["z"], zmin, zmax, D)
    olut = orc.build_lut(lam, pitch, zd, W, L, gamma, threads=NPROC)
    lut = w.build_lut(lam, pitch, zd, W, L, gamma)
    for d in range(D):
        assert np.array_equal(lut.selection(d), olut.depth(d)[0]), d
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    ref = orc.hologram(olut, pts, Nh)
    bnd = FieldBound(orc, olut, pts, Nh).window(Nh, 0, 0)
    out = w.hologram(lut, p, Nh, Nh, want=want)
    w.sync_status()
    bits = out if want == "bits" else out[1]
    mine = np.unpackbits(bits.view(Nh, Nh // 8).cpu().numpy(), axis=1, bitorder="little").astype(bool)
    flips = check_bits(mine, ref, bnd)
    if want == "both":
        got = out[0].cpu().numpy()
        assert rel_l2(got, ref) <= TOL
        check_field(got, ref, bnd)
    print(f"{want} T={T}: {flips} bit flips of {Nh * Nh}")
    lut.close()


@pytest.mark.parametrize("want,T", [("both", 192), ("bits", 256)])
def test_pass_list_overflow_is_exact(w, monkeypatch, want, T):
    """Dense points: every candidate batch has more passes than the pass list
    holds (at its smallest capacity, 1,024 passes), so the passes that do not
    fit are numbered by the block-wide scan and visited in further lists.  The
    fixed-point sums are exact, so the result must equal, bit for bit, the
    same launch with the default capacity (whose batches overflow less)."""
    monkeypatch.setenv("WASABI_SUPERPOSE_T", str(T))
    monkeypatch.setenv("WASABI_SUPERPOSE_THREADS", "1024")
    lam, pitch, zmin, zmax, D, W, L, gamma, Nh, N = 633e-9, 1e-6, 0.1e-3, 1.0e-3, 16, 1024, 4, 0.01, 768, 2500
    r = np.random.default_rng(5)
    x = r.integers(-200, Nh + 200, N).astype(np.int32)
    y = r.integers(-200, Nh + 200, N).astype(np.int32)
    a = r.uniform(0.2, 1.0, N).astype(np.float32)
    d = r.integers(0, D, N).astype(np.int32)
    zd = np.linspace(zmin, zmax, D)
    lut = w.build_lut(lam, pitch, zd, W, L, gamma)
    p = w.pack_points(x, y, a, d)
    outs = []
    for rcap in (None, "1024"):
        if rcap:
            monkeypatch.setenv("WASABI_RANGE_CAP", rcap)
        out = w.hologram(lut, p, Nh, Nh, want=want)
        w.sync_status()
        outs.append([t.cpu().numpy() for t in (out if want == "both" else (out,))])
    for u, v in zip(*outs):
        assert np.array_equal(u, v)
    assert np.count_nonzero(outs[0][-1]) > 0
    lut.close()
