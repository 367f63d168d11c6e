"""Frames on the GPU: sub-holograms (Sec. 1, large-scale steps 2-4: the
coordinate transform x'_j = x_j - s N_h) and binarisation against a
spherical reference wave (Sec. 2; reading R12), against the oracle, through
the fused path, the two-pass path, batches and the server."""
import numpy as np
import pytest
import torch

from tests._helpers import rel_l2
from workloads import uniform_cloud

pytestmark = pytest.mark.gpu
LAM, PITCH, ZMIN, ZMAX = 633e-9, 1e-6, 20e-6, 150e-6
# Phase error of the GPU's reference wave: below 4e-5 cycles (2.5e-4 rad);
# bits may differ from the oracle's only where |Re(u conj R)| is that close
# to zero, on top of the field's own rounding.
PHASE_TOL = 5e-4


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


def _lut(w, orc, L, W, gamma, D, dtype="f32"):
    """The GPU LUT in `dtype` and the oracle's FP32 LUT (reading R8)."""
    zd = orc.depth_grid(ZMIN, ZMAX, D)
    return (w.build_lut(LAM, PITCH, zd, W, L, gamma, dtype=dtype),
            orc.build_lut(LAM, PITCH, zd, W, L, gamma))


def _points(w, orc, seed, n, side, D, lo=0):
    pts = uniform_cloud(seed, n, side, ZMIN, ZMAX)
    pts["x"] = (pts["x"] + lo).astype(np.int32)
    pts["y"] = (pts["y"] + lo).astype(np.int32)
    pts["d"], _ = orc.quantize(pts["z"], ZMIN, ZMAX, D)
    return pts, w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])


def _oracle_u(orc, olut, pts, N, L, ox, oy, rule):
    """Sub-hologram of side N at plane pixel (ox, oy): Eq. (2) with the
    coordinate transform, then the inverse transform."""
    return orc.haar_inv(orc.superpose(olut, pts, N, ox, oy, rule), L)


def _unpack(bits, h, w_):
    return np.unpackbits(bits.cpu().numpy(), bitorder="little")[: h * w_].reshape(h, w_).astype(bool)


def _check_ref_bits(orc, bits, u_or, ref, ox, oy):
    """bits against the oracle's Re(u_or conj R) > 0 for the field u_or."""
    h, w_ = u_or.shape
    _, val = orc.binarize_ref(u_or, ref["lam"], ref["pitch"], ref["x"], ref["y"], ref["z"], ox, oy)
    mine = _unpack(bits, h, w_)
    diff = mine != (val > 0)
    rms = np.sqrt(np.mean(np.abs(u_or) ** 2))
    margin = PHASE_TOL * np.abs(u_or) + 1e-5 * rms
    assert np.all(np.abs(val[diff]) <= margin[diff]), int(diff.sum())
    assert diff.mean() < 1e-3
    return diff


@pytest.mark.parametrize("origin", [(512, 0), (-256, 384), (100, -36), (5000, 5000)])
@pytest.mark.parametrize("rule", [0, 1])
def test_subhologram_matches_the_oracle(w, orc, origin, rule):
    L, W, N = 4, 128, 512
    lut, olut = _lut(w, orc, L, W, 0.1, 8)
    pts, p = _points(w, orc, 3, 900, 1024, 8, lo=-200)
    u = w.hologram(lut, p, N, N, want="complex", rule=rule, origin=origin)
    w.sync_status()
    ref = _oracle_u(orc, olut, pts, N, L, *origin, rule)
    if not np.any(ref):
        assert not torch.any(u)  # no point reaches this sub-hologram
    else:
        assert rel_l2(u.cpu().numpy(), ref) <= 1e-5
    # The two-pass path: superposition of the sub-hologram, inverse transform.
    wb = w.superpose(lut, p, N, N, rule=rule, origin=origin)
    u2 = w.inverse_haar(wb, N, N, L)
    assert torch.equal(u, u2)
    lut.close()


def test_subholograms_tile_the_full_hologram(w, orc):
    """Origins on the 2^L grid: the sub-holograms are crops of the whole
    hologram (tiles of the Haar transform are independent)."""
    L, W = 4, 128
    lut, _ = _lut(w, orc, L, W, 0.1, 8)
    _, p = _points(w, orc, 4, 1500, 1024, 8)
    full = w.hologram(lut, p, 1024, 1024).cpu().numpy()
    for oy in (0, 512):
        for ox in (0, 512):
            sub = w.hologram(lut, p, 512, 512, origin=(ox, oy)).cpu().numpy()
            assert rel_l2(sub, full[oy:oy + 512, ox:ox + 512]) <= 1e-6
    w.sync_status()
    lut.close()


REF_CASES = [  # L, W, gamma, D, w, h, rule, dtype, origin, (x_r, y_r, z_r)
    (4, 128, 0.1, 8, 512, 512, 0, "f32", (0, 0), (256.0, 30256.0, -0.4)),      # paper: 30 mm up, 400 mm behind
    (4, 128, 0.1, 8, 320, 176, 1, "f32", (64, -32), (-90.5, 40.25, -0.05)),    # ragged, fractional source
    (2, 128, 0.2, 6, 264, 136, 0, "f32", (8, 8), (130.0, 70.0, 2e-3)),         # w % 32 != 0, source in front
    (3, 128, 1.0, 6, 384, 256, 1, "f32", (0, 0), (10.0, -4000.0, -0.1)),       # level 1 present
    (5, 128, 0.05, 4, 512, 384, 0, "bf16s", (-96, 160), (0.0, 0.0, 0.4)),
]


@pytest.mark.parametrize("case", REF_CASES)
def test_spherical_reference_bits(w, orc, case):
    L, W, gamma, D, wd, ht, rule, dtype, origin, (xr, yr, zr) = case
    lut, olut = _lut(w, orc, L, W, gamma, D, dtype)
    pts, p = _points(w, orc, 11, 500, max(wd, ht), D, lo=min(origin))
    ref = w.spherical_reference(LAM, PITCH, xr, yr, zr)
    N = max(wd, ht)
    u_or = _oracle_u(orc, olut, pts, N, L, *origin, rule)[:ht, :wd]
    # Bits alone (complex accumulation all the same), and with the field.
    bits = w.hologram(lut, p, wd, ht, want="bits", rule=rule, origin=origin, reference=ref)
    u, bits2 = w.hologram(lut, p, wd, ht, want="both", rule=rule, origin=origin, reference=ref)
    w.sync_status()
    assert torch.equal(bits, bits2)
    # The field against the oracle's (FP32 LUT: reduced-precision forms carry
    # their own quantisation error), the bits against the oracle's reference
    # binarisation of the field they come from.
    u_np = u.cpu().numpy()
    assert rel_l2(u_np, u_or) <= (1e-5 if dtype == "f32" else 1e-2)
    _check_ref_bits(orc, bits, u_np, ref, *origin)
    if dtype == "f32":
        _check_ref_bits(orc, bits, u_or, ref, *origin)
    # The two-pass path anchors the reference phase per strip instead of per
    # super-tile: same bits up to the same margin.
    wb = w.superpose(lut, p, wd, ht, rule=rule, origin=origin)
    u3, bits3 = w.inverse_haar(wb, wd, ht, L, want="both", origin=origin, reference=ref)
    w.sync_status()
    assert torch.equal(u3, u)
    _check_ref_bits(orc, bits3, u_np, ref, *origin)
    # Without a reference the bits are those of Re u > 0.
    plain = w.hologram(lut, p, wd, ht, want="bits", rule=rule, origin=origin)
    diff = _unpack(plain, ht, wd) != (u_np.real > 0)
    assert np.all(np.abs(u_np.real[diff]) <= 1e-5 * np.abs(u_np).max())
    lut.close()


def test_batch_and_server_carry_frames(w, orc):
    """Jobs with and without frames in one batch, and server requests, equal
    the one-hologram calls."""
    L, W, D = 4, 128, 8
    lut, _ = _lut(w, orc, L, W, 0.1, D)
    ref = w.spherical_reference(LAM, PITCH, 100.0, -30000.0, -0.4)
    specs = [(31, 300, 512, "bits", 0, (0, 0), ref), (32, 200, 256, "both", 1, (128, 64), None),
             (33, 250, 384, "bits", 0, (-64, 0), None), (34, 100, 256, "both", 0, (32, 32), ref)]
    jobs = []
    for seed, n, side, want, rule, origin, r in specs:
        _, p = _points(w, orc, seed, n, side, D)
        jobs.append({"points": p, "w": side, "h": side, "rule": rule, "want": want, "origin": origin,
                     "reference": r})
    batch = w.Batch(lut, 8, side_hint=512, use_graph=True)
    stream = torch.cuda.Stream()
    for _ in range(2):  # capture, then replay
        with torch.cuda.stream(stream):
            res = batch.run(jobs, stream=stream)
        stream.synchronize()
        w.sync_status(stream)
        for j, r in zip(jobs, res):
            single = w.hologram(lut, j["points"], j["w"], j["h"], want="both", rule=j["rule"],
                                origin=j["origin"], reference=j["reference"])
            assert torch.equal(r["bits"], single[1])
            if r["u"] is not None:
                assert torch.equal(r["u"], single[0])
    batch.close()

    srv = w.Server(lut, 512 << 20, streams=2, max_batch=4, side_hint=512)
    ids = []
    for j in jobs:
        ids.append(srv.submit(j["points"].cpu().pin_memory(), j["w"], j["h"], want="bits", rule=j["rule"],
                              origin=j["origin"], reference=j["reference"]))
    for j, rid in zip(jobs, ids):
        got = srv.wait(rid, 30.0)["bits"]
        single = w.hologram(lut, j["points"], j["w"], j["h"], want="bits", rule=j["rule"], origin=j["origin"],
                            reference=j["reference"])
        assert torch.equal(got, single.cpu())
    srv.close()
    lut.close()


def test_invalid_frames_are_refused(w, orc):
    lut, _ = _lut(w, orc, 4, 128, 0.1, 8)
    _, p = _points(w, orc, 5, 50, 256, 8)
    bad = [w.spherical_reference(LAM, PITCH, 0.0, 0.0, 0.0),
           w.spherical_reference(-LAM, PITCH, 0.0, 0.0, 0.1),
           w.spherical_reference(LAM, 0.0, 0.0, 0.0, 0.1),
           w.spherical_reference(LAM, PITCH, float("nan"), 0.0, 0.1),
           w.spherical_reference(LAM, PITCH, 0.0, 0.0, float("inf"))]
    for ref in bad:
        with pytest.raises(w.WasabiError, match="INVALID"):
            w.hologram(lut, p, 256, 256, want="bits", reference=ref)
        wb = w.superpose(lut, p, 256, 256)
        with pytest.raises(w.WasabiError, match="INVALID"):
            w.inverse_haar(wb, 256, 256, 4, want="bits", reference=ref)
    w.sync_status()
    lut.close()


@pytest.mark.parametrize("want,band_h", [("bits", 256), ("both", 192), ("complex", 4096)])
def test_streamed_bands_equal_the_sub_holograms(w, orc, want, band_h):
    """wasabi_hologram_stream: band k equals the one-call sub-hologram at
    (origin_x, origin_y + k band_h) (each band is its own job, so its
    fixed-point scale is its own: equal to rounding; bits up to flips at
    |Re u| within rounding of zero); the last band is shorter."""
    L, W, D = 4, 128, 8
    lut, olut = _lut(w, orc, L, W, 0.1, D)
    pts, p = _points(w, orc, 41, 3000, 1024, D)
    wd, ht, origin = 768, 1008, (64, -32)
    ref = w.spherical_reference(LAM, PITCH, 300.0, -20000.0, -0.4) if want == "both" else None
    out = w.hologram_stream(lut, p, wd, ht, band_h, want=want, origin=origin, reference=ref)
    w.sync_status()
    u_s, bits_s = (out if want == "both" else (out, None) if want == "complex" else (None, out))
    one_u, one_bits = w.hologram(lut, p, wd, ht, want="both", origin=origin, reference=ref)
    one_u = one_u.cpu().numpy()
    if u_s is not None:
        assert not u_s.is_cuda and rel_l2(u_s.numpy(), one_u) <= 1e-6
    if bits_s is not None:
        assert not bits_s.is_cuda
        if ref is None:
            diff = _unpack(bits_s, ht, wd) != _unpack(one_bits, ht, wd)
            assert np.all(np.abs(one_u.real[diff]) <= 1e-5 * np.abs(one_u).max())
        else:
            _check_ref_bits(orc, bits_s, one_u, ref, *origin)
    # Against the oracle too: the streamed field is the sub-hologram's.
    if u_s is not None:
        N = 1024
        u_or = _oracle_u(orc, olut, pts, N, L, *origin, 0)[:ht, :wd]
        assert rel_l2(u_s.numpy(), u_or) <= 1e-5
    lut.close()
