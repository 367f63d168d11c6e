"""Superposition fused with the inverse transform and binarisation
(wasabi_hologram) against the two-pass path (wasabi_superpose +
wasabi_inverse_haar): same super-tile configuration, so the pixels and bits
must agree exactly, and a wavelet buffer written on the way must equal the
one wasabi_superpose writes."""
import numpy as np
import pytest
import torch

from tests._helpers import rel_l2
from workloads import uniform_cloud

pytestmark = pytest.mark.gpu
LAM, PITCH, ZMIN, ZMAX = 633e-9, 1e-6, 20e-6, 150e-6


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


def _points(w, orc, seed, n, side, D):
    pts = uniform_cloud(seed, n, side, ZMIN, ZMAX)
    pts["d"], _ = orc.quantize(pts["z"], ZMIN, ZMAX, D)
    return pts, w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])


CASES = [  # L, W, gamma, D, w, h, rule, dtype, n
    (4, 128, 0.1, 8, 512, 512, 0, "f32", 400),
    (4, 128, 0.1, 8, 320, 176, 1, "f32", 300),      # ragged super-tiles, partial bit words
    (2, 128, 0.2, 6, 264, 136, 0, "f32", 250),      # w % 32 != 0: byte stores
    (3, 128, 1.0, 6, 384, 256, 1, "f32", 200),      # keep all: level 1 present
    (5, 128, 0.05, 4, 512, 384, 0, "f32", 300),
    (4, 128, 0.1, 8, 512, 512, 0, "f16s", 400),
    (4, 128, 0.1, 8, 512, 512, 1, "bf16s", 400),
]


@pytest.mark.parametrize("case", CASES, ids=[f"L{c[0]}-g{c[2]}-{c[4]}x{c[5]}-r{c[6]}-{c[7]}" for c in CASES])
def test_fused_equals_two_pass(w, orc, case):
    L, W, gamma, D, hw, hh, rule, dt, n = case
    zd = w.depth_grid(ZMIN, ZMAX, D)
    lut = w.build_lut(LAM, PITCH, zd, W, L, gamma, dtype=dt)
    _, p = _points(w, orc, 100 + L, n, min(hw, hh), D)
    wb2 = w.superpose(lut, p, hw, hh, rule=rule)
    u2, b2 = w.inverse_haar(wb2, hw, hh, L, want="both")
    wb1 = torch.empty_like(wb2)
    u1, b1 = w.hologram(lut, p, hw, hh, want="both", rule=rule, wbuf=wb1)
    w.sync_status()
    assert torch.equal(wb1, wb2)
    assert torch.equal(u1, u2)
    assert torch.equal(b1, b2)
    # Outputs one at a time.
    assert torch.equal(w.hologram(lut, p, hw, hh, want="bits", rule=rule), b2)
    assert torch.equal(w.hologram(lut, p, hw, hh, want="complex", rule=rule), u2)
    assert float(u2.abs().max()) > 0
    lut.close()


def test_fused_float_accumulator(w, orc, monkeypatch):
    monkeypatch.setenv("WASABI_ACC_FLOAT", "1")
    zd = w.depth_grid(ZMIN, ZMAX, 8)
    lut = w.build_lut(LAM, PITCH, zd, 128, 4, 0.1)
    pts, p = _points(w, orc, 7, 300, 512, 8)
    u1 = w.hologram(lut, p, 512, 512).cpu().numpy()
    olut = orc.build_lut(LAM, PITCH, zd, 128, 4, 0.1)
    assert rel_l2(u1, orc.hologram(olut, pts, 512)) <= 1e-5
    lut.close()


def test_fused_empty_and_invalid(w, orc):
    zd = w.depth_grid(ZMIN, ZMAX, 4)
    lut = w.build_lut(LAM, PITCH, zd, 128, 2, 0.1)
    empty = torch.zeros((0, 4), dtype=torch.int32, device="cuda")
    u, b = w.hologram(lut, empty, 256, 128, want="both")
    w.sync_status()
    assert not u.any() and not b.any()
    _, p = _points(w, orc, 3, 10, 64, 4)
    with pytest.raises(w.WasabiError, match="INVALID"):
        w.hologram(lut, p, 12, 16, want="bits")   # bits need holo_w % 8 == 0
    scratch = torch.empty(w.scratch_bytes(lut, 10, 64, 64), dtype=torch.uint8, device="cuda")
    from paper_1708_04233_gb300 import _abi
    with pytest.raises(w.WasabiError, match="INVALID"):  # no output at all
        _abi.check(_abi.load().wasabi_hologram(lut.handle, p.data_ptr(), 10, 64, 64, 0, None, None, None,
                                               scratch.data_ptr(), scratch.numel(), None))
    lut.close()


def test_points_outside_the_hologram(w, orc):
    """Points up to 100 pixels outside the hologram still contribute the part
    of their footprint that lands inside it (Eq. (2) drops only the
    coefficients that land outside)."""
    D = 6
    zd = w.depth_grid(ZMIN, ZMAX, D)
    lut = w.build_lut(LAM, PITCH, zd, 128, 4, 0.2)
    olut = orc.build_lut(LAM, PITCH, zd, 128, 4, 0.2)
    g = np.random.default_rng(5)
    n = 400
    pts = {"x": g.integers(-100, 356, n).astype(np.int32), "y": g.integers(-100, 356, n).astype(np.int32),
           "a": (1.0 - g.random(n)).astype(np.float32), "z": g.uniform(ZMIN, ZMAX, n)}
    pts["d"], _ = orc.quantize(pts["z"], ZMIN, ZMAX, D)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    for rule in (0, 1):
        u = w.hologram(lut, p, 256, 256, rule=rule).cpu().numpy()
        assert rel_l2(u, orc.hologram(olut, pts, 256, rule=rule)) <= 1e-5
    w.sync_status()
    lut.close()
