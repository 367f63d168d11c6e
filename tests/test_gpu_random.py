"""Randomised parity sweep: seeded configurations drawn over levels, window,
keep ratio, depth range (both sides of the plane), hologram shape, shift
rule, point count, LUT dtype, sub-hologram origin and output form; each one
checked against the oracle (LUT index sets bit for bit, the field within
1e-5 for the FP32 LUT, bits only where |Re u| is within rounding of zero)."""
import numpy as np
import pytest
import torch

from tests._helpers import rel_l2
from workloads import uniform_cloud

pytestmark = pytest.mark.gpu
LAM = 633e-9


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


def _draw(seed):
    rng = np.random.default_rng(1000 + seed)
    L = int(rng.integers(2, 6))
    pitch = float(rng.choice([1e-6, 2e-6]))
    zlo = float(rng.uniform(-0.3e-3, 0.1e-3))
    zhi = zlo + float(rng.uniform(0.02e-3, 0.3e-3))
    D = int(rng.integers(1, 9))
    R = max(abs(zlo), abs(zhi)) * np.tan(np.arcsin(LAM / (2 * pitch))) / pitch
    unit = 2 << L
    W = int(np.ceil((2 * R + 1 + 1) / unit) * unit)
    gamma = float(rng.choice([0.01, 0.05, 0.2, 1.0]))
    side = int(rng.choice([256, 384, 512]))
    ts = 1 << L
    wd = side if rng.random() < 0.5 else max(ts * 8, (side - int(rng.integers(1, 8)) * 32) // ts * ts)
    ht = side
    rule = int(rng.integers(0, 2))
    n = int(rng.integers(0, 400))
    origin = (0, 0) if rng.random() < 0.5 else (int(rng.integers(-64, 64)), int(rng.integers(-64, 64)))
    want = str(rng.choice(["complex", "bits", "both"]))
    return L, pitch, zlo, zhi, D, W, gamma, wd, ht, rule, n, origin, want


@pytest.mark.parametrize("seed", range(48))
def test_random_configuration(w, orc, seed):
    L, pitch, zlo, zhi, D, W, gamma, wd, ht, rule, n, origin, want = _draw(seed)
    zd = orc.depth_grid(zlo, zhi, D)
    lut = w.build_lut(LAM, pitch, zd, W, L, gamma)
    olut = orc.build_lut(LAM, pitch, zd, W, L, gamma, threads=2)
    assert np.array_equal(lut.counts(), olut.nr), seed
    for d in range(D):
        assert np.array_equal(lut.selection(d), olut.depth(d)[0]), (seed, d)
    N = max(wd, ht)
    pts = uniform_cloud(seed, n, N, zlo, zhi)
    pts["x"] = (pts["x"] + origin[0]).astype(np.int32)
    pts["y"] = (pts["y"] + origin[1]).astype(np.int32)
    pts["d"], _ = orc.quantize(pts["z"], zlo, zhi, D)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"]) if n else torch.zeros((0, 4), dtype=torch.int32,
                                                                                   device="cuda")
    out = w.hologram(lut, p, wd, ht, want="both" if want == "both" else want, rule=rule, origin=origin)
    w.sync_status()
    ref = orc.haar_inv(orc.superpose(olut, pts, N, origin[0], origin[1], rule), L)[:ht, :wd]
    if want in ("complex", "both"):
        u = (out[0] if want == "both" else out).cpu().numpy()
        if np.any(ref):
            assert rel_l2(u, ref) <= 1e-5, seed
        else:
            assert not np.any(u), seed
    if want in ("bits", "both"):
        b = (out[1] if want == "both" else out).cpu().numpy()
        mine = np.unpackbits(b, bitorder="little")[: wd * ht].reshape(ht, wd).astype(bool)
        diff = mine != (ref.real > 0)
        scale = max(np.abs(ref).max(), 1e-30)
        assert np.all(np.abs(ref.real[diff]) <= 1e-5 * scale), seed
    lut.close()
