"""GPU Eq. (1) (cgh_direct) against the FP64 oracle: rel-L2 <= 1e-5."""
import os

import numpy as np
import pytest
import torch

from tests._helpers import rel_l2
from workloads import CONFIGS, uniform_cloud

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


@pytest.mark.parametrize("aperture", [True, False])
def test_small_direct(w, orc, aperture):
    lam, pitch, zmin, zmax, D, Nh = 633e-9, 1e-6, 50e-6, 300e-6, 8, 160
    pts = uniform_cloud(3, 40, Nh, zmin, zmax)
    pts["x"][:3] = [-30, Nh + 20, 0]
    zd = orc.depth_grid(zmin, zmax, D)
    d, _ = orc.quantize(pts["z"], zmin, zmax, D)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], d)
    u = w.cgh_direct(lam, pitch, zd, p, Nh, 96, aperture=aperture).cpu().numpy()
    w.sync_status()
    ref = orc.cgh_direct(lam, pitch, pts["x"], pts["y"], pts["a"], zd[d], 0, 0, Nh, 96, aperture)
    assert rel_l2(u, ref) <= 1e-5


def test_c1_direct(w, orc):
    c = CONFIGS["C1"]
    pts = c.points()
    zd = orc.depth_grid(c.zmin, c.zmax, c.D)
    d, _ = orc.quantize(pts["z"], c.zmin, c.zmax, c.D)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], d)
    u = w.cgh_direct(c.lam, c.pitch, zd, p, c.Nh, c.Nh).cpu().numpy()
    ref = orc.cgh_direct(c.lam, c.pitch, pts["x"], pts["y"], pts["a"], zd[d], 0, 0, c.Nh, c.Nh,
                         True, threads=NPROC)
    assert rel_l2(u, ref) <= 1e-5


def test_empty_points(w, orc):
    u = w.cgh_direct(633e-9, 1e-6, [1e-4], torch.empty((0, 4), dtype=torch.int32, device="cuda"), 64, 64)
    assert not u.abs().max().item()


def test_far_points_and_large_depths(w, orc):
    """Aperture off, depths of +-15 mm and points up to 20,000 pixels away:
    phases of some 4e4 cycles and pixel distances^2 beyond 2^24, where FP32
    alone would be off by ~1e-3 cycles; the double-float reduction holds the
    FP64 oracle's rel-L2 <= 1e-5."""
    lam, pitch, D, Nh, Nv = 633e-9, 1e-6, 4, 96, 64
    rng = np.random.default_rng(5)
    n = 24
    x = rng.integers(-20000, 20000, size=n).astype(np.int32)
    y = rng.integers(-20000, 20000, size=n).astype(np.int32)
    x[:4] = [10, 50, -3, 20000]
    y[:4] = [5, 60, 30, -19999]
    a = rng.uniform(0.5, 1.0, size=n).astype(np.float32)
    zd = orc.depth_grid(-15e-3, 15e-3, D)
    d = rng.integers(0, D, size=n).astype(np.int32)
    p = w.pack_points(x, y, a, d)
    u = w.cgh_direct(lam, pitch, zd, p, Nh, Nv, aperture=False).cpu().numpy()
    w.sync_status()
    ref = orc.cgh_direct(lam, pitch, x, y, a, zd[d], 0, 0, Nh, Nv, False)
    assert rel_l2(u, ref) <= 1e-5


def test_c2_direct_sampled_regions(w, orc):
    """Eq. (1) at the full C2 size (8,192^2, 100,000 height-field points, 64
    depths) as the benchmark runs it, against the FP64 oracle on 256 x 256
    regions (a corner and two interior regions).  Points farther than the
    largest support radius from a region add nothing to it (aperture form),
    so only those within reach are handed to the oracle."""
    c = CONFIGS["C2"]
    pts = c.points()
    zd = orc.depth_grid(c.zmin, c.zmax, c.D)
    d, bad = orc.quantize(pts["z"], c.zmin, c.zmax, c.D)
    assert bad == 0
    p = w.pack_points(pts["x"], pts["y"], pts["a"], d)
    u = w.cgh_direct(c.lam, c.pitch, zd, p, c.Nh, c.Nh)
    w.sync_status()
    rmax = float(orc.support_radius(c.lam, c.pitch, zd.max())) + 2
    S = 256
    g = np.random.default_rng(11)
    for ox, oy in [(0, 0)] + [tuple(int(v) for v in g.integers(0, c.Nh - S, 2)) for _ in range(2)]:
        near = ((pts["x"] >= ox - rmax) & (pts["x"] < ox + S + rmax) &
                (pts["y"] >= oy - rmax) & (pts["y"] < oy + S + rmax))
        ref = orc.cgh_direct(c.lam, c.pitch, pts["x"][near], pts["y"][near], pts["a"][near], zd[d[near]],
                             ox, oy, S, S, True, threads=NPROC)
        got = u[oy:oy + S, ox:ox + S].cpu().numpy()
        assert rel_l2(got, ref) <= 1e-5, (ox, oy)
