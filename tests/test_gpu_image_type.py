"""Image-type holograms (reading R11: points on both sides of the hologram
plane; a point behind it has the conjugate PSF, a point on it is a delta)
on the GPU against the oracle: LUT bit for bit, hologram and bits within
tolerance, Eq. (1) within tolerance."""
import os

import numpy as np
import pytest
import torch

from tests._helpers import rel_l2
from workloads import uniform_cloud

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1
LAM, PITCH, W, L = 532e-9, 1e-6, 256, 4


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


@pytest.fixture(scope="module")
def case(w, orc):
    zmin, zmax, D = -0.4e-3, 0.4e-3, 9  # bin centres include 0 (the middle bin)
    zd = orc.depth_grid(zmin, zmax, D)
    pts = uniform_cloud(21, 600, 512, zmin, zmax)
    pts["d"], bad = orc.quantize(pts["z"], zmin, zmax, D)
    assert bad == 0 and np.any(zd < 0) and np.any(zd > 0)
    return zd, pts


def test_lut_both_sides_bit_exact(w, orc, case):
    zd, _ = case
    lut = w.build_lut(LAM, PITCH, zd, W, L, 0.05)
    olut = orc.build_lut(LAM, PITCH, zd, W, L, 0.05, threads=NPROC)
    assert np.array_equal(lut.counts(), olut.nr)
    for d in range(len(zd)):
        oidx, oval = olut.depth(d)
        assert np.array_equal(lut.selection(d), oidx)
        idx, val = lut.entries(d)
        order = np.argsort(idx)
        assert np.array_equal(val[order], oval), d
    lut.close()


@pytest.mark.parametrize("rule", [0, 1])
def test_hologram_both_sides(w, orc, case, rule):
    zd, pts = case
    lut = w.build_lut(LAM, PITCH, zd, W, L, 0.05)
    olut = orc.build_lut(LAM, PITCH, zd, W, L, 0.05, threads=NPROC)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    u, bits = w.hologram(lut, p, 512, 512, want="both", rule=rule)
    w.sync_status()
    ref = orc.hologram(olut, pts, 512, rule=rule)
    assert rel_l2(u.cpu().numpy(), ref) <= 1e-5
    mine = np.unpackbits(bits.cpu().numpy(), bitorder="little").reshape(512, 512).astype(bool)
    diff = mine != (ref.real > 0)
    assert np.all(np.abs(ref.real[diff]) <= 1e-5 * np.abs(ref).max())
    lut.close()


def test_direct_eq1_both_sides(w, orc, case):
    zd, pts = case
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    u = w.cgh_direct(LAM, PITCH, zd, p, 512, 512).cpu().numpy()
    w.sync_status()
    ref = orc.cgh_direct(LAM, PITCH, pts["x"], pts["y"], pts["a"], zd[pts["d"]], 0, 0, 512, 512, True)
    assert rel_l2(u, ref) <= 1e-5
