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
