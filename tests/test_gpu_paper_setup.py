"""The geometry of the paper's own experiment (Sec. 2): object depths up to
15 mm before and after the plane at 1 um pitch need PSF windows of 9,664
pixels (1,208 window tiles at L = 3; sub-band positions up to 4,831 at
level 1, hence 13-bit position fields), a point on the plane is a delta
(R11), and the bits are taken against the spherical reference at
(0, 30 mm, -400 mm) (R12).  Three of the 29 depth bins, one 512^2
sub-hologram at two origins, against the oracle."""
import os

import numpy as np
import pytest
import torch

from tests._helpers import rel_l2
from workloads import uniform_cloud

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1
LAM, PITCH, W, L, GAMMA, NH = 632.8e-9, 1e-6, 9664, 3, 0.01, 65536


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


@pytest.fixture(scope="module")
def luts(w, orc):
    zd = orc.depth_grid(-15e-3, 15e-3, 29)[[0, 14, 23]]  # -14.5 mm, the plane, +8.8 mm
    lut = w.build_lut(LAM, PITCH, zd, W, L, GAMMA)
    olut = orc.build_lut(LAM, PITCH, zd, W, L, GAMMA, threads=min(3, NPROC))
    yield zd, lut, olut
    lut.close()


def test_wide_window_lut_bit_exact(w, orc, luts):
    zd, lut, olut = luts
    assert np.array_equal(lut.counts(), olut.nr)
    assert olut.nr[1] == 3 * L + 1  # the delta at the plane keeps all its coefficients
    for d in range(len(zd)):
        oidx, oval = olut.depth(d)
        assert np.array_equal(lut.selection(d), oidx), d
        idx, val = lut.entries(d)
        order = np.argsort(idx)
        assert np.array_equal(val[order], oval), d


@pytest.mark.parametrize("origin", [(30720, 24576), (0, 65024)])
def test_sub_hologram_with_the_paper_reference(w, orc, luts, origin):
    _, lut, olut = luts
    ox, oy = origin
    reach = 4832 + 16
    side = 512 + 2 * reach
    pts = uniform_cloud(61 + ox, 300, side, 0.0, 3.0)
    pts["x"] = (pts["x"] + ox - reach).astype(np.int32)
    pts["y"] = (pts["y"] + oy - reach).astype(np.int32)
    pts["d"] = np.minimum(pts["z"].astype(np.uint32), 2).astype(np.uint32)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    ref = w.spherical_reference(LAM, PITCH, NH / 2, NH / 2 + 30e-3 / PITCH, -0.4)
    u, bits = w.hologram(lut, p, 512, 512, want="both", origin=origin, reference=ref)
    w.sync_status()
    u_or = orc.haar_inv(orc.superpose(olut, pts, 512, ox, oy), L)
    u_np = u.cpu().numpy()
    assert rel_l2(u_np, u_or) <= 1e-5
    _, val = orc.binarize_ref(u_or, LAM, PITCH, NH / 2, NH / 2 + 30e-3 / PITCH, -0.4, ox, oy)
    mine = np.unpackbits(bits.cpu().numpy(), bitorder="little").reshape(512, 512).astype(bool)
    diff = mine != (val > 0)
    rms = np.sqrt(np.mean(np.abs(u_or) ** 2))
    assert np.all(np.abs(val[diff]) <= 5e-4 * np.abs(u_or[diff]) + 1e-5 * rms)
    assert diff.mean() < 1e-3


def test_all_29_depths_sampled_against_the_oracle(w, orc):
    """The full depth grid of the experiment: the build reports no
    inconsistency, and sampled depths (ties at the threshold resolved by
    Mallat indices beyond 2^24) match the oracle bit for bit."""
    zd = orc.depth_grid(-15e-3, 15e-3, 29)
    lut = w.build_lut(LAM, PITCH, zd, W, L, GAMMA)
    w.sync_status()
    sample = [2, 9, 16, 27]
    olut = orc.build_lut(LAM, PITCH, zd[sample], W, L, GAMMA, threads=min(4, NPROC))
    counts = lut.counts()
    for i, d in enumerate(sample):
        oidx, oval = olut.depth(i)
        assert counts[d] == olut.nr[i], d
        assert np.array_equal(lut.selection(d), oidx), d
        idx, val = lut.entries(d)
        assert np.array_equal(val[np.argsort(idx)], oval), d
    lut.close()
