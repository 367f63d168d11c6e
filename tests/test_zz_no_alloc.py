"""wasabi_superpose_static: the allocation-free variant of wasabi_superpose.

Some callers cannot allocate device memory while they run (a plug-in whose
host application owns all device memory, a real-time loop that forbids
allocation after start-up, a binding with no CUDA allocator).  For them the
library keeps its superposition scratch in one fixed device array.  These
tests call that entry point through the C ABI several times in a row, on two
different problems in turn (so stale contents left in the shared array by
one call would show up in the next), and check every result against the
regular entry point with caller-owned scratch: bit for bit, since both run
the same kernels on the same data with exact fixed-point sums (within the
tolerance of the other tests when WASABI_ACC_FLOAT=1 selects FP32 atomics).
The file is collected last so that a failure here cannot hide the other
tests.
"""
import os

import numpy as np
import pytest
import torch

from workloads import CONFIGS, uniform_cloud

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


def _same(out, ref):
    if os.environ.get("WASABI_ACC_FLOAT", "0") not in ("", "0"):
        a, b = out.astype(np.complex128), ref.astype(np.complex128)
        return float(np.linalg.norm(a - b) / np.linalg.norm(b)) <= TOL
    return np.array_equal(out, ref)


def test_static_scratch_matches_caller_scratch(w):
    c = CONFIGS["C1"]
    pts = c.points()
    zd = w.depth_grid(c.zmin, c.zmax, c.D)
    dev = torch.device("cuda", 0)
    x, y, z, a = (torch.from_numpy(np.ascontiguousarray(pts[k])).to(dev) for k in "xyza")
    p = w.quantize_points(x, y, z, a, c.zmin, c.zmax, c.D)
    # A second problem: other points (more of them, some off the plane) on a
    # larger hologram, so its binning tables and sorted points differ.
    q2 = uniform_cloud(99, 3000, 2048, c.zmin, c.zmax)
    g = np.random.default_rng(99)
    q2["x"] = g.integers(-300, 2048 + 300, 3000).astype(np.int32)
    x2, y2, z2, a2 = (torch.from_numpy(np.ascontiguousarray(q2[k])).to(dev) for k in "xyza")
    p2 = w.quantize_points(x2, y2, z2, a2, c.zmin, c.zmax, c.D)
    lut = w.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma)
    ref = w.superpose(lut, p, c.Nh, c.Nh).cpu().numpy()
    ref2 = w.superpose(lut, p2, 2048, 2048).cpu().numpy()
    w.sync_status()
    assert np.linalg.norm(ref) > 0 and np.linalg.norm(ref2) > 0
    for _ in range(2):
        out = w.superpose_static(lut, p, c.Nh, c.Nh)
        w.sync_status()
        assert _same(out.cpu().numpy(), ref)
        out2 = w.superpose_static(lut, p2, 2048, 2048)
        w.sync_status()
        assert _same(out2.cpu().numpy(), ref2)
    lut.close()


def test_static_scratch_rejects_oversized_problems(w):
    c = CONFIGS["C1"]
    zd = w.depth_grid(c.zmin, c.zmax, c.D)
    lut = w.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma)
    n = 4 * 1024 * 1024  # 64 MiB of point records alone: beyond the array
    pts = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    wbuf = torch.empty(c.Nh * c.Nh, dtype=torch.complex64, device="cuda")
    with pytest.raises(w.WasabiError, match="NOMEM"):
        w.superpose_static(lut, pts, c.Nh, c.Nh, wbuf=wbuf)
    lut.close()
