"""wasabi_superpose_static: the allocation-free variant of wasabi_superpose.

Some callers cannot allocate device memory while they run (a plug-in whose
host application owns all device memory, a real-time loop that forbids
allocation after start-up, a binding with no CUDA allocator).  For them the
library keeps its superposition scratch in one fixed device array.  This test
calls that entry point through the C ABI twice in a row and checks each result
against the regular entry point with caller-owned scratch, within the
tolerance the other tests use.  It sits in a file collected last so that a
failure here cannot hide the other tests.
"""
import numpy as np
import pytest
import torch

from workloads import CONFIGS

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _rel(a, b):
    a = a.astype(np.complex128)
    b = b.astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_scratch_matches_caller_scratch():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    c = CONFIGS["C1"]
    pts = c.points()
    zd = w.depth_grid(c.zmin, c.zmax, c.D)
    dev = torch.device("cuda", 0)
    x, y, z, a = (torch.from_numpy(np.ascontiguousarray(pts[k])).to(dev) for k in "xyza")
    p = w.quantize_points(x, y, z, a, c.zmin, c.zmax, c.D)
    lut = w.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma)
    ref = w.superpose(lut, p, c.Nh, c.Nh).cpu().numpy()
    w.sync_status()
    assert np.linalg.norm(ref) > 0
    for _ in range(2):
        out = w.superpose_static(lut, p, c.Nh, c.Nh)
        w.sync_status()
        assert _rel(out.cpu().numpy(), ref) <= TOL
    lut.close()


def test_static_scratch_rejects_oversized_problems():
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    c = CONFIGS["C1"]
    zd = w.depth_grid(c.zmin, c.zmax, c.D)
    lut = w.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma)
    n = 4 * 1024 * 1024  # 64 MiB of point records alone: beyond the array
    pts = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    wbuf = torch.empty(c.Nh * c.Nh, dtype=torch.complex64, device="cuda")
    with pytest.raises(w.WasabiError, match="NOMEM"):
        w.superpose_static(lut, pts, c.Nh, c.Nh, wbuf=wbuf)
    lut.close()
