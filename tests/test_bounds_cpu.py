"""The element-wise error bound of the GPU parity tests (tests/_bounds.py),
pinned on the CPU: it holds between the FP32 oracle and the FP64 oracle on
the same index set (a different computation of the same sums), and it
rejects a result with one dropped or one misplaced coefficient (mistakes
planted in a copy of the oracle's LUT)."""
from dataclasses import replace

import numpy as np
import pytest

from tests._bounds import FieldBound, check_bits, check_field
from workloads import uniform_cloud

LAM, PITCH, ZMIN, ZMAX, D, W, L, NH = 633e-9, 1e-6, 20e-6, 150e-6, 4, 128, 4, 256


@pytest.fixture(scope="module")
def case(orc):
    pts = uniform_cloud(31, 80, NH, ZMIN, ZMAX)
    zd = orc.depth_grid(ZMIN, ZMAX, D)
    pts["d"], _ = orc.quantize(pts["z"], ZMIN, ZMAX, D)
    o32 = orc.build_lut(LAM, PITCH, zd, W, L, 0.1)
    o64 = orc.build_lut(LAM, PITCH, zd, W, L, 0.1, dtype="f64", select_fp32=True)
    return pts, o32, o64


def test_bound_holds_between_fp32_and_fp64(orc, case):
    pts, o32, o64 = case
    fb = FieldBound(orc, o32, pts, NH)
    u32 = orc.hologram(o32, pts, NH)
    u64 = orc.hologram(o64, pts, NH)
    check_field(u32, u64, fb.window(NH, 0, 0), factor=1.0)
    check_bits(u32.real > 0, u64, fb.window(NH, 0, 0), factor=1.0)
    psi32 = orc.superpose(o32, pts, NH)
    psi64 = orc.superpose(o64, pts, NH)
    check_field(psi32, psi64, fb.coeffs(NH, 0, 0), factor=1.0)


def _strongest(lut, d):
    idx, val = lut.depth(d)
    return int(lut.offsets[d] + np.argmax(np.abs(val)))


@pytest.mark.parametrize("mistake", ["dropped", "misplaced"])
def test_bound_rejects_a_planted_mistake(orc, case, mistake):
    pts, o32, _ = case
    d = int(np.bincount(pts["d"], minlength=D).argmax())
    e = _strongest(o32, d)
    if mistake == "dropped":
        val = o32.val.copy()
        val[e] = 0
        bad = replace(o32, val=val)
    else:
        idx = o32.idx.copy()
        taken = set(o32.depth(d)[0].tolist())
        step = 1
        while int(idx[e]) + step in taken:
            step += 1
        idx[e] += step
        order = np.argsort(idx[o32.offsets[d]:o32.offsets[d + 1]], kind="stable")
        sl = slice(o32.offsets[d], o32.offsets[d + 1])
        val = o32.val.copy()
        idx[sl], val[sl] = idx[sl][order], val[sl][order]
        bad = replace(o32, idx=idx, val=val)
    fb = FieldBound(orc, o32, pts, NH)
    ref = orc.hologram(o32, pts, NH)
    got = orc.hologram(bad, pts, NH)
    with pytest.raises(AssertionError):
        check_field(got, ref, fb.window(NH, 0, 0))
    with pytest.raises(AssertionError):
        check_field(orc.superpose(bad, pts, NH), orc.superpose(o32, pts, NH), fb.coeffs(NH, 0, 0))
