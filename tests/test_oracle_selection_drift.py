"""How far the FP32 phase recipe of the LUT (reading R8: an FP32 root with
one FP64 Newton step, FP32 sincos) moves the selection of "the N_r strong
coefficients" (Sec. 1, step 1) away from selecting on the definition: the
FP64 PSF u_z = exp(i 2 pi r / lambda) circ(...) rounded to complex64, then
the same FP32 Haar transform and the same selection rule (R5).

Both index sets come from the oracle alone.  Indices in one set and not the
other must all be near-ties at the N_r-th key: their keys (FP64 squares of
the FP32 coefficients, either form) lie within a small relative margin of
that threshold key.  The counts are printed (the design notes record them)."""
import numpy as np
import pytest

from workloads import CONFIGS

MARGIN = 1e-6  # relative: a few FP32 ulps of the key


def _keys(c):
    c = c.ravel()
    return c.real.astype(np.float64) ** 2 + c.imag.astype(np.float64) ** 2


@pytest.mark.parametrize("name", ["C1", "C2"])
def test_r8_selection_differs_only_at_near_ties(orc, name):
    c = CONFIGS[name]
    zd = orc.depth_grid(c.zmin, c.zmax, c.D)
    total_diff = 0
    total_kept = 0
    worst = 0.0
    for z in zd:
        R = orc.support_radius(c.lam, c.pitch, z)
        c_r8 = orc.haar_fwd(orc.psf_f32(c.lam, c.pitch, z, c.W), c.L)
        c_def = orc.haar_fwd(orc.psf_f64(c.lam, c.pitch, z, c.W).astype(np.complex64), c.L)
        s_r8 = orc.select(c_r8, c.gamma, R)
        s_def = orc.select(c_def, c.gamma, R)
        assert s_r8.size == s_def.size
        total_kept += s_r8.size
        diff = np.setxor1d(s_r8, s_def)
        total_diff += diff.size
        if diff.size == 0:
            continue
        for keys, sel in ((_keys(c_r8), s_r8), (_keys(c_def), s_def)):
            thr = keys[sel].min()  # the N_r-th key of this form
            rel = np.abs(keys[diff] - thr) / thr
            worst = max(worst, float(rel.max()))
            assert np.all(rel <= MARGIN), (float(z), float(rel.max()))
    print(f"{name}: {total_diff} indices differ (symmetric difference) of {total_kept} kept over "
          f"{c.D} depths; worst distance from the threshold key {worst:.2e} (relative)")
