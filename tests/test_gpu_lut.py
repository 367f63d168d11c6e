"""GPU LUT builder (Sec. 1, step 1) against the oracle: kept index sets bit for
bit, FP32 values bit for bit, reduced-precision values within their rounding."""
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


def _compare(w, orc, lam, pitch, zd, W, L, gamma, threads=os.cpu_count() or 1):
    lut = w.build_lut(lam, pitch, zd, W, L, gamma)
    olut = orc.build_lut(lam, pitch, zd, W, L, gamma, threads=threads)
    assert np.array_equal(lut.counts(), olut.nr)
    for d in range(len(zd)):
        oidx, oval = olut.depth(d)
        sel = lut.selection(d)
        assert np.array_equal(sel, oidx), f"depth {d}: {np.setxor1d(sel, oidx).size} indices differ"
        idx, val = lut.entries(d)
        order = np.argsort(idx)
        assert np.array_equal(idx[order], oidx)
        assert np.array_equal(val[order], oval), f"depth {d}: values differ"
    return lut, olut


def test_c1_lut_bit_exact(w, orc):
    zd = orc.depth_grid(0.2e-3, 0.9e-3, 16)
    _compare(w, orc, 532e-9, 1e-6, zd, 512, 3, 0.05)


def test_c2_lut_bit_exact(w, orc):
    zd = orc.depth_grid(0.3e-3, 1.0e-3, 64)
    _compare(w, orc, 633e-9, 1e-6, zd, 1024, 4, 0.02)


@pytest.mark.parametrize("L,W", [(1, 128), (2, 128), (3, 128), (5, 128)])
def test_levels(w, orc, L, W):
    zd = orc.depth_grid(20e-6, 150e-6, 5)
    _compare(w, orc, 633e-9, 1e-6, zd, W, L, 0.1)


def test_keep_all_is_nonzero_set(w, orc):
    zd = orc.depth_grid(20e-6, 150e-6, 3)
    lut, olut = _compare(w, orc, 633e-9, 1e-6, zd, 128, 3, 1.0)
    for d in range(3):
        coef = orc.haar_fwd(orc.psf_f32(633e-9, 1e-6, zd[d], 128), 3)
        assert np.array_equal(lut.selection(d), np.flatnonzero(coef.ravel()).astype(np.int32))


def test_tiny_budget(w, orc):
    zd = orc.depth_grid(20e-6, 60e-6, 2)
    _compare(w, orc, 633e-9, 1e-6, zd, 64, 3, 1e-4)   # budgets of one coefficient


@pytest.mark.parametrize("dtype,ulp", [("f16s", 2.0 ** -11), ("bf16s", 2.0 ** -8)])
def test_reduced_precision_values(w, orc, dtype, ulp):
    zd = orc.depth_grid(0.3e-3, 1.0e-3, 8)
    ref = w.build_lut(633e-9, 1e-6, zd, 1024, 4, 0.02)
    lut = w.build_lut(633e-9, 1e-6, zd, 1024, 4, 0.02, dtype=dtype)
    for d in range(8):
        i0, v0 = ref.entries(d)
        i1, v1 = lut.entries(d)
        assert np.array_equal(i0, i1)
        # Per block of 32 entries: scale = max |re|, |im|; error <= half an ulp of the
        # stored value (|q| <= 1) times the scale.
        for b in range(0, v0.size, 32):
            blk = v0[b:b + 32]
            s = max(np.abs(blk.real).max(), np.abs(blk.imag).max())
            err = np.abs(v1[b:b + 32] - blk)
            assert err.max() <= ulp * s * 1.0001
