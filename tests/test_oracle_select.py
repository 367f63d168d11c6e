"""Pins for the oracle's shrinkage step (readings R3, R5; Sec. 1, step 1)."""
import numpy as np
import pytest


def _rank_count_select(coef, k):
    """Brute force by rank counting: entry i is kept iff fewer than k entries
    are stronger (larger key, or equal key and lower index)."""
    flat = coef.ravel()
    key = flat.real.astype(np.float64) ** 2 + flat.imag.astype(np.float64) ** 2
    kept = []
    for i in range(flat.size):
        if key[i] == 0:
            continue
        stronger = np.sum((key > key[i]) | ((key == key[i]) & (np.arange(flat.size) < i)))
        if stronger < k:
            kept.append(i)
    return np.array(kept, np.int32)


@pytest.mark.parametrize("seed", range(6))
def test_matches_rank_count_with_ties(orc, seed):
    rng = np.random.default_rng(seed)
    W = 16
    c = (rng.integers(-3, 4, (W, W)) + 1j * rng.integers(-3, 4, (W, W))).astype(np.complex64)
    # Zero one part of the grid so exact zeros are present.
    c[rng.random((W, W)) < 0.2] = 0
    for R in [3.0, 5.5, 8.0]:
        for gamma in [0.05, 0.2, 0.5]:
            k = min(orc.keep_target(gamma, R), int(np.count_nonzero(c)))
            got = orc.select(c, gamma, R)
            assert np.array_equal(got, _rank_count_select(c, k))


def test_tie_goes_to_lower_index(orc):
    W = 8
    c = np.zeros((W, W), np.complex64)
    c[5, 2] = 3 + 0j
    c[1, 6] = 3j          # same magnitude as c[5,2], lower index
    c[0, 1] = 1
    R = 2.0                         # gamma * pi * R^2 = 1: budget 1
    got = orc.select(c, 1.0 / (4.0 * np.pi), R)
    assert list(got) == [1 * W + 6]


def test_keep_all_is_nonzero_set(orc):
    rng = np.random.default_rng(7)
    W = 32
    c = (rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))).astype(np.complex64)
    c[rng.random((W, W)) < 0.5] = 0
    got = orc.select(c, 1.0, 3.0)
    assert np.array_equal(got, np.flatnonzero(c.ravel()).astype(np.int32))


def test_never_selects_zeros(orc):
    W = 8
    c = np.zeros((W, W), np.complex64)
    c[2, 3] = 1e-30
    got = orc.select(c, 0.5, 10.0)   # budget 158 > nnz = 1
    assert list(got) == [2 * W + 3]


def test_lut_sizes_c1(orc):
    zd = orc.depth_grid(0.2e-3, 0.9e-3, 16)
    lut = orc.build_lut(532e-9, 1e-6, zd, 512, 3, 0.05, threads=4)
    want = [orc.keep_target(0.05, orc.support_radius(532e-9, 1e-6, z)) for z in zd]
    assert list(lut.nr) == want
    for d in range(16):
        idx, val = lut.depth(d)
        assert np.all(np.diff(idx) > 0)
        assert np.all(val != 0)


def test_fp64_values_with_fp32_selection(orc):
    """The precision reference keeps the FP32 index set and carries FP64
    values, which differ from the FP32 values only by FP32 rounding."""
    zd = orc.depth_grid(20e-6, 150e-6, 6)
    l32 = orc.build_lut(633e-9, 1e-6, zd, 256, 4, 0.05, dtype="f32")
    l64 = orc.build_lut(633e-9, 1e-6, zd, 256, 4, 0.05, dtype="f64", select_fp32=True)
    assert np.array_equal(l32.nr, l64.nr)
    assert np.array_equal(l32.idx, l64.idx)
    assert l64.val.dtype == np.complex128
    assert np.max(np.abs(l64.val - l32.val.astype(np.complex128))) < 2e-6
