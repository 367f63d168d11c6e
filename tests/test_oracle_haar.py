"""Pins for the oracle's Haar transform (reading R4; Sec. 1 steps 1 and 3, Fig. 2(a))."""
import numpy as np
import pytest


def _cplx(rng, n, dtype=np.complex128):
    return (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(dtype)


def test_hand_2x2(orc):
    a = np.array([[1, 2], [3, 4]], np.complex128) * (1 + 2j)
    c = orc.haar_fwd(a, 1)
    # s = 10/2, LH = -2/2, HL = -4/2, HH = 0
    want = np.array([[5, -1], [-2, 0]], np.complex128) * (1 + 2j)
    assert np.array_equal(c, want)


def test_hand_delta_4x4_two_levels(orc):
    a = np.zeros((4, 4), np.complex128)
    a[0, 0] = 1
    c = orc.haar_fwd(a, 2)
    want = np.array([[0.25, 0.25, 0.5, 0.0],
                     [0.25, 0.25, 0.0, 0.0],
                     [0.5, 0.0, 0.5, 0.0],
                     [0.0, 0.0, 0.0, 0.0]])
    assert np.array_equal(c.real, want) and not c.imag.any()


def test_lh_is_high_pass_along_x(orc):
    # A pattern alternating along x (columns) only: all level-1 energy in LH,
    # which sits at rows [0, n/2) x columns [n/2, n).
    n = 8
    a = np.tile(np.array([1.0, -1.0] * (n // 2)), (n, 1)).astype(np.complex128)
    c = orc.haar_fwd(a, 1)
    h = n // 2
    assert np.allclose(c[:h, h:], 2.0)
    c[:h, h:] = 0
    assert not np.any(c)


def _matrix_haar(x, L):
    """Independent textbook form: one level is Y = A X A^T with A the
    orthonormal analysis matrix (low-pass rows [1 1]/sqrt2 over high-pass
    rows [1 -1]/sqrt2); the levels recurse on the low-low quadrant."""
    x = x.copy()
    n = x.shape[0]
    for l in range(L):
        S = n >> l
        h = S // 2
        A = np.zeros((S, S))
        for i in range(h):
            A[i, 2 * i] = A[i, 2 * i + 1] = 1 / np.sqrt(2)
            A[h + i, 2 * i] = 1 / np.sqrt(2)
            A[h + i, 2 * i + 1] = -1 / np.sqrt(2)
        x[:S, :S] = A @ x[:S, :S] @ A.T
    return x


@pytest.mark.parametrize("n,L", [(8, 1), (16, 3), (64, 4), (32, 5)])
def test_matches_matrix_form(orc, n, L):
    x = _cplx(np.random.default_rng(n + L), n)
    assert np.allclose(orc.haar_fwd(x, L), _matrix_haar(x, L), atol=1e-12)


@pytest.mark.parametrize("L", [1, 3, 4])
def test_round_trip_and_parseval(orc, L):
    rng = np.random.default_rng(L)
    x = _cplx(rng, 128)
    c = orc.haar_fwd(x, L)
    assert abs(np.sum(np.abs(c) ** 2) - np.sum(np.abs(x) ** 2)) < 1e-9 * np.sum(np.abs(x) ** 2)
    y = orc.haar_inv(c, L)
    assert np.max(np.abs(y - x)) <= 1e-15 * np.max(np.abs(x)) * 8
    xf = x.astype(np.complex64)
    yf = orc.haar_inv(orc.haar_fwd(xf, L), L)
    eps = np.finfo(np.float32).eps
    assert np.max(np.abs(yf - xf)) <= 2 * L * eps * np.max(np.abs(xf)) * 4


def test_constant_block_has_only_scaling(orc):
    L = 4
    x = np.full((16, 16), 0.75 - 0.5j, np.complex128)
    c = orc.haar_fwd(x, L)
    assert c[0, 0] == (0.75 - 0.5j) * 2 ** L
    c[0, 0] = 0
    assert not np.any(c)


def test_delta_pattern(orc):
    # A unit delta gives one coefficient of magnitude 2^-l in each of the
    # three detail bands at every level l, and 2^-L in the scaling band.
    L, n = 3, 32
    x = np.zeros((n, n), np.complex128)
    x[13, 6] = 1
    c = orc.haar_fwd(x, L)
    mags = sorted(np.abs(c[c != 0]).tolist())
    want = sorted([2.0 ** -l for l in range(1, L + 1) for _ in range(3)] + [2.0 ** -L])
    assert np.allclose(mags, want, rtol=0, atol=0)


def test_mallat_decode_round_trip(orc):
    n, L = 64, 4
    seen = set()
    for row in range(n):
        for col in range(n):
            lev, band, p, q = orc.mallat_decode(row, col, n, L)
            S = n >> lev
            assert 0 <= p < S and 0 <= q < S
            assert (band == 0) == (row < (n >> L) and col < (n >> L))
            seen.add((lev, band, p, q))
    assert len(seen) == n * n
