"""GPU Haar transforms (tile-major layout) and binary hologram against the oracle."""
import numpy as np
import pytest
import torch

from tests._helpers import tile_major_to_mallat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


def _img(seed, h, w_):
    r = np.random.default_rng(seed)
    return (r.standard_normal((h, w_)) + 1j * r.standard_normal((h, w_))).astype(np.complex64)


@pytest.mark.parametrize("L,n", [(1, 32), (2, 64), (3, 256), (4, 512), (5, 256)])
def test_forward_matches_oracle(w, orc, L, n):
    x = _img(L, n, n)
    wb = w.haar_forward(torch.from_numpy(x).cuda(), L).cpu().numpy()
    assert np.array_equal(tile_major_to_mallat(wb, n, n, L), orc.haar_fwd(x, L))


@pytest.mark.parametrize("L,h,w_", [(3, 64, 200), (4, 48, 1040)])
def test_wbuf_to_mallat_matches_layout(w, L, h, w_):
    wb = _img(9, 1, h * w_).ravel()
    got = w.wbuf_to_mallat(torch.from_numpy(wb).cuda(), w_, h, L).cpu().numpy()
    assert np.array_equal(got, tile_major_to_mallat(wb, w_, h, L))


@pytest.mark.parametrize("L,n", [(2, 64), (3, 256), (4, 512), (4, 1024), (5, 512)])
def test_inverse_matches_oracle(w, orc, L, n):
    wb = _img(L + 10, 1, n * n).ravel()
    u = w.inverse_haar(torch.from_numpy(wb).cuda(), n, n, L).cpu().numpy()
    ref = orc.haar_inv(tile_major_to_mallat(wb, n, n, L), L)
    assert np.array_equal(u, ref)


@pytest.mark.parametrize("L,h,w_", [(4, 32, 272), (3, 24, 1000), (4, 16, 16), (5, 64, 800)])
def test_inverse_ragged_and_rectangular(w, orc, L, h, w_):
    """Widths that leave a partial strip, single-tile images, w != h."""
    wb = _img(h + w_, 1, h * w_).ravel()
    u, bits = w.inverse_haar(torch.from_numpy(wb).cuda(), w_, h, L, want="both")
    u = u.cpu().numpy()
    # Tiles are independent, so each 2^L x 2^L block of u is the oracle's
    # inverse of that tile's coefficients (a one-tile Mallat image).
    ts, tsl = 1 << L, 1 << (2 * L)
    blocks = wb.reshape(h >> L, w_ >> L, tsl)
    for ty in range(h >> L):
        for tx in range(w_ >> L):
            ref = orc.haar_inv(tile_major_to_mallat(blocks[ty, tx], ts, ts, L), L)
            assert np.array_equal(u[ty * ts:(ty + 1) * ts, tx * ts:(tx + 1) * ts], ref)
    assert np.array_equal(bits.cpu().numpy(), orc.binarize(u))


def test_round_trip(w):
    n, L = 1024, 4
    x = _img(3, n, n)
    wb = w.haar_forward(torch.from_numpy(x).cuda(), L)
    y = w.inverse_haar(wb, n, n, L).cpu().numpy()
    assert np.max(np.abs(y - x)) <= 2 * L * np.finfo(np.float32).eps * 4 * np.max(np.abs(x))


def test_bits_match_oracle(w, orc):
    n, L = 512, 4
    wb = _img(77, 1, n * n).ravel()
    u, bits = w.inverse_haar(torch.from_numpy(wb).cuda(), n, n, L, want="both")
    assert np.array_equal(bits.cpu().numpy(), orc.binarize(u.cpu().numpy()))
    ref = orc.haar_inv(tile_major_to_mallat(wb, n, n, L), L)
    assert np.array_equal(bits.cpu().numpy(), orc.binarize(ref))
