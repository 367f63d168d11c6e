"""The order-1 coiflet (reading R14) on the GPU against the oracle: LUT index
sets and values bit for bit (both sides transform in the same FP32 order),
holograms through wasabi_superpose + wasabi_inverse_wavelet within 1e-5,
keep-all exactness against Eq. (1), bits under both reference waves, and the
fused path refusing a coiflet LUT."""
import os

import numpy as np
import pytest
import torch

from tests._helpers import rel_l2
from workloads import uniform_cloud

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1
LAM, PITCH = 633e-9, 1e-6


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


LUT_CASES = [  # L, W, gamma, depths (m)
    (3, 256, 0.05, [30e-6, 120e-6, -80e-6, 200e-6]),
    (2, 128, 1.0, [20e-6, -50e-6]),
    (4, 512, 0.02, [100e-6, 350e-6, 600e-6]),
]


@pytest.mark.parametrize("case", LUT_CASES)
def test_coiflet_lut_bit_exact(w, orc, case):
    L, W, gamma, zd = case
    lut = w.build_lut(LAM, PITCH, zd, W, L, gamma, wavelet="coif1")
    olut = orc.build_lut(LAM, PITCH, zd, W, L, gamma, wavelet="coif1", threads=min(4, NPROC))
    w.sync_status()
    assert np.array_equal(lut.counts(), olut.nr)
    for d in range(len(zd)):
        oidx, oval = olut.depth(d)
        assert np.array_equal(lut.selection(d), oidx), d
        idx, val = lut.entries(d)
        assert np.array_equal(val[np.argsort(idx)], oval), d
    lut.close()


@pytest.mark.parametrize("rule", [0, 1])
def test_coiflet_hologram_matches_the_oracle(w, orc, rule):
    L, W, gamma, N, D = 3, 256, 0.05, 512, 6
    zmin, zmax = 30e-6, 250e-6
    zd = orc.depth_grid(zmin, zmax, D)
    lut = w.build_lut(LAM, PITCH, zd, W, L, gamma, wavelet="coif1")
    olut = orc.build_lut(LAM, PITCH, zd, W, L, gamma, wavelet="coif1", threads=min(4, NPROC))
    pts = uniform_cloud(71 + rule, 500, N, zmin, zmax)
    pts["d"], _ = orc.quantize(pts["z"], zmin, zmax, D)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    wb = w.superpose(lut, p, N, N, rule=rule)
    u, bits = w.inverse_wavelet(wb, N, N, L, "coif1", want="both")
    w.sync_status()
    ref = orc.hologram(olut, pts, N, rule=rule)
    u_np = u.cpu().numpy()
    assert rel_l2(u_np, ref) <= 1e-5
    mine = np.unpackbits(bits.cpu().numpy(), bitorder="little").reshape(N, N).astype(bool)
    diff = mine != (u_np.real > 0)
    assert np.all(np.abs(u_np.real[diff]) <= 1e-6 * np.abs(u_np).max())
    # The spherical reference under a sub-hologram origin: bits against the
    # oracle's reference binarisation of the same field.
    refd = w.spherical_reference(LAM, PITCH, 40.0, 9000.0, -0.2)
    b2 = w.inverse_wavelet(wb, N, N, L, "coif1", want="bits", origin=(64, 0), reference=refd)
    _, val = orc.binarize_ref(u_np, LAM, PITCH, 40.0, 9000.0, -0.2, 64, 0)
    mine2 = np.unpackbits(b2.cpu().numpy(), bitorder="little").reshape(N, N).astype(bool)
    d2 = mine2 != (val > 0)
    assert np.all(np.abs(val[d2]) <= 1e-5 * np.abs(u_np).max())
    # The fused path is Haar's.
    with pytest.raises(w.WasabiError, match="INVALID"):
        w.hologram(lut, p, N, N, want="bits")
    lut.close()


def test_coiflet_keep_all_aligned_equals_eq1(w, orc):
    L, W, N = 3, 160, 256
    zd = np.array([60e-6, 95e-6])
    lut = w.build_lut(LAM, PITCH, zd, W, L, 1.0, wavelet="coif1")
    rng = np.random.default_rng(4)
    n = 6
    x = (W // 2 + 8 * rng.integers(3, 12, n) - 24).astype(np.int32)
    y = (W // 2 + 8 * rng.integers(3, 12, n) - 24).astype(np.int32)
    d = rng.integers(0, 2, n).astype(np.uint32)
    a = rng.uniform(0.2, 1.0, n).astype(np.float32)
    p = w.pack_points(x, y, a, d)
    u = w.inverse_wavelet(w.superpose(lut, p, N, N), N, N, L, "coif1").cpu().numpy()
    w.sync_status()
    ref = orc.cgh_direct(LAM, PITCH, x, y, a, zd[d], 0, 0, N, N, aperture=True)
    assert rel_l2(u, ref) <= 1e-5
    lut.close()


def test_generic_inverse_with_haar_is_the_haar_inverse(w, orc):
    L, W, N = 4, 128, 256
    zd = orc.depth_grid(20e-6, 150e-6, 4)
    lut = w.build_lut(LAM, PITCH, zd, W, L, 0.1)
    pts = uniform_cloud(5, 200, N, 20e-6, 150e-6)
    pts["d"], _ = orc.quantize(pts["z"], 20e-6, 150e-6, 4)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    wb = w.superpose(lut, p, N, N)
    assert torch.equal(w.inverse_wavelet(wb, N, N, L, "haar"), w.inverse_haar(wb, N, N, L))
    with pytest.raises(w.WasabiError, match="INVALID"):
        w.inverse_wavelet(wb[: 256 * 128], 256, 128, L, "coif1")  # the coiflet inverse is square only
    lut.close()


@pytest.mark.parametrize("N,L", [(8, 3), (40, 3), (96, 2), (160, 5)])
def test_coiflet_inverse_small_and_ragged_regions(w, orc, N, L):
    """The per-level synthesis on regions narrower than a 32-pixel CTA tile
    and not multiples of it (wrap-around of the periodic filters inside one
    tile): field and bits against the oracle's inverse of the same Mallat
    array."""
    g = torch.Generator(device="cuda").manual_seed(N + L)
    wb = torch.randn(N * N, dtype=torch.complex64, device="cuda", generator=g)
    mallat = w.wbuf_to_mallat(wb, N, N, L).cpu().numpy().astype(np.complex128)
    ref = orc.wavelet_inv(mallat, L, "coif1")
    u, bits = w.inverse_wavelet(wb, N, N, L, "coif1", want="both")
    u_np = u.cpu().numpy()
    assert rel_l2(u_np, ref) <= 1e-5
    mine = np.unpackbits(bits.cpu().numpy(), bitorder="little").reshape(N, N).astype(bool)
    diff = mine != (ref.real > 0)
    assert np.all(np.abs(ref.real[diff]) <= 1e-5 * np.abs(ref).max())
