"""Numerical reconstruction on the GPU (wasabi_reconstruct: angular spectrum
method, cuFFT) against the oracle's FP64 numpy form (reading R13): complex
fields, binary holograms under the plane and the spherical reference wave,
and a WASABI hologram of a point refocused at d = -z."""
import numpy as np
import pytest
import torch

from tests._helpers import rel_l2

pytestmark = pytest.mark.gpu
LAM, PITCH = 633e-9, 1e-6


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


# 20 mm: about 3.2e4 cycles of phase, far beyond what FP32 alone carries.
@pytest.mark.parametrize("h,wd,d", [(256, 384, -0.5e-3), (200, 136, 1.2e-3), (512, 512, 0.0), (128, 160, 20e-3)])
def test_field_reconstruction_matches_the_oracle(w, orc, h, wd, d):
    rng = np.random.default_rng(h + wd)
    u0 = (rng.normal(size=(h, wd)) + 1j * rng.normal(size=(h, wd))).astype(np.complex64)
    t = torch.from_numpy(u0).cuda()
    ref = orc.reconstruct(u0, LAM, PITCH, d)
    got = w.reconstruct(t, wd, h, LAM, PITCH, d, want="complex").cpu().numpy()
    assert rel_l2(got, ref) <= 1e-5
    inten = w.reconstruct(t, wd, h, LAM, PITCH, d).cpu().numpy()
    assert rel_l2(inten, np.abs(ref) ** 2) <= 2e-5


@pytest.mark.parametrize("spherical", [False, True])
def test_bits_reconstruction_under_the_reference(w, orc, spherical):
    h, wd, origin = 256, 320, (96, -40)
    rng = np.random.default_rng(7)
    bits = rng.integers(0, 256, size=h * wd // 8, dtype=np.uint8)
    refd = w.spherical_reference(LAM, PITCH, 150.0, 30000.0, -0.4) if spherical else None
    got = w.reconstruct(torch.from_numpy(bits).cuda(), wd, h, LAM, PITCH, -0.3e-3, want="complex",
                        origin=origin, reference=refd).cpu().numpy()
    R = (orc.reference_wave(LAM, PITCH, 150.0, 30000.0, -0.4, wd, h, *origin) if spherical
         else np.ones((h, wd)))
    ref = orc.reconstruct(orc.transmittance(bits, wd, h) * R, LAM, PITCH, -0.3e-3)
    assert rel_l2(got, ref) <= 1e-5


def test_wasabi_point_refocuses(w, orc):
    """A keep-all WASABI hologram of one point refocuses to the point's
    pixel at d = -z."""
    zd = orc.depth_grid(0.3e-3, 0.5e-3, 1)
    lut = w.build_lut(LAM, PITCH, zd, 512, 3, 1.0)
    p = w.pack_points([200], [180], [1.0], [0])
    u = w.hologram(lut, p, 384, 384, want="complex")
    inten = w.reconstruct(u, 384, 384, LAM, PITCH, -float(zd[0])).cpu().numpy()
    w.sync_status()
    assert np.unravel_index(np.argmax(inten), inten.shape) == (180, 200)
    lut.close()


def test_bad_arguments_are_refused(w):
    t = torch.zeros((64, 60), dtype=torch.uint8, device="cuda").view(-1)[: 64 * 60 // 8]
    with pytest.raises(w.WasabiError, match="INVALID"):
        w.reconstruct(t, 60, 64, LAM, PITCH, 1e-3)  # bits need w % 8 == 0
    f = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(w.WasabiError, match="INVALID"):
        w.reconstruct(f, 64, 64, -LAM, PITCH, 1e-3)


def test_plan_cache_shapes_and_streams(w, orc):
    """More shapes than the plan cache holds (the later ones get a plan per
    call), then a cached shape again on a side stream: every result matches
    the oracle."""
    rng = np.random.default_rng(11)
    fields = []
    for i in range(10):
        h, wd = 32 + 8 * i, 40
        u0 = (rng.normal(size=(h, wd)) + 1j * rng.normal(size=(h, wd))).astype(np.complex64)
        got = w.reconstruct(torch.from_numpy(u0).cuda(), wd, h, LAM, PITCH, 0.2e-3, want="complex")
        assert rel_l2(got.cpu().numpy(), orc.reconstruct(u0, LAM, PITCH, 0.2e-3)) <= 1e-5
        fields.append(u0)
    side = torch.cuda.Stream()
    u0 = fields[0]
    src = torch.from_numpy(u0).cuda()
    side.wait_stream(torch.cuda.current_stream())
    got = w.reconstruct(src, 40, 32, LAM, PITCH, -0.1e-3, want="complex", stream=side)
    side.synchronize()
    assert rel_l2(got.cpu().numpy(), orc.reconstruct(u0, LAM, PITCH, -0.1e-3)) <= 1e-5
