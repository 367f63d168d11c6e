"""Parity at the full measured sizes: the coefficient index sets of every
depth bit-exact, and sampled 512 x 512 sub-holograms (the paper's own
sub-hologram procedure, computed by the oracle one by one) against the GPU
hologram -- within rel-L2 1e-5 and, element by element, within the FP32 /
fixed-point error bound of each pixel (tests/_bounds.py); binarised pixels
may differ only where |Re u| is within that bound of zero.

Two launch configurations per size: the complex field + bits call, and the
bits-only call the benchmark times (real-part accumulation on the widest
super-tile), made exactly as the benchmark makes it.  The C4 precision forms
are measured against the FP64 oracle on the same samples."""
import os

import numpy as np
import pytest
import torch

from tests._bounds import FieldBound, check_bits, check_field
from tests._helpers import rel_l2
from workloads import CONFIGS

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1
NS = 512


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


def _case(w, orc, name):
    c = CONFIGS[name]
    pts = c.points()
    pts["d"], bad = orc.quantize(pts["z"], c.zmin, c.zmax, c.D)
    assert bad == 0
    zd = orc.depth_grid(c.zmin, c.zmax, c.D)
    p = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"])
    return c, pts, zd, p


def _samples(c, k, seed):
    g = np.random.default_rng(seed)
    per = c.Nh // NS
    cells = [(0, 0), (per - 1, per - 1)] + [tuple(int(v) for v in g.integers(0, per, 2)) for _ in range(k)]
    return cells


def _check_selection(w, orc, c, zd, lut):
    olut = orc.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma, threads=NPROC)
    for d in range(c.D):
        assert np.array_equal(lut.selection(d), olut.depth(d)[0]), d
    return olut


def _window_bits(bits, c, s, t):
    rows = bits.view(c.Nh, c.Nh // 8)[t * NS:(t + 1) * NS, s * NS // 8:(s + 1) * NS // 8].cpu().numpy()
    return np.unpackbits(rows, axis=1, bitorder="little").astype(bool)


@pytest.mark.parametrize("name", ["C2", "C3"])
def test_fullsize_sampled_parity(w, orc, name):
    c, pts, zd, p = _case(w, orc, name)
    lut = w.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma)
    olut = _check_selection(w, orc, c, zd, lut)
    fb = FieldBound(orc, olut, pts, c.Nh)
    cells = _samples(c, 2, 3)
    refs = {st: orc.subhologram(olut, pts, NS, *st) for st in cells}
    bounds = {st: fb.window(NS, *st) for st in cells}

    # Complex field and bits in one call (complex accumulation).
    u, bits = w.hologram(lut, p, c.Nh, c.Nh, want="both")
    w.sync_status()
    flips = 0
    for (s, t) in cells:
        ref, bnd = refs[(s, t)], bounds[(s, t)]
        got = u[t * NS:(t + 1) * NS, s * NS:(s + 1) * NS].cpu().numpy()
        assert rel_l2(got, ref) <= 1e-5, (s, t)
        check_field(got, ref, bnd)
        flips += check_bits(_window_bits(bits, c, s, t), ref, bnd)
    del u, bits
    torch.cuda.empty_cache()

    # Bits alone, as the benchmark calls it (real-part accumulation).
    bits = w.hologram(lut, p, c.Nh, c.Nh, want="bits")
    w.sync_status()
    flips_re = 0
    for (s, t) in cells:
        flips_re += check_bits(_window_bits(bits, c, s, t), refs[(s, t)], bounds[(s, t)])
    n = len(cells) * NS * NS
    print(f"{name}: sampled bit flips {flips} (complex accumulation), {flips_re} (bits alone) of {n}")
    del bits
    lut.close()


def test_c4_precision_forms_vs_fp64(w, orc):
    c, pts, zd, p = _case(w, orc, "C4")
    o64 = orc.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma, dtype="f64", threads=NPROC, select_fp32=True)
    cells = _samples(c, 1, 4)
    refs = [orc.subhologram(o64, pts, NS, s, t) for s, t in cells]
    errs = {}
    for dt in ("f32", "f16s", "bf16s"):
        lut = w.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma, dtype=dt)
        u = w.hologram(lut, p, c.Nh, c.Nh)
        num = den = 0.0
        for (s, t), ref in zip(cells, refs):
            got = u[t * NS:(t + 1) * NS, s * NS:(s + 1) * NS].cpu().numpy().astype(np.complex128)
            num += float(np.sum(np.abs(got - ref) ** 2))
            den += float(np.sum(np.abs(ref) ** 2))
        errs[dt] = (num / den) ** 0.5
        lut.close()
    w.sync_status()
    print("C4 rel-L2 vs FP64 oracle (sampled sub-holograms):", errs)
    assert errs["f32"] <= 1e-5
    assert errs["f16s"] <= 2e-3
    assert errs["bf16s"] <= 2e-2
