"""The serving loop: results are the same alone and in a mix of concurrent
requests, admission respects the device-memory budget, and served results
match the one-hologram call and the oracle."""
import numpy as np
import pytest
import torch

from tests._helpers import rel_l2
from workloads import heightfield_cloud

pytestmark = pytest.mark.gpu
LAM, PITCH, ZMIN, ZMAX, D, W, L, GAMMA = 532e-9, 1e-6, 0.1e-3, 0.4e-3, 16, 256, 4, 0.05


@pytest.fixture(scope="module")
def setup(orc):
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    zd = w.depth_grid(ZMIN, ZMAX, D)
    lut = w.build_lut(LAM, PITCH, zd, W, L, GAMMA)
    return w, lut, zd


def _job(w, orc, seed, n, side):
    pts = heightfield_cloud(seed, n, side, ZMIN, ZMAX)
    pts["d"], _ = orc.quantize(pts["z"], ZMIN, ZMAX, D)
    host = w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"], device="cpu").pin_memory()
    return pts, host


SPECS = [(11, 2000, 512), (12, 300, 256), (13, 5000, 1024), (14, 0, 256), (15, 1200, 768), (16, 800, 512),
         (17, 4000, 1024), (18, 50, 256), (19, 2500, 512), (20, 700, 384)]


def test_same_result_alone_and_in_mix(setup, orc):
    w, lut, zd = setup
    jobs = [_job(w, orc, *s) for s in SPECS]
    _, heavy = _job(w, orc, 99, 200_000, 8192)
    srv = w.Server(lut, 1 << 30, streams=1, max_batch=4, side_hint=512)
    alone = []
    for (_, host), s in zip(jobs, SPECS):
        rid = srv.submit(host, s[2], s[2], want="both")
        alone.append(srv.wait(rid, timeout=60))
        assert alone[-1]["batch_jobs"] == 1
    # A long request first: the others queue behind it and share launches.
    hid = srv.submit(heavy, 8192, 8192, want="bits")
    ids = [srv.submit(host, s[2], s[2], want="both") for (_, host), s in zip(jobs, SPECS)]
    mixed = [srv.wait(i, timeout=60) for i in ids]
    srv.wait(hid, timeout=60)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 2 * len(SPECS) + 1
    assert max(m["batch_jobs"] for m in mixed) > 1
    for a, m in zip(alone, mixed):
        assert torch.equal(a["u"], m["u"]) and torch.equal(a["bits"], m["bits"])
    # Several streams: launches overlap on the device; the same results.
    srv = w.Server(lut, 1 << 30, streams=3, max_batch=4, side_hint=512)
    ids = [srv.submit(host, s[2], s[2], want="both") for (_, host), s in zip(jobs, SPECS)]
    for a, i in zip(alone, ids):
        m = srv.wait(i, timeout=60)
        assert torch.equal(a["u"], m["u"]) and torch.equal(a["bits"], m["bits"])
    srv.close()
    # Served results against the one-hologram call and the oracle.
    for (pts, host), s, a in zip(jobs, SPECS, alone):
        u1 = w.hologram(lut, host.cuda(), s[2], s[2]).cpu()
        assert rel_l2(a["u"].numpy(), u1.numpy()) <= 1e-5
    olut = orc.build_lut(LAM, PITCH, zd, W, L, GAMMA)
    pts, _ = jobs[1]
    assert rel_l2(alone[1]["u"].numpy(), orc.hologram(olut, pts, SPECS[1][2])) <= 1e-5
    w.sync_status()


def test_admission_by_memory_budget(setup, orc):
    w, lut, _ = setup
    jobs = [_job(w, orc, 30 + i, 1500, 1024) for i in range(8)]
    # One 1024^2 request holds 8 MiB of complex output + 128 KiB of bits +
    # points + binning scratch: a 20 MiB budget admits two at a time.
    budget = 20 << 20
    srv = w.Server(lut, budget, streams=4, max_batch=8, side_hint=1024)
    ids = [srv.submit(h, 1024, 1024, want="both") for _, h in jobs]
    res = [srv.wait(i, timeout=120) for i in ids]
    st = srv.stats()
    assert st["peak_bytes"] <= budget and st["launches"] >= 4
    assert max(r["batch_jobs"] for r in res) <= 2
    # Alone, through a roomy server: the same result.
    big = w.Server(lut, 1 << 30, streams=1, max_batch=1, side_hint=1024)
    for (_, h), r in zip(jobs[:3], res[:3]):
        a = big.wait(big.submit(h, 1024, 1024, want="both"), timeout=60)
        assert torch.equal(a["u"], r["u"]) and torch.equal(a["bits"], r["bits"])
    big.close()
    srv.close()


def test_requests_refused(setup, orc):
    w, lut, _ = setup
    srv = w.Server(lut, 4 << 20, streams=1, max_batch=2)
    _, h = _job(w, orc, 40, 100, 256)
    with pytest.raises(w.WasabiError, match="NOMEM"):
        srv.submit(h, 2048, 2048, want="complex")   # 32 MiB of output alone
    with pytest.raises(w.WasabiError, match="INVALID"):
        srv.submit(h, 250, 256)
    bad = h.clone()
    bad[3, 3] = D
    with pytest.raises(w.WasabiError, match="RANGE"):
        srv.submit(bad, 256, 256)
    r = srv.wait(srv.submit(h, 256, 256), timeout=30)
    assert r["bits"] is not None and r["latency_s"] >= 0
    srv.close()


def test_bits_only_requests_match_the_one_hologram_call(setup, orc):
    w, lut, _ = setup
    srv = w.Server(lut, 1 << 28, streams=2, max_batch=8, side_hint=512)
    jobs = [_job(w, orc, *s) for s in SPECS[:6]]
    ids = [srv.submit(h, s[2], s[2], want="bits") for (_, h), s in zip(jobs, SPECS[:6])]
    for (_, h), s, i in zip(jobs, SPECS[:6], ids):
        r = srv.wait(i, timeout=60)
        ref = w.hologram(lut, h.cuda(), s[2], s[2], want="bits").cpu()
        assert torch.equal(r["bits"], ref)
    srv.close()
