"""Batched launches (many holograms, one launch sequence, graph replay) and
the autotuner, against the one-job calls and the oracle."""
import numpy as np
import pytest
import torch

from tests._helpers import rel_l2, tile_major_to_mallat
from workloads import uniform_cloud

pytestmark = pytest.mark.gpu
TOL = 1e-5
LAM, PITCH, ZMIN, ZMAX, D, W, L, GAMMA = 633e-9, 1e-6, 20e-6, 150e-6, 6, 128, 4, 0.1


@pytest.fixture(scope="module")
def setup(orc):
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    zd = w.depth_grid(ZMIN, ZMAX, D)
    lut = w.build_lut(LAM, PITCH, zd, W, L, GAMMA)
    olut = orc.build_lut(LAM, PITCH, zd, W, L, GAMMA)
    return w, lut, olut


def _job(w, orc, seed, N, side, want, rule=0):
    pts = uniform_cloud(seed, N, side, ZMIN, ZMAX)
    pts["d"], _ = orc.quantize(pts["z"], ZMIN, ZMAX, D)
    return pts, {"points": w.pack_points(pts["x"], pts["y"], pts["a"], pts["d"]), "w": side,
                 "h": side, "rule": rule, "want": want}


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_single_calls(setup, orc, use_graph):
    w, lut, olut = setup
    specs = [(1, 50, 256, "bits", 0), (2, 300, 512, "complex", 1), (3, 0, 128, "both", 0),
             (4, 120, 1024, "none", 0), (5, 80, 384, "both", 1)]
    made = [_job(w, orc, *s) for s in specs]
    batch = w.Batch(lut, 8, side_hint=512, use_graph=use_graph)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        res = batch.run([dict(j, keep_wbuf=True) for _, j in made], stream=stream)
    stream.synchronize()
    w.sync_status(stream)
    for (pts, j), r in zip(made, res):
        single = w.superpose(lut, j["points"], j["w"], j["h"], rule=j["rule"])
        assert rel_l2(r["wbuf"].cpu().numpy(), single.cpu().numpy()) <= TOL
        u_ref = w.inverse_haar(single, j["w"], j["h"], L, want="both")
        if r["u"] is not None:
            assert rel_l2(r["u"].cpu().numpy(), u_ref[0].cpu().numpy()) <= TOL
        if r["bits"] is not None:
            diff = np.unpackbits(r["bits"].cpu().numpy() ^ u_ref[1].cpu().numpy()).sum()
            assert diff <= 2   # flips only where Re u is within rounding of 0
    # One job against the oracle.
    pts, j = made[1]
    psi = orc.superpose(olut, pts, 512, rule=1)
    assert rel_l2(tile_major_to_mallat(res[1]["wbuf"].cpu().numpy(), 512, 512, L), psi) <= TOL
    batch.close()


def test_graph_replay_with_a_new_job_mix(setup, orc):
    w, lut, _ = setup
    batch = w.Batch(lut, 6, side_hint=512, use_graph=True)
    stream = torch.cuda.Stream()
    for round_, specs in enumerate([[(7, 200, 512, "bits", 0), (8, 10, 256, "complex", 0)],
                                    [(9, 40, 256, "complex", 1), (10, 400, 768, "both", 0),
                                     (11, 90, 512, "bits", 0)]]):
        made = [_job(w, orc, *s) for s in specs]
        with torch.cuda.stream(stream):
            res = batch.run([dict(j, keep_wbuf=True) for _, j in made], stream=stream)
        stream.synchronize()
        w.sync_status(stream)
        for (_, j), r in zip(made, res):
            single = w.superpose(lut, j["points"], j["w"], j["h"], rule=j["rule"])
            assert rel_l2(r["wbuf"].cpu().numpy(), single.cpu().numpy()) <= TOL, f"round {round_}"
    batch.close()


def test_batch_rejects_bad_jobs(setup, orc):
    w, lut, _ = setup
    batch = w.Batch(lut, 2, use_graph=False)
    _, j = _job(w, orc, 1, 10, 256, "bits")
    with pytest.raises(w.WasabiError, match="INVALID"):
        batch.run([dict(j, w=250)])
    with pytest.raises(w.WasabiError, match="INVALID"):
        batch.run([j, j, j])  # over capacity
    batch.close()


def test_autotune_picks_a_valid_configuration(setup, orc):
    w, lut, _ = setup
    cell, threads = w.autotune(lut, 512, 2000)
    assert cell in (64, 128, 192, 256) and threads in (256, 384, 512, 1024)
    _, j = _job(w, orc, 12, 300, 512, "none")
    a = w.superpose(lut, j["points"], 512, 512).cpu().numpy()
    b = w.Batch(lut, 1, side_hint=512, use_graph=False)
    assert b.config() == (cell, threads)
    r = b.run([j])
    torch.cuda.synchronize()
    assert rel_l2(r[0]["wbuf"].cpu().numpy(), a) <= TOL
    b.close()


def test_bits_only_batch_uses_real_accumulation_and_matches(setup, orc):
    """A batch whose jobs all want bits alone accumulates real parts only (its
    own graph); the bits equal the one-hologram call's, across a replay with a
    new mix and after a complex batch on the same stream."""
    w, _, _ = setup
    # A LUT of its own: no autotuned entry, so every call here uses the
    # default super-tile and the fixed-point results agree exactly.
    lut = w.build_lut(LAM, PITCH, w.depth_grid(ZMIN, ZMAX, D), W, L, GAMMA)
    batch = w.Batch(lut, 6, side_hint=512, use_graph=True)
    stream = torch.cuda.Stream()
    for specs in ([(21, 300, 512, "bits", 0), (22, 40, 256, "bits", 1), (23, 0, 128, "bits", 0)],
                  [(24, 250, 384, "both", 0)],
                  [(25, 500, 768, "bits", 1), (26, 90, 512, "bits", 0)]):
        made = [_job(w, orc, *s) for s in specs]
        with torch.cuda.stream(stream):
            res = batch.run([j for _, j in made], stream=stream)
        stream.synchronize()
        w.sync_status(stream)
        for (_, j), r in zip(made, res):
            ref = w.hologram(lut, j["points"], j["w"], j["h"], want="bits", rule=j["rule"])
            assert torch.equal(r["bits"], ref)
    batch.close()
    lut.close()
