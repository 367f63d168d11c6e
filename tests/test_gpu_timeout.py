"""Failure detection without a GPU fault: a bounded stage wait of the
inverse kernel that runs out (its bulk copy is never issued, so nothing
completes the mbarrier) makes the call report WASABI_E_TIMEOUT through the
status word, and the context stays usable for the next call."""
import numpy as np
import pytest
import torch

from tests._helpers import rel_l2, tile_major_to_mallat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    from paper_1708_04233_gb300 import build
    build.build()
    import paper_1708_04233_gb300 as w
    torch.cuda.set_device(0)
    return w


def test_stage_wait_runs_out_then_normal_call_passes(w, orc):
    Nh, L = 1024, 4
    g = np.random.default_rng(5)
    wb = (g.standard_normal(Nh * Nh) + 1j * g.standard_normal(Nh * Nh)).astype(np.complex64)
    wbuf = torch.from_numpy(wb).cuda()
    w.sync_status()
    from paper_1708_04233_gb300 import api
    api.inverse_stall_for_test(wbuf, Nh, Nh, L, skip_strip=1, wait_cycles=2_000_000)
    with pytest.raises(w.WasabiError, match="TIMEOUT"):
        w.sync_status()
    w.sync_status()  # cleared
    u = w.inverse_haar(wbuf, Nh, Nh, L).cpu().numpy()
    w.sync_status()
    ref = orc.haar_inv(tile_major_to_mallat(wb, Nh, Nh, L), L)
    assert rel_l2(u, ref) <= 1e-6
    # The stall entry rejects an unbounded or negative request before any launch.
    with pytest.raises(w.WasabiError, match="INVALID"):
        api.inverse_stall_for_test(wbuf, Nh, Nh, L, skip_strip=1, wait_cycles=0)
