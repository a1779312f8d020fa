"""The tensor-core pipeline's bounded waits end a stuck solve with
DM_ETIMEOUT and leave the plan and the CUDA context usable (the failure
detection of the batched path, tested without faulting the GPU).

dm_test_tc_withhold makes one converter thread of the spin-0 analysis withhold
a plain arrival on a stage barrier that no copy or MMA targets; the MMA warp's
wait gives up after 1 s, the CTA drains its copies and frees its tensor memory.
The solve must report DM_ETIMEOUT; with the hook off the same plan must then
give the oracle's transform and solve."""
import time

import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import alm_dev, dev, make_plan, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_05358_gb300 import dmwf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_withheld_arrival_times_out_and_the_plan_recovers(orc):
    B = 8
    wl = W.make_workload("nside16", list(range(B)))
    d = np.stack([wl.data([orc.alm2map(wl.nside, wl.lmax, a)])[0] for a in wl.alm_true])
    p = make_plan(wl, B, lambda0=100.0, n_levels=2, iters_per_level=2, check_every=1)
    p.set_precision(dmwf.DM_MIXED_FP32)
    s = torch.zeros((B, 3, wl.npix), dtype=torch.float64, device="cuda")
    p.test_tc_withhold(True)
    t0 = time.perf_counter()
    with pytest.raises(dmwf.DmError) as ei:
        p.wiener_filter(dev(d), s)
    assert ei.value.status == dmwf.DM_ETIMEOUT
    assert time.perf_counter() - t0 >= 0.9  # the wait ran to its limit
    torch.cuda.synchronize()  # the context is intact
    p.test_tc_withhold(False)
    alm = W.random_alm(wl.lmax, B, 5)
    m = torch.zeros_like(s)
    p.alm2map(alm_dev(alm), m)
    torch.cuda.synchronize()
    assert rel(m.cpu().numpy()[0], orc.alm2map(wl.nside, wl.lmax, alm[0])) < 2e-5
    st, stats = p.wiener_filter(dev(d), s)
    lam = W.lambda_schedule(100.0, 2)
    ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[0], lam, forced_iters=[2, 2])
    assert rel(s.cpu().numpy()[0], ref["s"]) < 1e-5
    p.close()
