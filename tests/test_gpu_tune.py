"""dm_autotune: the launch autotuner of the batched iteration.  It picks, per
ring-size class, the radix and lanes per block of the ring kernel, and the
pipeline depth and l tiles of the tensor-core Legendre kernels, by timing
them on the plan; the picks must be valid launch configurations, leave every
result within its precision's bar of the oracle (the configuration changes
rounding only), come from the process cache for a second plan of the same
kind, and survive a get/set round trip."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import dev, make_plan, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_05358_gb300 import dmwf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _data(orc, wl):
    return np.stack([wl.data([orc.alm2map(wl.nside, wl.lmax, a)])[0] for a in wl.alm_true])


@pytest.mark.parametrize("prec,B,bar", [(dmwf.DM_MIXED_FP32, 8, 1e-5), (dmwf.DM_FP64, 2, 1e-10)])
def test_autotuned_plan_matches_oracle(orc, prec, B, bar):
    wl = W.make_workload("nside16", list(range(B)), nside=128, lmax=256)
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 3)
    p = make_plan(wl, B, lambda0=1000.0, n_levels=3, iters_per_level=3, check_every=4)
    p.set_precision(prec)
    t = p.autotune(force=True)
    n = t["n_ring_classes"]
    assert n >= 2 and len(t["ring_lanes"]) == n
    assert all(1 <= g <= 16 for g in t["ring_lanes"]) and all(lr in (0, 3, 4) for lr in t["ring_radix_lr"])
    assert 0 < t["ms_ring"] <= t["ms_ring_default"] + 1e-6
    if prec == dmwf.DM_MIXED_FP32:
        assert all(2 <= s <= 8 for s in t["syn_stages"]) and all(1 <= x <= 4 for x in t["ana_ltiles"])
        assert all(2 <= s <= 4 for s in t["ana_stages"])
        assert 0 < t["ms_synthesis"] <= t["ms_synthesis_default"] + 1e-6
        assert 0 < t["ms_analysis"] <= t["ms_analysis_default"] + 1e-6
    s = torch.zeros((B, 3, wl.npix), dtype=torch.float64, device="cuda")
    p.wiener_filter(dev(d), s)
    got = s.cpu().numpy()
    for b in [0, B - 1]:
        ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=[3, 3, 3])
        assert rel(got[b], ref["s"]) < bar
    # a second plan of the same kind takes the cached picks without measuring
    q = make_plan(wl, B)
    q.set_precision(prec)
    t2 = q.autotune()
    assert t2["from_cache"] == 1 and t2["ring_lanes"] == t["ring_lanes"]
    # round trip through get / set
    r = make_plan(wl, B)
    r.set_precision(prec)
    r.set_tuning(t)
    t3 = r.tuning()
    assert t3["ring_lanes"] == t["ring_lanes"] and t3["ring_radix_lr"] == t["ring_radix_lr"]
    assert t3["syn_stages"] == t["syn_stages"] and t3["ana_ltiles"] == t["ana_ltiles"]
    for x in (p, q, r):
        x.close()


def test_autotune_refused_during_a_solve(orc):
    wl = W.make_workload("nside16", [0])
    d = _data(orc, wl)
    p = make_plan(wl, 1, lambda0=10.0, n_levels=2, iters_per_level=2)
    p.solve_begin(dev(d))
    with pytest.raises(dmwf.DmError) as ei:
        p.autotune()
    assert ei.value.status == dmwf.DM_EBUSY
    p.solve_iterate(4)
    p.solve_end()
    p.close()
