"""The FP64-class analysis with fewer partial-sum slots than pair chunks
(dm_set_analysis_slots): the chunks of 64 ring pairs run in waves, slot 0
keeping the running sum.  Against the oracle through the C ABI, at nside 128
(4 chunks) and nside 256 (8 chunks) with 2 and 3 slots: the FP64 and
float-float map2alm (with and without per-slab float-float tables), and a
mixed solve whose float-float anchors run in waves.  Bars: 1e-12 for the
FP64-class transforms, 1e-10 for the FP64 solve, 1e-5 for the mixed one."""
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


@pytest.mark.parametrize("nside,slots,prec,slab", [(128, 2, "fp64", 0), (128, 3, "ff", 0), (256, 3, "ff", 300_000),
                                                   (256, 2, "fp64", 0)])
def test_map2alm_in_waves(orc, nside, slots, prec, slab):
    lmax, B = 2 * nside, 2
    maps = W.random_maps(nside, B, 71)
    p = dmwf.Plan(nside, lmax, B)
    if prec == "ff":
        p.set_precision(dmwf.DM_FLOAT_FLOAT)
    if slab:
        p.set_ff_slab_bytes(slab)
    p.set_analysis_slots(slots)
    a_out = torch.zeros((B, 3, (lmax + 1) * (lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    p.map2alm(dev(maps), a_out)
    ga = a_out.cpu().numpy().view(np.complex128)[..., 0]
    p.close()
    for b in range(B):
        assert rel(ga[b], orc.map2alm(nside, lmax, maps[b])) < 1e-12


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_solve_in_waves(orc, prec, bar):
    wl = W.make_workload("nside16", [7, 8], nside=128, lmax=256)
    d = np.stack([wl.data([orc.alm2map(wl.nside, wl.lmax, a)])[0] for a in wl.alm_true])
    lam = W.lambda_schedule(1000.0, 2)
    p = make_plan(wl, 2, lambda0=1000.0, n_levels=2, iters_per_level=2, check_every=8)
    if prec == "mixed":
        p.set_precision(dmwf.DM_MIXED_FP32)
        p.set_anchor_precision(dmwf.DM_FLOAT_FLOAT)
        p.set_refinement(2)
    p.set_analysis_slots(3)
    s = torch.zeros((2, 3, wl.npix), dtype=torch.float64, device="cuda")
    p.wiener_filter(dev(d), s)
    got = s.cpu().numpy()
    p.close()
    for b in range(2):
        ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=[2, 2])
        assert rel(got[b], ref["s"]) < bar
