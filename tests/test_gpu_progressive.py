"""Progressive working resolution (dm_set_progressive; the paper's Section 4
proposal, l_iter of Section 2) against the oracle's dm_solve_progressive:
each level's (nside_k, L_k), and the final map and coefficients element by
element at the oracle's per-level counts (FP64 bar 1e-10; mixed 1e-5), and
the free-running Cauchy schedule's per-level counts."""
import numpy as np
import pytest

import workloads as W
from oracle import progressive as P
from tests.gpu_helpers import alm_host, dev, make_plan, rel

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


@pytest.mark.parametrize("prec,B,bar", [(dmwf.DM_FP64, 2, 1e-10), (dmwf.DM_MIXED_FP32, 8, 1e-5)])
def test_progressive_forced_matches_oracle(orc, prec, B, bar):
    wl = W.make_workload("nside16", list(range(20, 20 + B)), nside=32, lmax=64)
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 4)
    counts = [3, 3, 3, 3]
    p = make_plan(wl, B, lambda0=1000.0, n_levels=4, iters_per_level=3, check_every=4)
    p.set_precision(prec)
    p.set_progressive(0.25, 8)
    s = torch.zeros((B, 3, wl.npix), dtype=torch.float64, device="cuda")
    a = torch.zeros((B, 3, p.nalm, 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s, a)
    levels = p.progressive_levels(4)
    gs, ga = s.cpu().numpy(), alm_host(a, (B, 3, -1))
    p.close()
    for b in [0, B - 1]:
        ref = P.dm_solve_progressive(32, 64, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=counts, margin=0.25,
                                     lmin=8)
        assert levels == [tuple(x) for x in ref["levels"]]
        assert levels[0][0] < 32  # the first level really runs coarse
        assert stats[b]["iters_per_level"][:4] == counts and stats[b]["iters_total"] == 12
        assert rel(gs[b], ref["s"]) < bar
        assert rel(ga[b], ref["alm"]) < bar


def test_progressive_cauchy_counts_match_oracle(orc):
    wl = W.make_workload("nside16", [31], nside=32, lmax=64)
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 3)
    eps = W.eps_schedule(3, 1e-3, 1e-5)
    p = make_plan(wl, 1, lambda0=1000.0, n_levels=3, iters_per_level=0, eps0=1e-3, eps_final=1e-5, eta=0.0,
                  check_every=1)
    p.set_progressive(0.25, 8)
    s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s)
    p.close()
    ref = P.dm_solve_progressive(32, 64, wl.cl, wl.sigma, wl.mask, d[0], lam, eps=eps, margin=0.25, lmin=8)
    assert list(stats[0]["iters_per_level"][:3]) == list(ref["iters_per_level"])
    assert rel(s.cpu().numpy()[0], ref["s"]) < 1e-10
