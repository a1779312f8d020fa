"""The end-of-solve diagnostics in dm_stats against the oracle's definitions
(Section 3.2, Table 1; Appendix C): the true residual ||A x - y|| / ||y||
(orc_wf_residual) and chi^2 of Eq. 3 (orc_chi2), each evaluated by the
oracle on its own solve of the same data at the same per-level counts, and
by the library on the device on its final iterate.

Bars: FP64 solves 1e-10 (chi^2 relative, residual absolute: it is itself a
ratio); mixed solves 1e-5 (the mixed-mode map bound)."""
import math

import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import dev, make_plan

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


@pytest.mark.parametrize("prec,B,bar", [(dmwf.DM_FP64, 2, 1e-10), (dmwf.DM_FLOAT_FLOAT, 2, 1e-10),
                                         (dmwf.DM_MIXED_FP32, 8, 1e-5)])
def test_diagnostics_match_oracle(orc, prec, B, bar):
    wl = W.make_workload("nside16", list(range(B)))
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 10)
    p = make_plan(wl, B, lambda0=1000.0, n_levels=10, iters_per_level=10, check_every=16)
    p.set_precision(prec)
    s = torch.zeros((B, 3, wl.npix), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s)
    for b in [0, B - 1]:
        ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=[10] * 10)
        r_ref = orc.wf_residual(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], ref["alm"])
        c_ref = orc.chi2(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], ref["s"], ref["alm"])
        assert 1e-4 < r_ref < 1.0  # 100 iterations: far from converged, well away from zero
        assert abs(stats[b]["true_resid"] - r_ref) < bar, (b, stats[b]["true_resid"], r_ref)
        assert abs(stats[b]["chi2"] - c_ref) < bar * c_ref, (b, stats[b]["chi2"], c_ref)
        assert stats[b]["ms_total"] > 0.0
    p.close()


def test_diagnostics_of_session_and_constrained_realisation(orc):
    """dm_solve_end reports them too; a constrained realisation reports those
    of its Wiener-filter solve W(d - dhat); switched off they are NaN."""
    wl = W.make_workload("nside16", [3])
    d = _data(orc, wl)
    lam = W.lambda_schedule(100.0, 3)
    p = make_plan(wl, 1, lambda0=100.0, n_levels=3, iters_per_level=4)
    p.solve_begin(dev(d))
    p.solve_iterate(12)
    st, stats = p.solve_end()
    ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[0], lam, forced_iters=[4, 4, 4])
    assert abs(stats[0]["true_resid"] - orc.wf_residual(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[0],
                                                        ref["alm"])) < 1e-10
    seed = 77
    s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    st, stats = p.constrained_realization(dev(d), [seed], s)
    cr = orc.constrained_realization(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[0], seed, lam,
                                     forced_iters=[4, 4, 4])
    dd = d[0] - cr["dhat"]
    r_ref = orc.wf_residual(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, dd, cr["alm"])
    c_ref = orc.chi2(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, dd, cr["s"], cr["alm"])
    assert abs(stats[0]["true_resid"] - r_ref) < 1e-10
    assert abs(stats[0]["chi2"] - c_ref) < 1e-10 * c_ref
    p.set_diagnostics(False)
    st, stats = p.wiener_filter(dev(d), s)
    assert math.isnan(stats[0]["true_resid"]) and math.isnan(stats[0]["chi2"])
    assert stats[0]["ms_total"] > 0.0
    p.close()
