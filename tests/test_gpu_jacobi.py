"""dm_jacobi_refine: the modified Jacobi refinement of Appendix A on the
device, a <- a + W~(P g(a)), against the oracle's jacobi_refine (the same
solve at the same per-level counts, then the same refinement steps), element
by element: FP64-class modes at the FP64 bar, the mixed mode at its bar.  The
refinement must also lower the true residual the stats report."""
import numpy as np
import pytest

import workloads as W
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


@pytest.mark.parametrize("prec,B,bar", [(dmwf.DM_FP64, 2, 1e-10), (dmwf.DM_FLOAT_FLOAT, 2, 1e-10),
                                         (dmwf.DM_MIXED_FP32, 8, 1e-5)])
def test_jacobi_refine_matches_oracle(orc, prec, B, bar):
    wl = W.make_workload("nside16", list(range(10, 10 + B)))
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 3)
    counts = [6, 6, 6]
    p = make_plan(wl, B, lambda0=1000.0, n_levels=3, iters_per_level=6, check_every=4)
    p.set_precision(prec)
    if prec == dmwf.DM_MIXED_FP32:
        p.set_refinement(8)
    s = torch.zeros((B, 3, wl.npix), dtype=torch.float64, device="cuda")
    a = torch.zeros((B, 3, (wl.lmax + 1) * (wl.lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    st, base = p.wiener_filter(dev(d), s)
    st, stats = p.jacobi_refine(dev(d), 2, s, a)
    gs, ga = s.cpu().numpy(), alm_host(a, (B, 3, -1))
    p.close()
    for b in [0, B - 1]:
        assert stats[b]["iters_total"] == 3 * sum(counts)
        assert stats[b]["true_resid"] < 0.5 * base[b]["true_resid"]
        ref = orc.jacobi_refine(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=counts,
                                n_refine=2)
        assert rel(ga[b], ref["alm"]) < bar, b
        assert rel(gs[b], ref["s"]) < bar, b


def test_jacobi_refine_rejects_correlated_noise_and_sessions(orc):
    wl = W.make_cov_workload([50], 8, 16)
    p = dmwf.Plan(8, 16, 1)
    p.set_spectra(wl.cl)
    p.set_noise_cov(wl.sigma, wl.rho, wl.mask, wl.mask_p)
    d = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    with pytest.raises(dmwf.DmError) as ei:
        p.jacobi_refine(d, 1, torch.zeros_like(d))
    assert ei.value.status == dmwf.DM_EINVAL
    p.set_noise_mask(wl.sigma, wl.mask)
    p.set_schedule(lambda0=10.0, n_levels=2, iters_per_level=2)
    p.solve_begin(d)
    with pytest.raises(dmwf.DmError) as ei:
        p.jacobi_refine(d, 1, torch.zeros_like(d))
    assert ei.value.status == dmwf.DM_EBUSY
    p.solve_iterate(4)
    p.solve_end()
    p.close()
