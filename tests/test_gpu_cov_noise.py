"""Correlated 3x3 per-pixel noise with distinct temperature and polarisation
masks (dm_set_noise_cov; Section 2.1 and Appendix B) against the oracle's
orc_dm_solve_cov, through the C ABI: FP64 and float-float solves at the FP64
bar (relative L2 <= 1e-10) and mixed solves (FP32 ring stage with the 3x3
weights per pixel, FP64-class anchors every few iterations) at the mixed bar
1e-5, on the CUDA-core and the tensor-core Legendre stages; batches, the
free-running Cauchy schedule, constrained realisations (their conditional
noise draws, Eq. 18 and 19) and the calls the mode rejects."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import alm_host, dev, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_05358_gb300 import dmwf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _plan(wl, B, **sched):
    p = dmwf.Plan(wl.nside, wl.lmax, B)
    p.set_spectra(wl.cl)
    p.set_noise_cov(wl.sigma, wl.rho, wl.mask, wl.mask_p)
    p.set_schedule(**sched)
    return p


def _data(orc, wl):
    return np.stack([wl.data([orc.alm2map(wl.nside, wl.lmax, a)])[0] for a in wl.alm_true])


@pytest.mark.parametrize("nside,B,prec", [(8, 1, dmwf.DM_FP64), (16, 3, dmwf.DM_FP64),
                                          (16, 2, dmwf.DM_FLOAT_FLOAT), (16, 2, dmwf.DM_MIXED_FP32),
                                          (16, 8, dmwf.DM_MIXED_FP32)])
def test_cov_fixed_schedule_matches_oracle(orc, nside, B, prec):
    wl = W.make_cov_workload(list(range(20, 20 + B)), nside, 2 * nside)
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 4)
    p = _plan(wl, B, lambda0=1000.0, n_levels=4, iters_per_level=4)
    p.set_precision(prec)
    bar = 1e-10
    if prec == dmwf.DM_MIXED_FP32:
        p.set_refinement(6)  # anchors inside the 16 iterations
        bar = 1e-5
    s = torch.zeros((B, 3, wl.npix), dtype=torch.float64, device="cuda")
    a = torch.zeros((B, 3, (wl.lmax + 1) * (wl.lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s, a)
    p.close()
    assert all(x["iters_total"] == 16 for x in stats)
    gs, ga = s.cpu().numpy(), alm_host(a, (B, 3, -1))
    for b in range(0, B, max(1, B // 3)):
        ref = orc.dm_solve_cov(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, d[b], lam,
                               forced_iters=[4, 4, 4, 4])
        assert rel(gs[b], ref["s"]) < bar
        assert rel(ga[b], ref["alm"]) < bar


@pytest.mark.parametrize("prec,B,bar", [(dmwf.DM_FP64, 2, 1e-10), (dmwf.DM_MIXED_FP32, 8, 1e-5)])
def test_cov_diagnostics_match_oracle(orc, prec, B, bar):
    """The true residual and chi^2 in dm_stats under correlated noise with
    distinct T/P masks, against orc_wf_residual_cov / orc_chi2_cov on the
    oracle's own solve at the same counts (bars as for the diagonal model:
    chi^2 relative, the residual absolute)."""
    wl = W.make_cov_workload(list(range(50, 50 + B)), 16, 32)
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 4)
    p = _plan(wl, B, lambda0=1000.0, n_levels=4, iters_per_level=4)
    p.set_precision(prec)
    if prec == dmwf.DM_MIXED_FP32:
        p.set_refinement(6)
    s = torch.zeros((B, 3, wl.npix), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s)
    p.close()
    for b in [0, B - 1]:
        ref = orc.dm_solve_cov(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, d[b], lam,
                               forced_iters=[4, 4, 4, 4])
        r_ref = orc.wf_residual_cov(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, d[b],
                                    ref["alm"])
        c_ref = orc.chi2_cov(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, d[b], ref["s"],
                             ref["alm"])
        assert 1e-4 < r_ref < 1.0  # 16 iterations: far from converged, well away from zero
        assert abs(stats[b]["true_resid"] - r_ref) < bar, (b, stats[b]["true_resid"], r_ref)
        assert abs(stats[b]["chi2"] - c_ref) < bar * c_ref, (b, stats[b]["chi2"], c_ref)


def test_cov_cauchy_schedule_matches_oracle(orc):
    """Free-running levels (Cauchy 1e-3 -> 1e-5): the same per-level counts."""
    wl = W.make_cov_workload([30], 8, 16)
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 3)
    eps = W.eps_schedule(3, 1e-3, 1e-5)
    ref = orc.dm_solve_cov(8, 16, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, d[0], lam, eps=eps)
    p = _plan(wl, 1, lambda0=1000.0, n_levels=3, iters_per_level=0, eps0=1e-3, eps_final=1e-5, eta=0.0,
              check_every=1)
    s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s)
    p.close()
    assert list(stats[0]["iters_per_level"][:3]) == list(ref["iters_per_level"])
    assert rel(s.cpu().numpy()[0], ref["s"]) < 1e-10


def test_cov_rejections():
    wl = W.make_cov_workload([31], 4, 8)
    p = dmwf.Plan(4, 8, 1)
    p.set_spectra(wl.cl)
    bad = wl.rho.copy()
    bad[:, 0] = [0.9, 0.9, -0.9]  # not positive definite
    with pytest.raises(RuntimeError):
        p.set_noise_cov(wl.sigma, bad, wl.mask, wl.mask_p)
    p.set_noise_cov(wl.sigma, wl.rho, wl.mask, wl.mask_p)
    with pytest.raises(RuntimeError):  # the working resolution needs the diagonal model
        p.set_progressive(0.25, 2)
        p.set_schedule(lambda0=10.0, n_levels=2, iters_per_level=1)
        d = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
        p.wiener_filter(d, torch.zeros_like(d))
    p.close()


def test_cov_cr_inputs_match_oracle(orc):
    """The constrained-realisation draws under correlated noise: the signal
    draw, its synthesis and the conditional noise draw of Eq. 18 (zero on
    masked components), against orc_cr_inputs_cov, seed by seed."""
    wl = W.make_cov_workload([40], 16, 32)
    seeds = [901, 12345678901]
    p = _plan(wl, 2, lambda0=10.0, n_levels=2, iters_per_level=2)
    ah = torch.zeros((2, 3, (wl.lmax + 1) * (wl.lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    sh = torch.zeros((2, 3, wl.npix), dtype=torch.float64, device="cuda")
    dh = torch.zeros_like(sh)
    p.draw_cr_inputs(seeds, ahat=ah, shat=sh, dhat=dh)
    ga, gs, gd = alm_host(ah, (2, 3, -1)), sh.cpu().numpy(), dh.cpu().numpy()
    p.close()
    for b, sd in enumerate(seeds):
        a_ref, s_ref, d_ref = orc.cr_inputs_cov(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, sd)
        assert rel(ga[b], a_ref) < 1e-13
        assert rel(gs[b], s_ref) < 1e-13
        assert rel(gd[b], d_ref) < 1e-13
        assert np.all(gd[b][0][wl.mask == 0] == 0.0) and np.all(gd[b][1:][:, wl.mask_p == 0] == 0.0)


@pytest.mark.parametrize("prec", [dmwf.DM_FP64, dmwf.DM_FLOAT_FLOAT, dmwf.DM_MIXED_FP32])
def test_cov_constrained_realization_matches_oracle(orc, prec):
    """s_CR = W(d - dhat) + shat (Eq. 19) under correlated noise, one dual
    messenger run per realisation, against the oracle at the FP64 bar."""
    wl = W.make_cov_workload([41, 42], 16, 32)
    d = _data(orc, wl)
    lam = W.lambda_schedule(100.0, 3)
    seeds = [5, 6]
    p = _plan(wl, 2, lambda0=100.0, n_levels=3, iters_per_level=4)
    p.set_precision(prec)
    bar = 1e-10
    if prec == dmwf.DM_MIXED_FP32:
        p.set_refinement(5)
        bar = 1e-5
    s = torch.zeros((2, 3, wl.npix), dtype=torch.float64, device="cuda")
    a = torch.zeros((2, 3, (wl.lmax + 1) * (wl.lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    st, stats = p.constrained_realization(dev(d), seeds, s, a)
    gs, ga = s.cpu().numpy(), alm_host(a, (2, 3, -1))
    p.close()
    for b, sd in enumerate(seeds):
        ref = orc.constrained_realization_cov(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, d[b],
                                              sd, lam, forced_iters=[4, 4, 4])
        assert rel(gs[b], ref["s_cr"]) < bar
        assert rel(ga[b], ref["alm_cr"]) < bar
