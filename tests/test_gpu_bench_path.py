"""Whole iterations of the benchmarked configurations against the oracle
(Algorithm 1 at the oracle's per-level counts, element by element).

- The bench's own iteration: nside 512 / lmax 1024, 64 right-hand sides
  (32 Wiener-filter data maps and 32 fluctuation data maps of constrained
  realisations), DM_MIXED_FP32 with the tcgen05 tensor-core Legendre stages,
  the default ring kernels (paired radix-8 fixed-size transforms), the FP32
  filtered step and the float-float anchors.  Four forced iterations over
  two levels (lambda 1000, 1) with an anchor period of 2, so that an anchor
  falls between tensor-core iterations and one RHS changes level between
  them.  RHS 0 and 31 (Wiener filter) and 63 (fluctuation) are compared with
  the oracle's solve of the same data, made on the host (the oracle's
  synthesis plus the drawn noise; the fluctuation data from the oracle's
  Philox draws).  Bar: the mixed-mode bound 1e-5 in relative L2.
- Configuration nside 256 / lmax 512 (one RHS), 30 forced iterations over
  three levels (lambda 1000 -> 1), in DM_FP64 (bar 1e-10) and DM_MIXED_FP32
  (bar 1e-5).
- The same configuration solved to convergence in both modes (Cauchy 1e-5,
  progressive working resolution): mixed against FP64 at 1e-5.

The oracle costs about 11 s per iteration at nside 512 and 1.5 s at nside
256 on 16 host cores, so these are slow tests."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import alm_host, dev, rel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_1801_05358_gb300 import dmwf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_bench_iteration_matches_oracle(orc):
    nside, lmax, B = 512, 1024, 64
    npix = 12 * nside * nside
    wl = W.make_workload("nside512", [100, 131], nside=nside, lmax=lmax)
    d_wf = [wl.data([orc.alm2map(nside, lmax, a)])[0] for a in wl.alm_true]
    dhat = orc.cr_inputs(nside, lmax, wl.cl, wl.sigma, wl.mask, 163)[2]
    sampled = {0: d_wf[0], 31: d_wf[1], 63: dhat}
    pool = [d_wf[0], d_wf[1], dhat]
    d = torch.zeros((B, 3, npix), dtype=torch.float64, device="cuda")
    for b in range(B):
        d[b] = dev(sampled.get(b, pool[b % 3]))
    lam = W.lambda_schedule(1000.0, 2)
    counts = [2, 2]
    p = dmwf.Plan(nside, lmax, B)
    p.set_spectra(wl.cl)
    p.set_noise_mask(wl.sigma, wl.mask)
    p.set_precision(dmwf.DM_MIXED_FP32)
    p.set_refinement(2)
    p.set_schedule(lambda0=1000.0, n_levels=2, iters_per_level=0, eps0=1e-4, eps_final=1e-6, check_every=1)
    p.set_forced_iters(counts)
    s = torch.zeros_like(d)
    a = torch.zeros((B, 3, p.nalm, 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(d, s, a)
    assert stats[0]["iters_total"] == 4 and stats[63]["iters_per_level"][:2] == counts
    del d
    got_s = {b: s[b].cpu().numpy() for b in sampled}
    got_a = {b: alm_host(a[b:b + 1], (1, 3, -1))[0] for b in sampled}
    p.close()
    del s, a
    for b, db in sampled.items():
        ref = orc.dm_solve(nside, lmax, wl.cl, wl.sigma, wl.mask, db, lam, forced_iters=counts)
        assert rel(got_s[b], ref["s"]) < 1e-5, b
        assert rel(got_a[b], ref["alm"]) < 1e-5, b


@pytest.mark.parametrize("prec,bar", [(dmwf.DM_FP64, 1e-10), (dmwf.DM_MIXED_FP32, 1e-5)])
def test_config1_nside256_three_levels(orc, prec, bar):
    wl = W.make_workload("nside256", [1])
    d = wl.data([orc.alm2map(wl.nside, wl.lmax, wl.alm_true[0])])[0]
    lam = W.lambda_schedule(1000.0, 3)
    counts = [10, 10, 10]
    ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d, lam, forced_iters=counts)
    p = dmwf.Plan(wl.nside, wl.lmax, 1)
    p.set_spectra(wl.cl)
    p.set_noise_mask(wl.sigma, wl.mask)
    p.set_precision(prec)
    p.set_schedule(lambda0=1000.0, n_levels=3, iters_per_level=10, check_every=8)
    s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    a = torch.zeros((1, 3, p.nalm, 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d[None]), s, a)
    assert stats[0]["iters_per_level"][:3] == counts
    assert rel(s.cpu().numpy()[0], ref["s"]) < bar
    assert rel(alm_host(a, (1, 3, -1))[0], ref["alm"]) < bar
    p.close()


def test_config1_converged_mixed_vs_fp64(orc):
    """Configuration nside 256 / lmax 512 solved to convergence (lambda 1000 ->
    1 over 10 levels, Cauchy threshold cooled from 1e-4 to 1e-5, progressive
    working resolution) in DM_FP64 and in DM_MIXED_FP32 from the same data:
    both converge, and the mixed map agrees with the FP64 map (itself held to
    the oracle at 1e-10 above) within the mixed-mode bound 1e-5.  The
    device FP64 true residuals of the two agree too."""
    wl = W.make_workload("nside256", [2])
    d = wl.data([orc.alm2map(wl.nside, wl.lmax, wl.alm_true[0])])[0]
    p = dmwf.Plan(wl.nside, wl.lmax, 1)
    p.set_spectra(wl.cl)
    p.set_noise_mask(wl.sigma, wl.mask)
    p.set_progressive(0.25, 8)
    out = {}
    for name, prec in (("mixed", dmwf.DM_MIXED_FP32), ("fp64", dmwf.DM_FP64)):
        p.set_precision(prec)
        p.set_schedule(lambda0=1000.0, n_levels=10, iters_per_level=0, eps0=1e-4, eps_final=1e-5, eta=0.0,
                       max_iter=200000, check_every=64)
        s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
        st, stats = p.wiener_filter(dev(d[None]), s)
        assert st == dmwf.DM_OK, (name, stats[0])
        assert stats[0]["cauchy_final"] < 1e-5
        assert stats[0]["true_resid"] < 1e-4, (name, stats[0]["true_resid"])
        out[name] = (s.cpu().numpy()[0], stats[0])
    p.close()
    assert rel(out["mixed"][0], out["fp64"][0]) < 1e-5
    tm, tf = out["mixed"][1]["true_resid"], out["fp64"][1]["true_resid"]
    assert abs(tm - tf) < 1e-2 * tf, (tm, tf)
