"""The flat-sky path on the GPU (the paper's own setting, Section 2.1 and 3.1:
2-D FFT transforms with the E/B rotation of Eqs. 13-16) against the flat-sky
oracle (oracle/flat.py), element by element through the C ABI:

- the analysis and synthesis alone (random maps, random Hermitian modes);
- the dual messenger solve at the oracle's per-level counts, batches of RHS,
  distinct temperature and polarisation masks, on grids of 64, 256 and
  1024 pixels (the paper's 1024^2, where the row transforms take the
  fixed-size ring kernels);
- the free-running Cauchy schedule: the same per-level counts;
- the end-of-solve true residual and chi^2 against the oracle's definitions;
- constrained realisations (the drawn inputs and the whole realisation),
  with the oracle fed the same Philox normals;
- the modified Jacobi refinement (Appendix A).

Layouts: the oracle's modes are [3, N, N] in numpy order (axis 0 = ky); the
library keeps kx = 0 .. N/2 - 1 with every ky, [3, N/2, N].  Bar: the FP64
bar, 1e-10 for solves and 1e-12 for single transforms."""
import numpy as np
import pytest

import workloads as W
from oracle import flat as F
from tests.gpu_helpers import dev, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_05358_gb300 import dmwf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _ours(a):
    """oracle modes [..., 3, N, N] (ky, kx) -> the library's [..., 3, N/2, N] (kx < N/2, ky)"""
    N = a.shape[-1]
    return np.swapaxes(a[..., :, :N // 2], -1, -2)


def _alm_of(t, B, N):
    return t.cpu().numpy().view(np.complex128)[..., 0].reshape(B, 3, N // 2, N)


def _plan(wl, B, **sched):
    p = dmwf.FlatPlan(wl.N, wl.L, B)
    p.set_spectra(wl.S)
    p.set_noise(wl.sigma.reshape(3, -1), wl.mask_t.ravel(), wl.mask_p.ravel())
    if sched:
        p.set_schedule(**sched)
    return p


@pytest.mark.parametrize("N", [64, 1024])
def test_flat_transforms(N):
    L = W.FLAT_L
    rng = np.random.default_rng(N)
    B = 2
    maps = rng.standard_normal((B, 3, N, N))
    ref_a = np.stack([F.analysis(m, L) for m in maps])
    alm_in = np.stack([F.analysis(m, L) for m in rng.standard_normal((B, 3, N, N))])  # Hermitian modes
    ref_m = np.stack([F.synthesis(a, L) for a in alm_in])
    p = dmwf.FlatPlan(N, L, B)
    a_out = torch.zeros((B, 3, N * N // 2, 2), dtype=torch.float64, device="cuda")
    m_out = torch.zeros((B, 3, N * N), dtype=torch.float64, device="cuda")
    p.map2alm(dev(maps.reshape(B, 3, -1)), a_out)
    p.alm2map(dev(np.ascontiguousarray(_ours(alm_in)).view(np.float64)), m_out)
    torch.cuda.synchronize()
    got_a = _alm_of(a_out, B, N)
    got_m = m_out.cpu().numpy().reshape(B, 3, N, N)
    p.close()
    for b in range(B):
        assert rel(got_a[b], _ours(ref_a[b])) < 1e-12
        assert rel(got_m[b], ref_m[b]) < 1e-12


@pytest.mark.parametrize("N,B", [(64, 2), (256, 1), (1024, 1)])
def test_flat_solve_matches_oracle(N, B):
    wl = W.make_flat_workload(list(range(3, 3 + B)), N=N)
    d = np.stack(wl.data([F.synthesis(a, wl.L) for a in wl.alm_true]))
    lam = W.lambda_schedule(1000.0, 3)
    counts = [3, 3, 3]
    p = _plan(wl, B, lambda0=1000.0, n_levels=3, iters_per_level=3, check_every=4)
    s = torch.zeros((B, 3, N * N), dtype=torch.float64, device="cuda")
    a = torch.zeros((B, 3, N * N // 2, 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d.reshape(B, 3, -1)), s, a)
    gs = s.cpu().numpy().reshape(B, 3, N, N)
    ga = _alm_of(a, B, N)
    p.close()
    for b in range(B):
        assert stats[b]["iters_per_level"][:3] == counts
        ref = F.dm_solve(d[b], wl.sigma, wl.mask_t, wl.mask_p, wl.S, wl.L, lam, forced_iters=counts)
        assert rel(gs[b], ref["s"]) < 1e-10
        assert rel(ga[b], _ours(ref["alm"])) < 1e-10


def test_flat_diagnostics_match_oracle():
    """The true residual and chi^2 in dm_stats of a flat-sky solve against the
    flat oracle's definitions (flat.wf_residual, flat.chi2) on the oracle's
    own solve at the same counts: the residual absolute, chi^2 relative, at
    the FP64 bar."""
    N, B = 64, 2
    wl = W.make_flat_workload([11, 12], N=N)
    d = np.stack(wl.data([F.synthesis(a, wl.L) for a in wl.alm_true]))
    lam = W.lambda_schedule(1000.0, 3)
    counts = [3, 3, 3]
    p = _plan(wl, B, lambda0=1000.0, n_levels=3, iters_per_level=3, check_every=4)
    s = torch.zeros((B, 3, N * N), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d.reshape(B, 3, -1)), s)
    p.close()
    for b in range(B):
        ref = F.dm_solve(d[b], wl.sigma, wl.mask_t, wl.mask_p, wl.S, wl.L, lam, forced_iters=counts)
        r_ref = F.wf_residual(ref["alm"], d[b], wl.sigma, wl.mask_t, wl.mask_p, wl.S, wl.L)
        c_ref = F.chi2(ref["alm"], d[b], wl.sigma, wl.mask_t, wl.mask_p, wl.S, wl.L)
        assert 1e-4 < r_ref < 1.0  # 9 iterations: far from converged, well away from zero
        assert abs(stats[b]["true_resid"] - r_ref) < 1e-10, (b, stats[b]["true_resid"], r_ref)
        assert abs(stats[b]["chi2"] - c_ref) < 1e-10 * c_ref, (b, stats[b]["chi2"], c_ref)


def test_flat_cauchy_schedule_matches_oracle():
    N = 64
    wl = W.make_flat_workload([9], N=N)
    d = wl.data([F.synthesis(wl.alm_true[0], wl.L)])[0]
    lam = W.lambda_schedule(100.0, 3)
    eps = W.eps_schedule(3, 1e-2, 1e-4)
    ref = F.dm_solve(d, wl.sigma, wl.mask_t, wl.mask_p, wl.S, wl.L, lam, eps=eps)
    p = _plan(wl, 1, lambda0=100.0, n_levels=3, iters_per_level=0, eps0=1e-2, eps_final=1e-4, eta=0.0,
              check_every=1)
    s = torch.zeros((1, 3, N * N), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d.reshape(1, 3, -1)), s)
    p.close()
    assert list(stats[0]["iters_per_level"][:3]) == list(ref["iters_per_level"])
    assert rel(s.cpu().numpy().reshape(3, N, N), ref["s"]) < 1e-10


def _flat_normals(orc, seed, N):
    """The unit normals the library draws for a flat constrained realisation,
    from the oracle's own Philox4x32-10 and Box-Muller (orc_gauss_pair):
    per pixel p = y N + x, signal maps (I, Q) from counter (p, 0, 2) and U
    from (p, 1, 2); noise (I, Q) from (p, 0, 1) and U from (p, 1, 1)."""
    zs = np.zeros((3, N * N))
    zn = np.zeros((3, N * N))
    for q in range(N * N):
        zs[0, q], zs[1, q] = orc.gauss_pair(seed, q, 0, 2)
        zs[2, q] = orc.gauss_pair(seed, q, 1, 2)[0]
        zn[0, q], zn[1, q] = orc.gauss_pair(seed, q, 0, 1)
        zn[2, q] = orc.gauss_pair(seed, q, 1, 1)[0]
    return zs.reshape(3, N, N), zn.reshape(3, N, N)


def test_flat_constrained_realization_matches_oracle(orc):
    """Constrained realisations on the flat patch (Section 2.2, Eq. 19): the
    drawn inputs (a_hat, s_hat, d_hat) at 1e-12 and the whole realisation at
    the oracle's per-level counts at 1e-10, distinct T/P masks, 2 RHS."""
    N, B = 64, 2
    seeds = [501, 502]
    wl = W.make_flat_workload([13, 14], N=N)
    d = np.stack(wl.data([F.synthesis(a, wl.L) for a in wl.alm_true]))
    lam = W.lambda_schedule(1000.0, 3)
    counts = [3, 3, 3]
    p = _plan(wl, B, lambda0=1000.0, n_levels=3, iters_per_level=3, check_every=4)
    ah = torch.zeros((B, 3, N * N // 2, 2), dtype=torch.float64, device="cuda")
    sh = torch.zeros((B, 3, N * N), dtype=torch.float64, device="cuda")
    dh = torch.zeros((B, 3, N * N), dtype=torch.float64, device="cuda")
    p.draw_cr_inputs(seeds, ahat=ah, shat=sh, dhat=dh)
    s = torch.zeros((B, 3, N * N), dtype=torch.float64, device="cuda")
    a = torch.zeros((B, 3, N * N // 2, 2), dtype=torch.float64, device="cuda")
    st, stats = p.constrained_realization(dev(d.reshape(B, 3, -1)), seeds, s, a)
    p.close()
    g_ah, g_sh, g_dh = _alm_of(ah, B, N), sh.cpu().numpy().reshape(B, 3, N, N), dh.cpu().numpy().reshape(B, 3, N, N)
    gs, ga = s.cpu().numpy().reshape(B, 3, N, N), _alm_of(a, B, N)
    for b in range(B):
        zs, zn = _flat_normals(orc, seeds[b], N)
        ref = F.constrained_realization(d[b], zs, zn, wl.sigma, wl.mask_t, wl.mask_p, wl.S, wl.L, lam,
                                        forced_iters=counts)
        assert rel(g_ah[b], _ours(ref["a_hat"])) < 1e-12
        assert rel(g_sh[b], ref["s_hat"]) < 1e-12
        assert rel(g_dh[b], ref["d_hat"]) < 1e-12
        assert stats[b]["iters_per_level"][:3] == counts
        assert rel(gs[b], ref["s_cr"]) < 1e-10
        assert rel(ga[b], _ours(ref["alm_cr"])) < 1e-10


def test_flat_jacobi_refine_matches_oracle():
    """The modified Jacobi refinement (Appendix A) on the flat patch against
    flat.jacobi_refine: the solve at the oracle's counts, then two refinement
    steps at those counts, at the FP64 bar; the true residual drops."""
    N, B = 64, 2
    wl = W.make_flat_workload([15, 16], N=N)
    d = np.stack(wl.data([F.synthesis(a, wl.L) for a in wl.alm_true]))
    lam = W.lambda_schedule(1000.0, 3)
    counts = [3, 3, 3]
    p = _plan(wl, B, lambda0=1000.0, n_levels=3, iters_per_level=3, check_every=4)
    s = torch.zeros((B, 3, N * N), dtype=torch.float64, device="cuda")
    a = torch.zeros((B, 3, N * N // 2, 2), dtype=torch.float64, device="cuda")
    st, base = p.wiener_filter(dev(d.reshape(B, 3, -1)), s)
    st, stats = p.jacobi_refine(dev(d.reshape(B, 3, -1)), 2, s, a)
    gs, ga = s.cpu().numpy().reshape(B, 3, N, N), _alm_of(a, B, N)
    p.close()
    for b in range(B):
        assert stats[b]["iters_total"] == 3 * sum(counts)
        assert stats[b]["true_resid"] < 0.5 * base[b]["true_resid"]
        ref = F.jacobi_refine(d[b], wl.sigma, wl.mask_t, wl.mask_p, wl.S, wl.L, lam, forced_iters=counts,
                              n_refine=2)
        assert rel(gs[b], ref["s"]) < 1e-10
        assert rel(ga[b], _ours(ref["alm"])) < 1e-10


def test_flat_plan_refuses_sphere_calls():
    p = dmwf.FlatPlan(32, W.FLAT_L, 1)
    with pytest.raises(dmwf.DmError):
        p.set_precision(dmwf.DM_MIXED_FP32)
    with pytest.raises(dmwf.DmError):
        dmwf.Plan.set_spectra(p, np.zeros((4, 3)))
    p.close()
