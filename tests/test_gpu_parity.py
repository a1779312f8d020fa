"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several CTAs and ragged tails: nside 8 (power-of-two rings),
nside 12 (Bluestein rings everywhere), nside 16 / lmax 47 (the configuration of
the 100-iteration fixed schedule) and batches of several right-hand sides.
FP64 tolerance: relative L2 <= 1e-10 (the stated bound for the FP64 mode);
single transforms are held to 1e-12."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import alm_dev, alm_host, dev, make_plan, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_05358_gb300 import dmwf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


GEOMS = [(2, 4), (8, 16), (12, 30), (16, 47)]


@pytest.mark.parametrize("nside,lmax", GEOMS)
def test_ring_fft_forward(orc, nside, lmax):
    B = 2
    maps = W.random_maps(nside, B, 100 + nside)
    p = dmwf.Plan(nside, lmax, B)
    rc = torch.zeros((B, 3, 4 * nside - 1, lmax + 1, 2), dtype=torch.float64, device="cuda")
    p.ring_fft_forward(dev(maps), rc)
    got = rc.cpu().numpy().view(np.complex128)[..., 0]
    for b in range(B):
        for f in range(3):
            ref = orc.ring_dft_forward(nside, lmax, maps[b, f])
            assert rel(got[b, f], ref) < 1e-13


@pytest.mark.parametrize("nside,lmax", GEOMS)
def test_ring_fft_inverse(orc, nside, lmax):
    B = 2
    rng = np.random.default_rng(nside)
    rc = rng.standard_normal((B, 3, 4 * nside - 1, lmax + 1)) + 1j * rng.standard_normal((B, 3, 4 * nside - 1, lmax + 1))
    rc[..., 0] = rc[..., 0].real
    p = dmwf.Plan(nside, lmax, B)
    out = torch.zeros((B, 3, 12 * nside * nside), dtype=torch.float64, device="cuda")
    p.ring_fft_inverse(alm_dev(rc), out)
    got = out.cpu().numpy()
    for b in range(B):
        for f in range(3):
            ref = orc.ring_dft_inverse(nside, lmax, rc[b, f])
            assert rel(got[b, f], ref) < 1e-13


@pytest.mark.parametrize("nside,lmax", GEOMS)
def test_legendre_synthesis(orc, nside, lmax):
    B = 2
    alm = W.random_alm(lmax, B, 7)
    p = dmwf.Plan(nside, lmax, B)
    rc = torch.zeros((B, 3, 4 * nside - 1, lmax + 1, 2), dtype=torch.float64, device="cuda")
    p.legendre_synthesis(alm_dev(alm), rc)
    got = rc.cpu().numpy().view(np.complex128)[..., 0]
    for b in range(B):
        ref = orc.legendre_synthesis(nside, lmax, alm[b])
        assert rel(got[b], ref) < 1e-12


@pytest.mark.parametrize("nside,lmax", GEOMS)
def test_legendre_analysis(orc, nside, lmax):
    B = 2
    rng = np.random.default_rng(3)
    rc = rng.standard_normal((B, 3, 4 * nside - 1, lmax + 1)) + 1j * rng.standard_normal((B, 3, 4 * nside - 1, lmax + 1))
    p = dmwf.Plan(nside, lmax, B)
    out = torch.zeros((B, 3, (lmax + 1) * (lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    p.legendre_analysis(alm_dev(rc), out)
    got = out.cpu().numpy().view(np.complex128)[..., 0]
    for b in range(B):
        ref = orc.legendre_analysis(nside, lmax, rc[b])
        assert rel(got[b], ref) < 1e-12


@pytest.mark.parametrize("nside,lmax", GEOMS)
def test_alm2map_map2alm(orc, nside, lmax):
    B = 3
    alm = W.random_alm(lmax, B, 8)
    maps = W.random_maps(nside, B, 9)
    p = dmwf.Plan(nside, lmax, B)
    m_out = torch.zeros((B, 3, 12 * nside * nside), dtype=torch.float64, device="cuda")
    a_out = torch.zeros((B, 3, (lmax + 1) * (lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    p.alm2map(alm_dev(alm), m_out)
    p.map2alm(dev(maps), a_out)
    gm = m_out.cpu().numpy()
    ga = a_out.cpu().numpy().view(np.complex128)[..., 0]
    for b in range(B):
        assert rel(gm[b], orc.alm2map(nside, lmax, alm[b])) < 1e-12
        assert rel(ga[b], orc.map2alm(nside, lmax, maps[b])) < 1e-12


@pytest.mark.parametrize("lam", [1.0, 7.5, 1000.0])
def test_filter(orc, lam):
    wl = W.make_workload("nside16", [0])
    p = make_plan(wl, 1)
    alpha, th = p.noise_info()
    assert alpha == pytest.approx(orc.alpha(wl.sigma, wl.mask), rel=1e-15)
    a = W.random_alm(wl.lmax, 1, 5)
    out = torch.zeros((1, 3, a.shape[-1], 2), dtype=torch.float64, device="cuda")
    p.apply_filter(lam, alm_dev(a), out)
    got = out.cpu().numpy().view(np.complex128)[..., 0][0]
    coef = orc.filter_coefs(wl.lmax, wl.cl, (lam - 1.0) * th, th)
    ref = orc.apply_filter(wl.lmax, coef, a[0])
    assert rel(got, ref) < 1e-14


def _data(orc, wl):
    return np.stack([wl.data([orc.alm2map(wl.nside, wl.lmax, a)])[0] for a in wl.alm_true])


def test_dm_fixed_schedule_nside16(orc):
    """Configuration nside 16 / lmax 47: lambda 1000 -> 1 over 10 levels, 10
    iterations each (100 iterations), FP64, relative L2 <= 1e-10."""
    wl = W.make_workload("nside16", [0])
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 10)
    ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[0], lam, forced_iters=[10] * 10)
    p = make_plan(wl, 1, lambda0=1000.0, n_levels=10, iters_per_level=10)
    s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    a = torch.zeros((1, 3, ref["alm"].shape[-1], 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s, a)
    assert stats[0]["iters_total"] == 100
    assert rel(s.cpu().numpy()[0], ref["s"]) < 1e-10
    assert rel(alm_host(a, (1, 3, -1))[0], ref["alm"]) < 1e-10


def test_dm_batch_equals_single(orc):
    """Three RHS in one launch give the single-RHS answers (and the oracle's)."""
    wl = W.make_workload("nside16", [1, 2, 3], nside=8, lmax=20)
    d = _data(orc, wl)
    lam = W.lambda_schedule(100.0, 4)
    p = make_plan(wl, 3, lambda0=100.0, n_levels=4, iters_per_level=5)
    s = torch.zeros((3, 3, wl.npix), dtype=torch.float64, device="cuda")
    p.wiener_filter(dev(d), s)
    got = s.cpu().numpy()
    for b in range(3):
        ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=[5] * 4)
        assert rel(got[b], ref["s"]) < 1e-10


def test_dm_cauchy_schedule_matches_oracle(orc):
    """Free-running Cauchy stopping: the per-level iteration counts agree with
    the oracle's, and so does the final map."""
    wl = W.make_workload("nside16", [0], nside=8, lmax=16)
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 5)
    eps = W.eps_schedule(5, 1e-3, 1e-6)
    ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[0], lam, eps=eps)
    p = make_plan(wl, 1, lambda0=1000.0, n_levels=5, iters_per_level=0, eps0=1e-3, eps_final=1e-6, eta=0.0,
                  check_every=16)
    s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s)
    assert stats[0]["iters_per_level"][:5] == list(ref["iters_per_level"])
    assert rel(s.cpu().numpy()[0], ref["s"]) < 1e-10


def test_dm_cauchy_schedule_nondefault_final_tolerance(orc):
    """dm_set_schedule's final tolerance reaches every RHS (a plan created with
    the default 1e-6, then scheduled 1e-3 -> 1e-5): the per-level counts agree
    with the oracle's."""
    wl = W.make_workload("nside16", [2, 3], nside=8, lmax=16)
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 3)
    eps = W.eps_schedule(3, 1e-3, 1e-5)
    p = make_plan(wl, 2, lambda0=1000.0, n_levels=3, iters_per_level=0, eps0=1e-3, eps_final=1e-5, eta=0.0,
                  check_every=8)
    s = torch.zeros((2, 3, wl.npix), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s)
    for b in range(2):
        ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, eps=eps)
        assert stats[b]["iters_per_level"][:3] == list(ref["iters_per_level"])
        assert rel(s.cpu().numpy()[b], ref["s"]) < 1e-10


def test_cr_inputs_match_oracle(orc):
    """Philox draws, ahat ~ S, shat = Y ahat, dhat = shat + nhat (Section 2.2)."""
    wl = W.make_workload("nside16", [0], nside=8, lmax=16)
    seeds = [11, 2 ** 40 + 5]
    p = make_plan(wl, 2)
    ah = torch.zeros((2, 3, (17 * 18) // 2, 2), dtype=torch.float64, device="cuda")
    sh = torch.zeros((2, 3, wl.npix), dtype=torch.float64, device="cuda")
    dh = torch.zeros((2, 3, wl.npix), dtype=torch.float64, device="cuda")
    p.draw_cr_inputs(seeds, ah, sh, dh)
    for b, sd in enumerate(seeds):
        a_ref, s_ref, d_ref = orc.cr_inputs(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, sd)
        assert rel(alm_host(ah, (2, 3, -1))[b], a_ref) < 1e-13
        assert rel(sh.cpu().numpy()[b], s_ref) < 1e-12
        assert rel(dh.cpu().numpy()[b], d_ref) < 1e-12


def test_constrained_realization(orc):
    wl = W.make_workload("nside16", [0], nside=8, lmax=16)
    d = _data(orc, wl)
    lam = W.lambda_schedule(100.0, 3)
    ref = orc.constrained_realization(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[0], 99, lam,
                                      forced_iters=[4, 4, 4])
    p = make_plan(wl, 1, lambda0=100.0, n_levels=3, iters_per_level=4)
    s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    p.constrained_realization(dev(d), [99], s)
    assert rel(s.cpu().numpy()[0], ref["s_cr"]) < 1e-10


@pytest.mark.parametrize("prec", [dmwf.DM_FP64, dmwf.DM_MIXED_FP32])
def test_session_api_equals_one_call(orc, prec):
    """dm_solve_begin + dm_solve_iterate in pieces + dm_solve_end gives the same
    iterate as dm_wiener_filter (the pieces are the same device work)."""
    wl = W.make_workload("nside16", [2], nside=8, lmax=16)
    d = _data(orc, wl)
    p = make_plan(wl, 1, lambda0=100.0, n_levels=3, iters_per_level=6, check_every=4)
    p.set_precision(prec)
    s1 = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    p.wiener_filter(dev(d), s1)
    s2 = torch.zeros_like(s1)
    p.solve_begin(dev(d))
    done = False
    for chunk in [1, 3, 5, 100]:
        done = p.solve_iterate(chunk)
        if done:
            break
    assert done
    st, stats = p.solve_end(s2)
    assert stats[0]["iters_total"] == 18
    assert rel(s2.cpu().numpy(), s1.cpu().numpy()) < (1e-15 if prec == dmwf.DM_FP64 else 1e-12)



def test_setters_refuse_changes_during_a_session(orc):
    """dm_set_schedule, dm_set_forced_iters and dm_set_spectra return DM_EBUSY
    between dm_solve_begin and dm_solve_end (they rewrite device-side level
    tables or filters); the session then ends normally and the plan accepts
    them again."""
    wl = W.make_workload("nside16", [2], nside=8, lmax=16)
    d = _data(orc, wl)
    p = make_plan(wl, 1, lambda0=100.0, n_levels=3, iters_per_level=6, check_every=4)
    s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    p.solve_begin(dev(d))
    for call in (lambda: p.set_schedule(lambda0=10.0, n_levels=2, iters_per_level=3),
                 lambda: p.set_forced_iters([1, 1, 1]),
                 lambda: p.set_spectra(wl.cl)):
        with pytest.raises(dmwf.DmError) as e:
            call()
        assert e.value.status == dmwf.DM_EBUSY
    assert p.solve_iterate(100)
    st, stats = p.solve_end(s)
    assert stats[0]["iters_total"] == 18
    p.set_schedule(lambda0=10.0, n_levels=2, iters_per_level=3)
    p.set_spectra(wl.cl)
    st, stats = p.wiener_filter(dev(d), s)
    assert stats[0]["iters_total"] == 6
    p.close()
