"""Float-float Legendre stages (DM_FLOAT_FLOAT) and float-float anchors of the
mixed mode, against the FP64 oracle through the C ABI.

The float-float transforms carry about 48 significant bits: single transforms
are held to 1e-12 relative L2 (like the FP64 kernels) and a whole 100-iteration
solve to the FP64 bar of 1e-10.  Mixed solves with float-float anchors must
agree with the same solves anchored by the FP64 kernels far below the mixed
tolerance, since both anchors are FP64-class."""
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


def _data(orc, wl):
    return np.stack([wl.data([orc.alm2map(wl.nside, wl.lmax, a)])[0] for a in wl.alm_true])


@pytest.mark.parametrize("nside,lmax,B", [(2, 4, 1), (8, 16, 3), (12, 30, 2), (16, 47, 5)])
def test_ff_transforms(orc, nside, lmax, B):
    alm = W.random_alm(lmax, B, 21)
    maps = W.random_maps(nside, B, 22)
    p = dmwf.Plan(nside, lmax, B)
    p.set_precision(dmwf.DM_FLOAT_FLOAT)
    m_out = torch.zeros((B, 3, 12 * nside * nside), dtype=torch.float64, device="cuda")
    a_out = torch.zeros((B, 3, (lmax + 1) * (lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    p.alm2map(alm_dev(alm), m_out)
    p.map2alm(dev(maps), a_out)
    gm = m_out.cpu().numpy()
    ga = a_out.cpu().numpy().view(np.complex128)[..., 0]
    for b in range(B):
        assert rel(gm[b], orc.alm2map(nside, lmax, alm[b])) < 1e-12
        assert rel(ga[b], orc.map2alm(nside, lmax, maps[b])) < 1e-12


def test_ff_legendre_stages(orc):
    nside, lmax, B = 12, 30, 2
    alm = W.random_alm(lmax, B, 23)
    rng = np.random.default_rng(24)
    rcin = rng.standard_normal((B, 3, 4 * nside - 1, lmax + 1)) + 1j * rng.standard_normal((B, 3, 4 * nside - 1, lmax + 1))
    p = dmwf.Plan(nside, lmax, B)
    p.set_precision(dmwf.DM_FLOAT_FLOAT)
    rc = torch.zeros((B, 3, 4 * nside - 1, lmax + 1, 2), dtype=torch.float64, device="cuda")
    p.legendre_synthesis(alm_dev(alm), rc)
    out = torch.zeros((B, 3, (lmax + 1) * (lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    p.legendre_analysis(alm_dev(rcin), out)
    gs = rc.cpu().numpy().view(np.complex128)[..., 0]
    ga = out.cpu().numpy().view(np.complex128)[..., 0]
    for b in range(B):
        assert rel(gs[b], orc.legendre_synthesis(nside, lmax, alm[b])) < 1e-12
        assert rel(ga[b], orc.legendre_analysis(nside, lmax, rcin[b])) < 1e-12


def test_ff_fixed_schedule_nside16(orc):
    """The 100-iteration schedule (lambda 1000 -> 1, 10 levels x 10) in
    DM_FLOAT_FLOAT meets the FP64 bar, relative L2 <= 1e-10."""
    wl = W.make_workload("nside16", [0])
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 10)
    ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[0], lam, forced_iters=[10] * 10)
    p = make_plan(wl, 1, lambda0=1000.0, n_levels=10, iters_per_level=10)
    p.set_precision(dmwf.DM_FLOAT_FLOAT)
    s = torch.zeros((1, 3, wl.npix), dtype=torch.float64, device="cuda")
    a = torch.zeros((1, 3, ref["alm"].shape[-1], 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s, a)
    assert stats[0]["iters_total"] == 100
    assert rel(s.cpu().numpy()[0], ref["s"]) < 1e-10
    assert rel(alm_host(a, (1, 3, -1))[0], ref["alm"]) < 1e-10


@pytest.mark.parametrize("batch", [2, 8])
def test_mixed_ff_anchor_equals_fp64_anchor(orc, batch):
    """Same mixed solve (anchors every 16 iterations), anchors in float-float
    and in FP64: both meet the mixed bar (1e-5) for every RHS and they agree
    to 1e-6.  The anchors themselves differ near 1e-13, but the FP32 / BF16
    roundings of the inner iterations are discontinuous in their inputs, so
    the two runs may part at the inner precision; 1e-6 keeps a factor of ten
    below the mixed bar."""
    wl = W.make_workload("nside16", list(range(batch)))
    d = _data(orc, wl)
    outs = []
    for ap in [dmwf.DM_FLOAT_FLOAT, dmwf.DM_FP64]:
        p = make_plan(wl, batch, lambda0=1000.0, n_levels=10, iters_per_level=10, check_every=16)
        p.set_precision(dmwf.DM_MIXED_FP32)
        p.set_refinement(16)
        p.set_anchor_precision(ap)
        s = torch.zeros((batch, 3, wl.npix), dtype=torch.float64, device="cuda")
        p.wiener_filter(dev(d), s)
        outs.append(s.cpu().numpy())
        p.close()
    assert rel(outs[0], outs[1]) < 1e-6
    lam = W.lambda_schedule(1000.0, 10)
    for b in range(batch):
        ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=[10] * 10)
        assert rel(outs[0][b], ref["s"]) < 1e-5
        assert rel(outs[1][b], ref["s"]) < 1e-5


def test_anchor_precision_rejects_mixed():
    p = dmwf.Plan(4, 8, 1)
    with pytest.raises(RuntimeError):
        p.set_anchor_precision(dmwf.DM_MIXED_FP32)


# Without full FP32 tables (DM_FLOAT_FLOAT never builds them) the float-float
# stages generate their tables per slab of orders m and contract each slab
# before the next; slabs of a few kilobytes force many slabs of uneven length.
@pytest.mark.parametrize("slab", [1, 40_000, 300_000])
def test_ff_slabs_match_oracle(orc, slab):
    nside, lmax, B = 16, 47, 3
    alm = W.random_alm(lmax, B, 61)
    maps = W.random_maps(nside, B, 62)
    p = dmwf.Plan(nside, lmax, B)
    p.set_precision(dmwf.DM_FLOAT_FLOAT)
    p.set_ff_slab_bytes(slab)
    m_out = torch.zeros((B, 3, 12 * nside * nside), dtype=torch.float64, device="cuda")
    a_out = torch.zeros((B, 3, (lmax + 1) * (lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    p.alm2map(alm_dev(alm), m_out)
    p.map2alm(dev(maps), a_out)
    gm = m_out.cpu().numpy()
    ga = a_out.cpu().numpy().view(np.complex128)[..., 0]
    p.close()
    for b in range(B):
        assert rel(gm[b], orc.alm2map(nside, lmax, alm[b])) < 1e-12
        assert rel(ga[b], orc.map2alm(nside, lmax, maps[b])) < 1e-12


def test_ff_slab_solve_matches_oracle(orc):
    wl = W.make_workload("nside16", [4, 5])
    d = _data(orc, wl)
    lam = W.lambda_schedule(1000.0, 4)
    p = make_plan(wl, 2, lambda0=1000.0, n_levels=4, iters_per_level=5)
    p.set_precision(dmwf.DM_FLOAT_FLOAT)
    p.set_ff_slab_bytes(100_000)
    s = torch.zeros((2, 3, wl.npix), dtype=torch.float64, device="cuda")
    p.wiener_filter(dev(d), s)
    got = s.cpu().numpy()
    p.close()
    for b in range(2):
        ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=[5] * 4)
        assert rel(got[b], ref["s"]) < 1e-10
