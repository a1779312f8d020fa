"""Configuration nside 2048 / lmax 4096 (FP64 path, and the mixed path with
the tensor-core Legendre operand generated in the kernels) against the oracle
on sampled outputs.

A full oracle transform at this size takes far too long, so the oracle
computes whole rings of alm2map and whole orders m of map2alm one at a time
(oracle.ring_alm2map / map2alm_m, pinned to the full transforms at small
sizes).  The GPU runs the full transforms and one dual messenger iteration in
the FP64 mode.  The mixed mode's stored tables would not fit this size
(about 1 TB of tiles and FP32 tables), so its plans generate the tensor-core
tiles in the kernels and the float-float anchors' tables per slab.  Its
analysis sums over 2048 ring pairs in the tensor cores' FP32 accumulators:
measured, the error of a mixed map2alm grows in proportion to the pairs it
sums (7.5e-6 at nside 512 with stored and generated tiles alike, 2.5e-5 at
nside 2048), so the analysis is held to 5e-5 here and the synthesis to the
usual 2e-5; the first iteration, whose anchor is FP64-class, to 1e-5.  The data map of the iteration is the nside 2048
recipe's noise realisation on the observed pixels of its mask (no GPU result
enters an expected value).  Bar: the FP64 one, 1e-10 relative L2 per sample,
except on the two rings nearest each pole (theta < 1e-3): there the oracle's
own FP64 spin-2 recurrences are accurate to 2e-9 relative at l = 4096 (pinned
against 60-digit Wigner-d values in test_oracle_harmonics.py), so those rings
are held to 5e-9."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import alm_dev, alm_host, dev, rel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_1801_05358_gb300 import dmwf  # noqa: E402

NSIDE, LMAX = 2048, 4096
NPIX = 12 * NSIDE * NSIDE
NALM = (LMAX + 1) * (LMAX + 2) // 2
# polar (Bluestein and power-of-two lengths), belt, equator and south rings (1-based)
RINGS = [1, 2, 3, 511, 512, 2047, 2048, 3000, 4095, 4096, 6144, 8190, 8191]
ORDERS = [0, 1, 2, 3, 1000, 2047, 4095, 4096]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_alm2map_sampled_rings(orc):
    alm = W.random_alm(LMAX, 1, 51)
    p = dmwf.Plan(NSIDE, LMAX, 1)
    m_out = torch.zeros((1, 3, NPIX), dtype=torch.float64, device="cuda")
    p.alm2map(alm_dev(alm), m_out)
    gm = m_out[0].cpu().numpy()
    p.close()
    for i in RINGS:
        nr, st = orc.ring_info(NSIDE, i)[:2]
        bar = 5e-9 if min(i, 4 * NSIDE - i) <= 2 else 1e-10
        assert rel(gm[:, st:st + nr], orc.ring_alm2map(NSIDE, LMAX, alm[0], i)) < bar, i


def test_map2alm_sampled_orders(orc):
    maps = W.random_maps(NSIDE, 1, 52)
    p = dmwf.Plan(NSIDE, LMAX, 1)
    a_out = torch.zeros((1, 3, NALM, 2), dtype=torch.float64, device="cuda")
    p.map2alm(dev(maps), a_out)
    ga = alm_host(a_out, (1, 3, -1))[0]
    p.close()
    for m in ORDERS:
        idx = [orc.almidx(LMAX, l, m) for l in range(m, LMAX + 1)]
        ref = orc.map2alm_m(NSIDE, LMAX, maps[0], m)[:, m:]
        assert rel(ga[:, idx], ref) < 1e-10, m


def test_first_iteration_sampled_orders(orc):
    """One iteration at lambda_0 = 1000 from a = 0, t_0 = d on observed pixels:
    a_1 = F_0 A t_0 (Algorithm 1), compared on sampled orders m."""
    wl = W.make_workload("nside2048", [0])
    d = (wl.noise[0] * wl.mask[None, :]).astype(np.float64)
    p = dmwf.Plan(NSIDE, LMAX, 1)
    p.set_spectra(wl.cl)
    p.set_noise_mask(wl.sigma, wl.mask)
    p.set_schedule(lambda0=1000.0, n_levels=2, iters_per_level=0, check_every=1)
    p.set_forced_iters([1, 0])
    s = torch.zeros((1, 3, NPIX), dtype=torch.float64, device="cuda")
    a = torch.zeros((1, 3, NALM, 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d[None]), s, a)
    assert stats[0]["iters_total"] == 1
    ga = alm_host(a, (1, 3, -1))[0]
    p.close()
    th = orc.alpha(wl.sigma, wl.mask) * 4.0 * np.pi / NPIX
    coef = orc.filter_coefs(LMAX, wl.cl, (1000.0 - 1.0) * th, th)
    cols = np.zeros((3, NALM), dtype=np.complex128)
    for m in ORDERS:
        idx = [orc.almidx(LMAX, l, m) for l in range(m, LMAX + 1)]
        cols[:, idx] = orc.map2alm_m(NSIDE, LMAX, d, m)[:, m:]
    ref = orc.apply_filter(LMAX, coef, cols)
    for m in ORDERS:
        idx = [orc.almidx(LMAX, l, m) for l in range(m, LMAX + 1)]
        assert rel(ga[:, idx], ref[:, idx]) < 1e-10, m


MB = 8  # a tensor-core batch


def test_mixed_alm2map_sampled_rings(orc):
    alm = W.random_alm(LMAX, MB, 53)
    p = dmwf.Plan(NSIDE, LMAX, MB)
    p.set_precision(dmwf.DM_MIXED_FP32)
    m_out = torch.zeros((MB, 3, NPIX), dtype=torch.float64, device="cuda")
    p.alm2map(alm_dev(alm), m_out)
    torch.cuda.synchronize()
    p.close()
    for b in (0, MB - 1):
        for i in RINGS:
            nr, st = orc.ring_info(NSIDE, i)[:2]
            got = m_out[b, :, st:st + nr].cpu().numpy()
            assert rel(got, orc.ring_alm2map(NSIDE, LMAX, alm[b], i)) < 2e-5, (b, i)


def test_mixed_map2alm_sampled_orders(orc):
    maps = W.random_maps(NSIDE, MB, 54)
    p = dmwf.Plan(NSIDE, LMAX, MB)
    p.set_precision(dmwf.DM_MIXED_FP32)
    a_out = torch.zeros((MB, 3, NALM, 2), dtype=torch.float64, device="cuda")
    p.map2alm(dev(maps), a_out)
    ga = alm_host(a_out, (MB, 3, -1))
    p.close()
    for b in (0, MB - 1):
        for m in ORDERS:
            idx = [orc.almidx(LMAX, l, m) for l in range(m, LMAX + 1)]
            ref = orc.map2alm_m(NSIDE, LMAX, maps[b], m)[:, m:]
            assert rel(ga[b][:, idx], ref) < 5e-5, (b, m)


def test_mixed_first_iteration_sampled_orders(orc):
    """The first mixed iteration (float-float anchor at the start, one
    tensor-core iteration) on the same data in every RHS, against the oracle's
    a_1 = F_0 A t_0 on sampled orders."""
    wl = W.make_workload("nside2048", [0])
    d = (wl.noise[0] * wl.mask[None, :]).astype(np.float64)
    p = dmwf.Plan(NSIDE, LMAX, MB)
    p.set_precision(dmwf.DM_MIXED_FP32)
    p.set_spectra(wl.cl)
    p.set_noise_mask(wl.sigma, wl.mask)
    p.set_schedule(lambda0=1000.0, n_levels=2, iters_per_level=0, check_every=1)
    p.set_forced_iters([1, 0])
    s = torch.zeros((MB, 3, NPIX), dtype=torch.float64, device="cuda")
    a = torch.zeros((MB, 3, NALM, 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(np.broadcast_to(d[None], (MB,) + d.shape)), s, a)
    assert stats[0]["iters_total"] == 1
    ga = alm_host(a[0:1], (1, 3, -1))[0]
    p.close()
    th = orc.alpha(wl.sigma, wl.mask) * 4.0 * np.pi / NPIX
    coef = orc.filter_coefs(LMAX, wl.cl, (1000.0 - 1.0) * th, th)
    cols = np.zeros((3, NALM), dtype=np.complex128)
    for m in ORDERS:
        idx = [orc.almidx(LMAX, l, m) for l in range(m, LMAX + 1)]
        cols[:, idx] = orc.map2alm_m(NSIDE, LMAX, d, m)[:, m:]
    ref = orc.apply_filter(LMAX, coef, cols)
    # the mixed state is FP32 between anchors: coefficients far below FP32's
    # range (1e-88 at the highest orders after the lambda_0 = 1000 filter)
    # flush to zero, so each order's error is taken against the largest order
    # norm of the sample
    scale = max(np.linalg.norm(ref[:, [orc.almidx(LMAX, l, m) for l in range(m, LMAX + 1)]]) for m in ORDERS)
    for m in ORDERS:
        idx = [orc.almidx(LMAX, l, m) for l in range(m, LMAX + 1)]
        assert np.linalg.norm(ga[:, idx] - ref[:, idx]) / scale < 1e-5, m
