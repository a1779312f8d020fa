"""Dual messenger iterations on rings of 512 to 2048 FFT points (nside 128, 256
and 512), where the ring stage of the iteration runs the fixed-size radix-16
transforms: the FP64 mode against the oracle at 1e-10 and the mixed mode at
1e-5 (the bounds of the two modes), over the direct (power-of-two) and the
Bluestein rings of every size class:

  nside 128: Bluestein M = 512 (and the generic classes up to 256 points);
  nside 256: direct M = 512 (equatorial belt), Bluestein M = 1024;
  nside 512: direct M = 1024 (equatorial belt), Bluestein M = 512 and 2048.

The inputs are the nside 256 recipe (band, 3-degree and 0.5-degree disks) at
each nside, lmax = 2 nside, with a forced number of iterations per level."""
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


def _case(orc, nside, seeds):
    wl = W.make_workload("nside256", seeds, nside=nside, lmax=2 * nside)
    d = np.stack([wl.data([orc.alm2map(wl.nside, wl.lmax, a)])[0] for a in wl.alm_true])
    return wl, d


def _run(orc, wl, d, iters, prec, lr=None, tuning=None):
    B = d.shape[0]
    lam = W.lambda_schedule(1000.0, len(iters)) if len(iters) > 1 else np.array([1000.0])
    if len(iters) == 1:  # iters[0] iterations at lambda = 1000, none at lambda = 1
        p = make_plan(wl, B, lambda0=1000.0, n_levels=2, iters_per_level=0, check_every=1)
        p.set_forced_iters([iters[0], 0])
    else:
        p = make_plan(wl, B, lambda0=1000.0, n_levels=len(iters), iters_per_level=iters[0])
    p.set_precision(prec)
    if lr is not None:
        p.set_ring_radix(lr)
    if tuning is not None:
        p.set_tuning(tuning)
    s = torch.zeros((B, 3, wl.npix), dtype=torch.float64, device="cuda")
    a = torch.zeros((B, 3, (wl.lmax + 1) * (wl.lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
    st, stats = p.wiener_filter(dev(d), s, a)
    p.close()
    assert all(x["iters_total"] == sum(iters) for x in stats)
    gs, ga = s.cpu().numpy(), alm_host(a, (B, 3, -1))
    errs = []
    for b in range(B):
        ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=list(iters))
        errs.append((rel(gs[b], ref["s"]), rel(ga[b], ref["alm"])))
    return errs


@pytest.mark.parametrize("lr", [3, 4, 0])
@pytest.mark.parametrize("nside,iters,B", [(128, [2, 2], 3), (256, [2], 1)])
def test_fp64_iterations_large_rings(orc, nside, iters, B, lr):
    """Radix 8, radix 16 and the generic kernels (dm_set_ring_radix)."""
    wl, d = _case(orc, nside, list(range(70, 70 + B)))
    for es, ea in _run(orc, wl, d, iters, dmwf.DM_FP64, lr):
        assert es < 1e-10 and ea < 1e-10, (es, ea)


@pytest.mark.parametrize("lr", [3, 4, 0])
def test_mixed_iterations_nside128(orc, lr):
    wl, d = _case(orc, 128, [80, 81])
    for es, ea in _run(orc, wl, d, [3, 3], dmwf.DM_MIXED_FP32, lr):
        assert es < 1e-5 and ea < 1e-5, (es, ea)


@pytest.mark.parametrize("nside", [128, 256])
def test_mixed_iterations_register_capped_radix16(orc, nside):
    """Tuning variant 2 (the FP32 radix-16 kernels compiled for 80 registers a
    thread) on every class it serves: 512 points at nside 128, 512 and 1024
    at nside 256; the generic classes keep their kernels."""
    wl, d = _case(orc, nside, [82])
    n = dmwf.DM_TUNE_MAX_CLASSES
    tuning = {"ring_radix_lr": [4] * n, "ring_lanes": [0] * n, "ring_fused": [2] * n}
    for es, ea in _run(orc, wl, d, [3, 3], dmwf.DM_MIXED_FP32, tuning=tuning):
        assert es < 1e-5 and ea < 1e-5, (es, ea)


def test_ring_radix_rejects_other_values():
    p = dmwf.Plan(8, 16, 1)
    for lr in (1, 2, 5, -1):
        with pytest.raises(RuntimeError):
            p.set_ring_radix(lr)
    p.close()


@pytest.mark.slow
@pytest.mark.parametrize("prec,bar", [(dmwf.DM_FP64, 1e-10), (dmwf.DM_MIXED_FP32, 1e-5)])
def test_iterations_nside512(orc, prec, bar):
    wl, d = _case(orc, 512, [90])
    for es, ea in _run(orc, wl, d, [2], prec):
        assert es < bar and ea < bar, (es, ea)
