"""The tensor-core Legendre stages in the benchmark's launch configuration:
nside 512 / lmax 1024, 64 right-hand sides, DM_MIXED_FP32 (tcgen05 products
of split-BF16 operands with FP32 accumulation), against the oracle on
sampled outputs.

A full oracle transform at this size is too slow, so the oracle computes
whole rings of alm2map and whole orders m of map2alm one at a time
(oracle.ring_alm2map / map2alm_m, pinned to the full transforms at small
sizes) for sampled right-hand sides: the first, a middle and the last of the
batch, so that every batch tile of the tensor-core operand is visited.  The
rings cover both polar caps (Bluestein and power-of-two lengths), the belt
edges and the equator; the orders cover m = 0, small m, the middle and
m = lmax.  Bar: 2e-5 relative L2 over the samples, the single-transform
bound of the smaller tensor-core tests.  A CPU model of the arithmetic (BF16
hi/lo operands, the three products, FP32 sums per K step of 16) gives
2e-6 to 5e-6 on spin-0 synthesis rings at this size."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import alm_dev, alm_host, dev, rel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_1801_05358_gb300 import dmwf  # noqa: E402

NSIDE, LMAX, B = 512, 1024, 64
NPIX = 12 * NSIDE * NSIDE
NALM = (LMAX + 1) * (LMAX + 2) // 2
RINGS = [1, 2, 3, 511, 512, 1024, 1536, 2045, 2047]  # 1-based, 2047 rings
ORDERS = [0, 1, 2, 511, 1000, 1024]
RHS = [0, 31, 63]


@pytest.fixture(scope="module")
def plan():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    p = dmwf.Plan(NSIDE, LMAX, B)
    p.set_precision(dmwf.DM_MIXED_FP32)
    yield p
    p.close()


def test_tc_alm2map_bench_size_sampled_rings(orc, plan):
    alm = W.random_alm(LMAX, B, 61)
    m_out = torch.zeros((B, 3, NPIX), dtype=torch.float64, device="cuda")
    plan.alm2map(alm_dev(alm), m_out)
    got, ref = [], []
    for b in RHS:
        gm = m_out[b].cpu().numpy()
        for i in RINGS:
            nr, st = orc.ring_info(NSIDE, i)[:2]
            got.append(gm[:, st:st + nr].ravel())
            ref.append(orc.ring_alm2map(NSIDE, LMAX, alm[b], i).ravel())
    assert rel(np.concatenate(got), np.concatenate(ref)) < 2e-5


def test_tc_map2alm_bench_size_sampled_orders(orc, plan):
    maps = W.random_maps(NSIDE, B, 62)
    a_out = torch.zeros((B, 3, NALM, 2), dtype=torch.float64, device="cuda")
    plan.map2alm(dev(maps), a_out)
    got, ref = [], []
    for b in RHS:
        ga = alm_host(a_out[b:b + 1], (1, 3, -1))[0]
        for m in ORDERS:
            ix = [orc.almidx(LMAX, l, m) for l in range(m, LMAX + 1)]
            got.append(ga[:, ix].ravel())
            ref.append(orc.map2alm_m(NSIDE, LMAX, maps[b], m)[:, m:].ravel())
    assert rel(np.concatenate(got), np.concatenate(ref)) < 2e-5
