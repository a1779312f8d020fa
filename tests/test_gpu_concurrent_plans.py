"""Plans driven concurrently from several host threads, each on its own CUDA
stream: every solve completes and equals the same solve run alone.

A plan's kernels take per-launch dynamic shared memory whose size depends on
the plan (ring sizes, tensor-core stages); the limit that admits it is a
process-wide attribute of the kernel, so plans of different sizes running at
once must not undo each other's limit.  The mixed plans anchor every 8
iterations, so their float-float and FP64 stages interleave with the other
plans' iterations."""
import threading

import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import dev, make_plan, rel

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


def _plan(orc, nside, lmax, B, prec, seed0):
    wl = W.make_workload("nside16", list(range(seed0, seed0 + B)), nside=nside, lmax=lmax)
    d = dev(_data(orc, wl))
    p = make_plan(wl, B, lambda0=1000.0, n_levels=3, iters_per_level=8)
    p.set_precision(prec)
    if prec == dmwf.DM_MIXED_FP32:
        p.set_tensor_cores(True)
        p.set_refinement(8)
    s = torch.zeros((B, 3, wl.npix), dtype=torch.float64, device="cuda")
    return wl, p, d, s


def test_concurrent_plans_match_solo(orc):
    cases = [(64, 128, 8, dmwf.DM_MIXED_FP32, 300), (128, 256, 8, dmwf.DM_MIXED_FP32, 400),
             (32, 64, 2, dmwf.DM_FP64, 500)]
    plans = [_plan(orc, *c) for c in cases]
    solo = []
    for wl, p, d, s in plans:
        p.wiener_filter(d, s)
        torch.cuda.synchronize()
        solo.append(s.cpu().numpy().copy())
    # the nside 64 plan against the oracle (RHS 0, same forced counts)
    wl0, _, d0, _ = plans[0]
    ref = orc.dm_solve(wl0.nside, wl0.lmax, wl0.cl, wl0.sigma, wl0.mask, d0[0].cpu().numpy(),
                       W.lambda_schedule(1000.0, 3), forced_iters=[8] * 3)
    assert rel(solo[0][0], ref["s"]) < 1e-5

    outs = [[torch.zeros_like(s) for _ in range(3)] for _, _, _, s in plans]
    errors = []
    start = threading.Barrier(len(plans))

    def work(i):
        wl, p, d, _ = plans[i]
        st = torch.cuda.Stream()
        try:
            start.wait()
            for rep in range(3):
                p.wiener_filter(d, outs[i][rep], stream=st)
            st.synchronize()
        except Exception as e:  # reported below with the plan it came from
            errors.append((i, repr(e)))

    th = [threading.Thread(target=work, args=(i,)) for i in range(len(plans))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for i, (wl, p, d, s) in enumerate(plans):
        for rep in range(3):
            got = outs[i][rep].cpu().numpy()
            assert np.all(np.isfinite(got)), (i, rep)
            assert rel(got, solo[i]) < 1e-6, (i, rep, rel(got, solo[i]))
        p.close()
