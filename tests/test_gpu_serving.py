"""Per-RHS noise models and the continuous-batching server (dm_serve_*).

- every RHS of a plan can carry its own noise and mask;
- served Wiener filters and constrained realisations of two geometries match
  the oracle run alone (FP64, relative L2 <= 1e-10, same iteration count);
- each result is bit-identical alone and in the mix (FP64 and mixed mode);
- queue bound, cancellation and a budget that can never fit are reported;
- requests tighter than the strict tolerance are routed to FP64-class pools."""
import time

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


def test_per_rhs_noise(orc):
    w1 = W.make_workload("nside16", [1], nside=8, lmax=16)
    w2 = W.make_workload("nside16", [2], nside=8, lmax=16)
    d = np.stack([_data(orc, w1)[0], _data(orc, w2)[0]])
    p = make_plan(w1, 2, lambda0=100.0, n_levels=3, iters_per_level=5)
    p.set_noise_mask_rhs(1, w2.sigma, w2.mask)
    s = torch.zeros((2, 3, w1.npix), dtype=torch.float64, device="cuda")
    p.wiener_filter(dev(d), s)
    lam = W.lambda_schedule(100.0, 3)
    for b, wl in enumerate([w1, w2]):
        ref = orc.dm_solve(wl.nside, wl.lmax, wl.cl, wl.sigma, wl.mask, d[b], lam, forced_iters=[5, 5, 5])
        assert rel(s.cpu().numpy()[b], ref["s"]) < 1e-10


def _requests(orc):
    """Four WF and two CR requests over nside 8 / lmax 16 and nside 16 / lmax 32."""
    reqs = []
    for i, (ns, lm, kind, tol) in enumerate([(8, 16, 0, 1e-5), (16, 32, 0, 1e-5), (8, 16, 1, 1e-5),
                                             (8, 16, 0, 1e-6), (16, 32, 1, 1e-5), (8, 16, 0, 1e-5)]):
        wl = W.make_workload("nside16", [40 + i], nside=ns, lmax=lm)
        d = _data(orc, wl)[0]
        reqs.append(dict(nside=ns, lmax=lm, kind=kind, tol=tol, cl=wl.cl, sigma=wl.sigma, mask=wl.mask, d=d,
                         seed=900 + i))
    return reqs


def _serve(reqs, prec, slots=3, n=16):
    srv = dmwf.Server(8 << 30, slots_per_plan=slots, iters_per_round=n, prec=prec)
    tickets = [srv.submit(r["nside"], r["lmax"], r["kind"], r["tol"], r["cl"], r["sigma"], r["d"], r["mask"],
                          r["seed"]) for r in reqs]
    out = {}
    t0 = time.time()
    while len(out) < len(tickets) and time.time() - t0 < 600:
        for t in tickets:
            if t not in out:
                got = srv.poll(t)
                if got is not None:
                    out[t] = got
        time.sleep(0.01)
    srv.close()
    assert len(out) == len(tickets)
    return [out[t] for t in tickets]


def test_serving_matches_oracle_and_alone(orc):
    reqs = _requests(orc)
    mix = _serve(reqs, dmwf.DM_FP64)
    for r, (res, s) in zip(reqs, mix):
        assert res["status"] == 0
        lam = W.lambda_schedule(1000.0, 10)
        eps = W.eps_schedule(10, 1e-4, r["tol"])
        if r["kind"] == 0:
            ref = orc.dm_solve(r["nside"], r["lmax"], r["cl"], r["sigma"], r["mask"], r["d"], lam, eps=eps)
            s_ref = ref["s"]
        else:
            ref = orc.constrained_realization(r["nside"], r["lmax"], r["cl"], r["sigma"], r["mask"], r["d"],
                                              r["seed"], lam, eps=eps)
            s_ref = ref["s_cr"]
        assert res["iters"] == ref["iters"]
        assert rel(s, s_ref) < 1e-10
    # alone: the same request through a server holding nothing else
    for r, (res, s) in list(zip(reqs, mix))[:3]:
        (res1, s1), = _serve([r], dmwf.DM_FP64, slots=1, n=7)
        assert res1["iters"] == res["iters"]
        assert np.array_equal(s1, s)


def test_serving_mixed_alone_equals_mix(orc):
    reqs = _requests(orc)[:4]
    mix = _serve(reqs, dmwf.DM_MIXED_FP32, slots=2, n=16)
    for r, (res, s) in zip(reqs, mix):
        (res1, s1), = _serve([r], dmwf.DM_MIXED_FP32, slots=1, n=16)
        assert res1["iters"] == res["iters"]
        assert np.array_equal(s1, s)


def test_serving_queue_bound_cancel_and_budget(orc):
    r = _requests(orc)[1]
    srv = dmwf.Server(8 << 30, slots_per_plan=1, iters_per_round=4, prec=dmwf.DM_FP64, max_pending=2)
    tickets, busy = [], 0
    for _ in range(8):
        try:
            tickets.append(srv.submit(r["nside"], r["lmax"], r["kind"], r["tol"], r["cl"], r["sigma"], r["d"],
                                      r["mask"]))
        except dmwf.DmError as e:
            assert e.status == dmwf.DM_EBUSY
            busy += 1
    assert busy >= 1
    # a mask with no observed pixel is refused at submission
    with pytest.raises(dmwf.DmError) as e:
        srv.submit(r["nside"], r["lmax"], r["kind"], r["tol"], r["cl"], r["sigma"], r["d"],
                   np.zeros_like(np.asarray(r["mask"], dtype=np.uint8)))
    assert e.value.status == dmwf.DM_EINVAL
    cancelled = [t for t in tickets if srv.cancel(t) == dmwf.DM_OK]
    assert cancelled
    for t in cancelled:
        got = None
        while got is None:
            got = srv.poll(t)
        assert got[0]["status"] == dmwf.DM_EAGAIN
    srv.close()
    # a budget no pool can ever fit
    srv = dmwf.Server(1 << 20, slots_per_plan=1, iters_per_round=4, prec=dmwf.DM_FP64)
    t = srv.submit(r["nside"], r["lmax"], r["kind"], r["tol"], r["cl"], r["sigma"], r["d"], r["mask"])
    got = None
    t0 = time.time()
    while got is None and time.time() - t0 < 60:
        got = srv.poll(t)
        time.sleep(0.01)
    assert got is not None and got[0]["status"] == dmwf.DM_ENOMEM
    srv.close()


def test_serving_routes_strict_tolerance_to_float_float(orc):
    """A mixed-mode server with strict_tol 1e-6: the 1e-7 request runs in a
    float-float pool and meets the FP64 bar against the oracle (same
    iteration count); the 1e-5 request runs in a mixed pool."""
    reqs = []
    for i, tol in enumerate([1e-5, 1e-7]):
        wl = W.make_workload("nside16", [60 + i], nside=8, lmax=16)
        reqs.append(dict(nside=8, lmax=16, kind=0, tol=tol, cl=wl.cl, sigma=wl.sigma, mask=wl.mask,
                         d=_data(orc, wl)[0]))
    srv = dmwf.Server(8 << 30, slots_per_plan=2, iters_per_round=16, prec=dmwf.DM_MIXED_FP32, strict_tol=1e-6,
                      strict_prec=dmwf.DM_FLOAT_FLOAT)
    tickets = [srv.submit(r["nside"], r["lmax"], r["kind"], r["tol"], r["cl"], r["sigma"], r["d"], r["mask"])
               for r in reqs]
    out = {}
    t0 = time.time()
    while len(out) < 2 and time.time() - t0 < 600:
        for t in tickets:
            if t not in out:
                got = srv.poll(t)
                if got is not None:
                    out[t] = got
        time.sleep(0.01)
    info = srv.info()
    srv.close()
    assert len(out) == 2 and info["pools"] == 2
    (res_m, _), (res_f, s_f) = out[tickets[0]], out[tickets[1]]
    assert res_m["status"] == 0 and res_f["status"] == 0
    r = reqs[1]
    lam = W.lambda_schedule(1000.0, 10)
    ref = orc.dm_solve(r["nside"], r["lmax"], r["cl"], r["sigma"], r["mask"], r["d"], lam,
                       eps=W.eps_schedule(10, 1e-4, r["tol"]))
    assert res_f["iters"] == ref["iters"]
    assert rel(s_f, ref["s"]) < 1e-9


def test_server_rejects_mixed_strict_precision():
    with pytest.raises(dmwf.DmError):
        dmwf.Server(1 << 30, prec=dmwf.DM_MIXED_FP32, strict_tol=1e-6, strict_prec=dmwf.DM_MIXED_FP32)
