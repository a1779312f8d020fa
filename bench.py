"""Benchmark of the dual messenger hot path on GB300.

One *step* is one dual messenger iteration (Algorithm 1) over one batch of
right-hand sides: Legendre analysis + per-l filter, Legendre synthesis, inverse
ring FFT + messenger update + Cauchy norms + forward ring FFT, and the level
control.  The workload is the nside 512 / lmax 1024 batched constrained
realisation configuration: 64 RHS per launch = 32 data maps (Wiener filter) and
32 fluctuation data maps dhat of constrained realisations, one shared mask and
noise map, seeds 100..163, synthetic inputs (analytic spectra, inhomogeneous
noise, band + disk mask).

Metric: DM iterations/s (RHS-iterations per second summed over the batch and
ranks); solves/s derives from it through the iteration count of a solve.
Multi-GPU: replicas only (independent batches per rank, weak scaling).
``--impl reference`` times the FP64 CPU oracle instead (bounded sample).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

# algorithmic FP64 flops per (l, m, ring-pair) triple per RHS per Legendre stage:
# accumulation 10 FMA (20 flops) + recurrence (spin 0: 4, spin +-2: 11) = 35
FLOPS_PER_TRIPLE = 35.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nside", type=int, default=512)
    ap.add_argument("--lmax", type=int, default=None)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="iterations of the plain FP64 GPU path timed beside (0 = skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, n in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def iters_split(k, nlev=10):
    return [k // nlev + (1 if j < k % nlev else 0) for j in range(nlev)]


def kernel_source_hash():
    h = hashlib.sha1()
    for fn in ["dm_legendre.cu", "dm_internal.h"]:
        h.update(open(os.path.join(ROOT, "paper_1801_05358_gb300", "csrc", fn), "rb").read())
    return h.hexdigest()[:12]


def traffic_for(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, null when stale."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        tab = json.load(open(path))
        e = tab.get(f"{kernel}@{workload}")
        if e and e.get("source_hash") == kernel_source_hash():
            return e.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


def cpu_baseline(nside, lmax, wl, d0):
    """The oracle as it stands, one dual messenger iteration of one RHS."""
    from oracle import oracle as O
    cores = os.cpu_count()
    t0 = time.perf_counter()
    O.dm_solve(nside, lmax, wl.cl, wl.sigma, wl.mask, d0, [1.0], forced_iters=[1])
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "DM iterations/s", "cores": cores, "kind": "oracle",
            "sample": f"1 dual messenger iteration of 1 RHS at nside {nside}, lmax {lmax} (FP64, {cores} OpenMP threads)",
            "seconds": dt}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    nside = args.nside
    lmax = args.lmax or 2 * nside
    from oracle import oracle as O
    O.build()
    wl = W.make_workload("nside512", [100], nside=nside, lmax=lmax)
    d0 = wl.data([O.alm2map(nside, lmax, wl.alm_true[0])])[0]
    steps = max(1, min(args.steps, 4))
    warm = min(args.warmup, 1)
    for _ in range(warm):
        O.dm_solve(nside, lmax, wl.cl, wl.sigma, wl.mask, d0, [1.0], forced_iters=[1])
    t0 = time.perf_counter()
    for _ in range(steps):
        O.dm_solve(nside, lmax, wl.cl, wl.sigma, wl.mask, d0, [1.0], forced_iters=[1])
    dt = time.perf_counter() - t0
    v = steps / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": "DM iterations/s", "value": v, "unit": "DM iterations/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": warm, "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"dual messenger WF, nside {nside}, lmax {lmax}, 1 RHS per step (oracle sample)",
                       "nside": nside, "lmax": lmax, "batch": 1, "parallelism": "none (host cores)"},
            "cpu_baseline": {"value": v, "unit": "DM iterations/s", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} dual messenger iterations of 1 RHS at nside {nside}"},
            "e2e": {"value": v, "unit": "DM iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    from paper_1801_05358_gb300 import dmwf

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nside = args.nside
    lmax = args.lmax or 2 * nside
    B = args.batch
    K, Wu = args.steps, max(3, args.warmup)
    npix = 12 * nside * nside
    nwf = B // 2 if B > 1 else 1
    seeds = [100 + b for b in range(B)]

    # ---- inputs: shared spectra, noise and mask; data maps per RHS ----
    wl = W.make_workload("nside512", seeds[:nwf], nside=nside, lmax=lmax)
    plan = dmwf.Plan(nside, lmax, B)
    plan.set_spectra(wl.cl)
    plan.set_noise_mask(wl.sigma, wl.mask)
    prec = dmwf.DM_MIXED_FP32 if args.precision == "mixed" else dmwf.DM_FP64
    nalm = plan.nalm
    d = torch.zeros((B, 3, npix), dtype=torch.float64, device=dev)
    alm_in = torch.zeros((B, 3, nalm, 2), dtype=torch.float64, device=dev)
    for b in range(nwf):
        alm_in[b] = torch.from_numpy(np.ascontiguousarray(wl.alm_true[b]).view(np.float64).reshape(3, nalm, 2))
    s_tmp = torch.zeros_like(d)
    plan.alm2map(alm_in, s_tmp)            # signal maps Y a (product synthesis)
    for b in range(nwf):
        d[b] = (s_tmp[b] + torch.from_numpy(wl.noise[b]).to(dev)) * torch.from_numpy(wl.mask).to(dev)
    if B > nwf:                               # fluctuation data dhat of constrained realisations
        dh = torch.zeros_like(d)
        plan.draw_cr_inputs(seeds, dhat=dh)
        d[nwf:] = dh[nwf:]
    del s_tmp, alm_in
    s_out = torch.zeros_like(d)
    torch.cuda.synchronize()

    # Schedule of a real solve: lambda 1000 -> 1 over 10 levels, Cauchy eps
    # cooled 1e-4 -> 1e-6; the timed steps are iterations of that solve.
    def real_schedule(check):
        plan.set_forced_iters(None)
        plan.set_schedule(lambda0=1000.0, n_levels=10, iters_per_level=0, eps0=1e-4, eps_final=1e-6, eta=0.0,
                          max_iter=1000000, check_every=check)

    # ---- the plain FP64 GPU solve, timed beside (same batch, same API) ----
    fp64_line = None
    if args.fp64_steps > 0 and prec != dmwf.DM_FP64:
        nf = args.fp64_steps
        real_schedule(nf)
        plan.solve_begin(d)
        plan.solve_iterate(1)            # warm
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        f0.record()
        plan.solve_iterate(nf)
        f1.record()
        torch.cuda.synchronize()
        plan.solve_end()
        fms = f0.elapsed_time(f1)
        fp64_line = {"value": B * nf / (fms * 1e-3), "unit": "DM iterations/s", "steps": nf,
                     "ms_per_step": fms / nf}
    plan.set_precision(prec)

    # ---- warm-up: begin a solve and run W iterations through the public API ----
    real_schedule(max(1, K))
    plan.profile_enable(True)
    plan.solve_begin(d)
    plan.solve_iterate(Wu)
    warm_prof = plan.profile_read()
    fp64_peak, fp32_peak = dmwf.measure_alu_peaks()

    # ---- timed: exactly K further iterations of the same solve ----
    plan.profile_enable(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        plan.solve_iterate(K)
        e1.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    prof = plan.profile_read()
    plan.profile_enable(False)
    st, stats = plan.solve_end(s_out)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    iters = prof["iterations"]
    assert iters == K, f"timed {iters} iterations, expected {K}"
    assert stats[0]["iters_total"] == Wu + K, stats[0]["iters_total"]
    value = B * K * ws / (ms_max * 1e-3)
    anchor = None
    if prec != dmwf.DM_FP64:
        ams = warm_prof["ms_anchor"] / max(1, warm_prof["anchors"])
        every = 256
        anchor = {"ms_per_anchor": ams, "anchor_every": every, "anchors_in_timed_window": prof["anchors"],
                  "amortized_value": B * K * ws / ((ms_max - prof["ms_anchor"] + ams * K / every) * 1e-3)}

    # ---- dominant kernel roofline (Legendre stage) ----
    npairs = 2 * nside
    triples = nalm * npairs
    ms_syn = prof["ms_synthesis"] / max(1, prof["iterations"])
    ms_ana = prof["ms_analysis"] / max(1, prof["iterations"])
    suffix = "64" if prec == dmwf.DM_FP64 else "32"
    if ms_syn >= ms_ana:
        kname, kms = "k_leg_syn" + suffix, ms_syn
    else:
        kname, kms = "k_leg_ana" + suffix, ms_ana
    workload_name = f"nside{nside}_lmax{lmax}_B{B}"
    stage = {k: prof[k] / max(1, prof["iterations"]) for k in
             ["ms_analysis", "ms_reduce", "ms_synthesis", "ms_ring", "ms_control"]}
    if prec == dmwf.DM_FP64:
        achieved = FLOPS_PER_TRIPLE * triples * B / (kms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak,
                    "peak_source": "FP64 FMA-chain probe measured live on this GPU (dm_measure_alu_peaks)"}
    else:
        # FP32 contraction from FP32 tables: 20 flops per triple per RHS on the
        # FP32 pipe; the 3 table values per triple are read once per launch.
        flops = 20.0 * triples * B
        tbytes = 12.0 * triples
        ach_f = flops / (kms * 1e-3) / 1e12
        ach_b = tbytes / (kms * 1e-3) / 1e9
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        hbm = peaks.get("hbm_gbs", 6800.0)
        if ach_f / fp32_peak >= ach_b / hbm:
            roofline = {"bound": "alu", "achieved": ach_f, "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": ach_f / fp32_peak,
                        "peak_source": "FP32 FMA-chain probe measured live on this GPU (dm_measure_alu_peaks)"}
        else:
            roofline = {"bound": "hbm", "achieved": ach_b, "peak": hbm, "unit": "GB/s", "frac": ach_b / hbm,
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"}
    roofline.update({"traffic": traffic_for(kname, workload_name), "kernel": kname, "ms_per_launch": kms,
                     "stage_ms_per_iter": stage, "fp64_peak_tflops": fp64_peak, "fp32_peak_tflops": fp32_peak})

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    if not args.no_e2e:
        plan.set_schedule(lambda0=1000.0, n_levels=10, iters_per_level=1, check_every=max(1, K))
        plan.set_forced_iters(iters_split(K))
        d_host = d.cpu().pin_memory()
        s_host = torch.empty_like(d_host).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        plan.wiener_filter_host(d_host, s_host)
        h1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ems = max(h0.elapsed_time(h1), wall * 1e3)
        nbytes = d_host.numel() * 8
        e2e = {"value": B * K / (ems * 1e-3), "unit": "DM iterations/s",
               "h2d_bytes_per_step": nbytes / K, "d2h_bytes_per_step": nbytes / K,
               "note": f"one dm_wiener_filter_host call of {K} iterations (a whole solve: begin, {K} "
                       f"iterations, end); d in and s out once per call"}

    # ---- CPU baseline (oracle), rank 0 at N = 1 only ----
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        cpu = cpu_baseline(nside, lmax, wl, d[0].cpu().numpy())

    if rank == 0:
        line = {"metric": "DM iterations/s", "value": value, "unit": "DM iterations/s", "n_gpus": ws,
                "steps": K, "warmup": Wu, "ms_per_step": ms_max / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == dmwf.DM_FP64 else "f32+f64",
                "data": "synthetic",
                "config": {"workload": f"batched constrained realisations nside {nside} lmax {lmax}: "
                                       f"{nwf} WF + {B - nwf} fluctuation RHS per launch (seeds 100..{99 + B})",
                           "nside": nside, "lmax": lmax, "batch": B, "precision": args.precision,
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                           "l2": "inputs larger than L2 (maps and ring coefficients exceed 129 MB)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": prof["launches"],
                "fp64_gpu": fp64_line, "refinement": anchor,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
