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
The mixed mode re-anchors in FP64-class arithmetic every 256 iterations; the
default timed window is exactly one such period (256 iterations, one anchor
inside), so ``value`` is the whole-job throughput of a long solve.  For other
--steps the anchor cost is prorated from the anchors measured in the run.
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

ANCHOR_EVERY = 256

# algorithmic FP64 flops per (l, m, ring-pair) triple per RHS per Legendre stage:
# accumulation 10 FMA (20 flops) + recurrence (spin 0: 4, spin +-2: 11) = 35
FLOPS_PER_TRIPLE = 35.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=256)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nside", type=int, default=512)
    ap.add_argument("--lmax", type=int, default=None)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=10,
                    help="iterations of the plain FP64 GPU path timed beside (0 = skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-solve", action="store_true",
                    help="skip the whole-solve leg of the default run (WF solves/s to --solve-leg-tol)")
    ap.add_argument("--solve-leg-tol", type=float, default=1e-5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ring-radix", type=int, default=None, choices=[0, 3, 4],
                    help="ring transforms of radix 2^k (3 or 4), 0 = generic kernels (default: autotuned)")
    ap.add_argument("--tc-tiles", default="auto", choices=["auto", "stored", "generated"],
                    help="tensor-core Legendre operand: stored tiles, generated in the kernels, or by size")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch heuristics instead of dm_autotune's picks")
    ap.add_argument("--tuning", default=None,
                    help="JSON of launch picks (a bench line's autotune object) applied instead of tuning")
    ap.add_argument("--solve-tol", type=float, default=None,
                    help="run whole solves to this final Cauchy threshold and report WF solves/s instead")
    ap.add_argument("--solve-max-iter", type=int, default=200000)
    ap.add_argument("--progressive", type=float, default=0.0,
                    help="whole solves with the progressive working resolution of this margin (0 = off)")
    ap.add_argument("--flat", type=int, default=0,
                    help="time the paper's own flat-sky setting on an N x N grid instead (e.g. 1024)")
    ap.add_argument("--serve", action="store_true", help="run a sample of the serving mix instead")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-warm", type=int, default=12)
    ap.add_argument("--serve-nsides", default="64,128")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-max-iter", type=int, default=30000)
    ap.add_argument("--serve-budget-gb", type=float, default=200.0)
    ap.add_argument("--serve-seed", type=int, default=4)
    return ap.parse_args()


def max_over_ranks(vals, device, ws):
    """Element-wise maximum of per-rank timings over all ranks (all_reduce MAX
    on the rank's device; identity for a single rank)."""
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_value(batch, steps, ws, ms):
    """RHS-iterations of every rank divided by the slowest rank's time."""
    return batch * steps * ws / (ms * 1e-3)


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


# source files that define each timed kernel (a stored ncu traffic figure is
# used only while they are unchanged)
KERNEL_SOURCES = {
    "k_ring_iter": ["dm_ring.cu", "dm_fft.cuh"],
    "k_leg_syn64": ["dm_legendre.cu", "dm_rec.cuh"],
    "k_leg_ana64": ["dm_legendre.cu", "dm_rec.cuh"],
    "k_syn_tc": ["dm_legendre_tc.cu", "dm_tc.cuh", "dm_tc_tiles.cuh"],
    "k_ana_tc": ["dm_legendre_tc.cu", "dm_tc.cuh", "dm_tc_tiles.cuh"],
    "k_reduce": ["dm_legendre.cu"],
}


def kernel_source_hash(kernel):
    h = hashlib.sha1()
    for fn in KERNEL_SOURCES.get(kernel, ["dm_legendre.cu"]):
        h.update(open(os.path.join(ROOT, "paper_1801_05358_gb300", "csrc", fn), "rb").read())
    return h.hexdigest()[:12]


def traffic_for(kernel, workload):
    """DRAM bytes per timed unit from the committed ncu summary, null when stale."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        tab = json.load(open(path))
        e = tab.get(f"{kernel}@{workload}")
        if e and e.get("source_hash") == kernel_source_hash(kernel):
            return e.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


ORACLE_ITERS = 3


def oracle_data(O, nside, lmax, wl):
    """Data map of RHS 0 made on the host: the oracle's synthesis of the drawn
    signal plus the drawn noise, masked (no value from the CUDA path)."""
    return wl.data([O.alm2map(nside, lmax, wl.alm_true[0])])[0]


def timed_single_steps(plan, d, nf, torch):
    """Median device time (ms) of nf iterations, each timed on its own with
    CUDA events after one warm-up iteration of the session."""
    plan.solve_begin(d)
    plan.solve_iterate(1)            # warm
    times = []
    for _ in range(nf):
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        f0.record()
        plan.solve_iterate(1)
        f1.record()
        torch.cuda.synchronize()
        times.append(f0.elapsed_time(f1))
    plan.solve_end()
    return float(np.median(times))


SINGLE_THREAD_SAMPLE = """
import sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import oracle as O
O.build()
wl = W.make_workload("nside512", [100], nside={ns}, lmax={lm})
d0 = wl.data([O.alm2map({ns}, {lm}, wl.alm_true[0])])[0]
best = None
for _ in range(2):
    t0 = time.perf_counter()
    O.dm_solve({ns}, {lm}, wl.cl, wl.sigma, wl.mask, d0, [1.0], forced_iters=[1])
    dt = time.perf_counter() - t0
    best = dt if best is None else min(best, dt)
print(best)
"""


def single_thread_baseline(nside, lmax):
    """The oracle on one host core (OMP_NUM_THREADS=1), the paper's own setting:
    one dual messenger iteration of one RHS at nside / 4 (best of two), timed
    in a child process, and its time scaled to nside by the ratio of
    (l, m, ring pair) triples, which sets the oracle's cost (a stated
    extrapolation: a full single-core iteration at nside 512 takes minutes)."""
    import subprocess
    ns, lm = max(16, nside // 4), max(32, lmax // 4)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", SINGLE_THREAD_SAMPLE.format(root=ROOT, ns=ns, lm=lm)],
                             env=env, capture_output=True, text=True, timeout=300)
        t = float(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the all-core baseline stands
        return {"error": str(e)[:200]}
    def triples(n, l):
        return (l + 1) * (l + 2) // 2 * 2 * n
    scale = triples(nside, lmax) / triples(ns, lm)
    return {"cores": 1, "sample": f"1 dual messenger iteration of 1 RHS at nside {ns}, lmax {lm} (best of 2, "
                                  f"OMP_NUM_THREADS=1)", "seconds_per_iteration_sample": t,
            "value_extrapolated": 1.0 / (t * scale), "unit": "DM iterations/s",
            "extrapolation": f"x {scale:.1f} (l, m, ring pair) triples to nside {nside}, lmax {lmax}"}


def cpu_baseline(nside, lmax, wl, d0):
    """The oracle as it stands: ORACLE_ITERS dual messenger iterations of one
    RHS at lambda = 1 (a bounded sample of the workload).  Its map is also the
    reference of the bench line's error_vs_oracle."""
    from oracle import oracle as O
    cores = os.cpu_count()
    t0 = time.perf_counter()
    ref = O.dm_solve(nside, lmax, wl.cl, wl.sigma, wl.mask, d0, [1.0], forced_iters=[ORACLE_ITERS])
    dt = time.perf_counter() - t0
    return {"value": ORACLE_ITERS / dt, "unit": "DM iterations/s", "cores": cores, "kind": "oracle",
            "sample": f"{ORACLE_ITERS} dual messenger iterations of 1 RHS at nside {nside}, lmax {lmax}, lambda 1 "
                      f"(FP64, {cores} OpenMP threads)",
            "seconds": dt, "single_thread": single_thread_baseline(nside, lmax)}, ref


def error_vs_oracle(plan, d, d0, ref, prec, torch):
    """The same ORACLE_ITERS iterations on the GPU in the bench's own launch
    configuration (the whole batch, its precision and kernels), with RHS 0
    holding the host-made data d0: relative L2 error of RHS 0's map and
    coefficients against the oracle, plus the device diagnostics."""
    from paper_1801_05358_gb300 import dmwf
    dd = d.clone()
    dd[0] = torch.from_numpy(d0).to(d.device)
    plan.set_forced_iters(None)
    plan.set_schedule(lambda0=1.0, n_levels=1, iters_per_level=ORACLE_ITERS, check_every=ORACLE_ITERS)
    s = torch.zeros_like(dd)
    a = torch.zeros((d.shape[0], 3, plan.nalm, 2), dtype=torch.float64, device=d.device)
    st, stats = plan.wiener_filter(dd, s, a)
    torch.cuda.synchronize()
    s0 = s[0].cpu().numpy()
    a0 = a[0].cpu().numpy().view(np.complex128)[..., 0]
    e_s = float(np.linalg.norm(s0 - ref["s"]) / np.linalg.norm(ref["s"]))
    e_a = float(np.linalg.norm(a0 - ref["alm"]) / np.linalg.norm(ref["alm"]))
    out = {"rel_l2_map": e_s, "rel_l2_alm": e_a, "rhs": 0, "iterations": ORACLE_ITERS, "lambda": 1.0,
           "bar": 1e-5 if prec != dmwf.DM_FP64 else 1e-10,
           "note": "the bench's plan, batch and precision; RHS 0's data made on the host by the oracle's synthesis"}
    for k in ("true_resid", "chi2"):
        if k in stats[0]:
            out["gpu_" + k] = stats[0][k]
    return out


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    nside = args.nside
    lmax = args.lmax or 2 * nside
    from oracle import oracle as O
    O.build()
    wl = W.make_workload("nside512", [100], nside=nside, lmax=lmax)
    d0 = oracle_data(O, nside, lmax, wl)
    steps = max(1, min(args.steps, 4))
    warm = min(args.warmup, 1)
    for _ in range(warm):
        O.dm_solve(nside, lmax, wl.cl, wl.sigma, wl.mask, d0, [1.0], forced_iters=[1])
    t0 = time.perf_counter()
    O.dm_solve(nside, lmax, wl.cl, wl.sigma, wl.mask, d0, [1.0], forced_iters=[steps])
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


def bench_inputs(dmwf, torch, dev, nside, lmax, B):
    """The batched constrained-realisation workload: one plan with the shared
    spectra, noise and mask; B // 2 data maps d = Y a + n (Wiener filter) and
    B - B // 2 fluctuation data maps dhat, seeds 100 .. 99 + B."""
    npix = 12 * nside * nside
    nwf = B // 2 if B > 1 else 1
    seeds = [100 + b for b in range(B)]
    wl = W.make_workload("nside512", seeds[:nwf], nside=nside, lmax=lmax)
    plan = dmwf.Plan(nside, lmax, B)
    plan.set_spectra(wl.cl)
    plan.set_noise_mask(wl.sigma, wl.mask)
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
    torch.cuda.synchronize()
    return plan, wl, d


def run_solves(args):
    """Whole solves of the batch, lambda 1000 -> 1 over 10 levels with the
    Cauchy threshold cooled from 1e-4 to --solve-tol, through dm_wiener_filter
    (the call a user makes): WF solves/s = B / the device time of the call."""
    import torch

    from paper_1801_05358_gb300 import dmwf

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    nside, B = args.nside, args.batch
    lmax = args.lmax or 2 * nside
    plan, wl, d = bench_inputs(dmwf, torch, dev, nside, lmax, B)
    prec = dmwf.DM_MIXED_FP32 if args.precision == "mixed" else dmwf.DM_FP64
    plan.set_tc_tiles({"auto": None, "stored": False, "generated": True}[args.tc_tiles])
    plan.set_precision(prec)
    if args.progressive > 0:
        plan.set_progressive(args.progressive, 8)
    tol = args.solve_tol
    s_out = torch.zeros_like(d)
    # warm-up: tables and first-use allocations, 3 iterations
    plan.set_schedule(lambda0=1000.0, n_levels=10, iters_per_level=0, eps0=1e-4, eps_final=tol, eta=0.0,
                      max_iter=args.solve_max_iter, check_every=64)
    plan.solve_begin(d)
    plan.solve_iterate(3)
    plan.solve_end()
    plan.profile_enable(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0.record(stream)
        st, stats = plan.wiener_filter(d, s_out)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = plan.profile_read()
    levels = plan.progressive_levels(10) if args.progressive > 0 else None
    plan.close()
    its = np.array([x["iters_total"] for x in stats])
    conv = int(sum(1 for x in stats if x["iters_total"] < args.solve_max_iter))
    per_level = np.array([x["iters_per_level"][:10] for x in stats]).mean(axis=0).tolist()
    line = {"metric": "WF solves/s", "value": B / (ms * 1e-3), "unit": "solves/s", "n_gpus": 1, "steps": 1,
            "warmup": 3, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == dmwf.DM_FP64 else "f32 (bf16x3 tensor-core Legendre, f64 harmonic state)",
            "data": "synthetic",
            "config": {"workload": f"whole solves of the batched constrained realisations, nside {nside} lmax {lmax}, "
                                   f"{B} RHS, lambda 1000 -> 1 in 10 levels, Cauchy 1e-4 -> {tol:g}",
                       "nside": nside, "lmax": lmax, "batch": B, "precision": args.precision, "tol": tol},
            "iterations_per_rhs": {"mean": float(its.mean()), "min": int(its.min()), "max": int(its.max())},
            "mean_iterations_per_level": per_level, "progressive_margin": args.progressive,
            "level_resolutions": levels,
            "true_resid": {"mean": float(np.mean([x["true_resid"] for x in stats])),
                           "max": float(np.max([x["true_resid"] for x in stats]))},
            "converged_rhs": conv, "dm_iterations_per_s": float(its.sum()) / (ms * 1e-3),
            "anchors": prof["anchors"], "gpu_launches": prof["launches"], "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_flat(args):
    """The paper's own flat-sky setting (Section 3.1): N x N grid of a 10 deg
    patch, batch of RHS, FP64, the dual messenger iteration timed in the
    middle of a lambda 1000 -> 1 schedule through the session API.  The
    paper's single i5-4690 core took 0.38 to 2.0 s per iteration at 1024^2
    (Table 1), quoted as context only (other hardware, CAMB spectra)."""
    import torch

    from paper_1801_05358_gb300 import dmwf

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N, B = args.flat, args.batch
    K, Wu = args.steps, max(3, args.warmup)
    seeds = list(range(200, 200 + B))
    wl = W.make_flat_workload(seeds, N=N)
    plan = dmwf.FlatPlan(N, wl.L, B)
    plan.set_spectra(wl.S)
    plan.set_noise(wl.sigma.reshape(3, -1), wl.mask_t.ravel(), wl.mask_p.ravel())
    alm = torch.from_numpy(np.ascontiguousarray(np.stack([np.swapaxes(a[:, :, :N // 2], -1, -2)
                                                          for a in wl.alm_true])).view(np.float64)).to(dev)
    s_sig = torch.zeros((B, 3, N * N), dtype=torch.float64, device=dev)
    plan.alm2map(alm, s_sig)  # the signal maps, the plan's own synthesis
    obs = torch.from_numpy(np.stack([wl.mask_t, wl.mask_p, wl.mask_p]).reshape(3, -1).astype(np.float64)).to(dev)
    noise = torch.from_numpy(np.stack(wl.noise).reshape(B, 3, -1)).to(dev)
    d = (s_sig + noise) * obs[None]
    del s_sig, noise, alm
    plan.set_schedule(lambda0=1000.0, n_levels=10, iters_per_level=0, eps0=1e-4, eps_final=1e-6, eta=0.0,
                      max_iter=1000000, check_every=max(1, K))
    plan.solve_begin(d)
    plan.solve_iterate(Wu)
    plan.profile_enable(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0.record(stream)
        plan.solve_iterate(K)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = plan.profile_read()
    plan.solve_end()
    plan.close()
    its = max(1, prof["iterations"])
    stage = {k: prof[k] / its for k in ["ms_analysis", "ms_reduce", "ms_synthesis", "ms_ring", "ms_control"]}
    line = {"metric": "DM iterations/s (flat sky)", "value": B * K / (ms * 1e-3), "unit": "DM iterations/s",
            "n_gpus": 1, "steps": K, "warmup": Wu, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"flat-sky dual messenger WF, {N}x{N} grid of a 10 deg patch, {B} RHS, "
                                   f"distinct T/P masks (fsky 0.78 / 0.82), lambda 1000 -> 1 in 10 levels",
                       "N": N, "batch": B, "precision": "fp64"},
            "seconds_per_rhs_iteration": ms * 1e-3 / (K * B),
            "paper_cpu_seconds_per_iteration": {"value": [2.0, 0.52, 0.38], "hardware": "1 core i5-4690 3.5 GHz",
                                                "workload": "1024^2 flat patch, CAMB spectra, correlated noise",
                                                "source": "Table 1 (minutes / iterations at eps 1e-4, 1e-5, 1e-6)"},
            "stage_ms_per_iter": stage, "gpu_launches": prof["launches"], "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """A sample of the serving mix through dm_serve_submit / dm_serve_poll:
    requests drawn by workloads.serving_stream (nside from --serve-nsides,
    lmax = 2 nside, 70 % Wiener filter / 30 % constrained realisation,
    tolerance 1e-5 or 1e-8, per-request seeds), the 1e-8 ones in float-float
    pools.  A closed-loop pass over the first --serve-warm requests measures
    the capacity; the rest then arrive as a Poisson stream at 0.8 x that
    capacity.  Reports solves/s and the p50 / p99 submit-to-result latency
    of the Poisson phase."""
    import torch

    from paper_1801_05358_gb300 import dmwf

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    nsides = [int(x) for x in args.serve_nsides.split(",")]
    reqs = W.serving_stream(args.serve_requests, args.serve_seed, nsides=nsides)
    # inputs of every request: its own mask, noise, signal and data map
    synth = {}
    for r in reqs:
        wl = W.make_workload("nside16", [r["seed"]], nside=r["nside"], lmax=r["lmax"])
        if r["nside"] not in synth:
            synth[r["nside"]] = dmwf.Plan(r["nside"], r["lmax"], 1)
        nalm = synth[r["nside"]].nalm
        a = torch.from_numpy(np.ascontiguousarray(wl.alm_true[0]).view(np.float64).reshape(1, 3, nalm, 2)).to(dev)
        m = torch.zeros((1, 3, 12 * r["nside"] ** 2), dtype=torch.float64, device=dev)
        synth[r["nside"]].alm2map(a, m)
        r.update(cl=wl.cl, sigma=wl.sigma, mask=wl.mask, d=wl.data([m[0].cpu().numpy()])[0])
    for p in synth.values():
        p.close()
    torch.cuda.synchronize()
    srv = dmwf.Server(int(args.serve_budget_gb * (1 << 30)), slots_per_plan=args.serve_slots, iters_per_round=16,
                      prec=dmwf.DM_MIXED_FP32, max_iter=args.serve_max_iter, strict_tol=1e-6,
                      strict_prec=dmwf.DM_FLOAT_FLOAT)

    def submit(r):
        return srv.submit(r["nside"], r["lmax"], r["kind"], r["tol"], r["cl"], r["sigma"], r["d"], r["mask"],
                          r["seed"])

    def drain(live, results):
        for t in list(live):
            got = srv.poll(t)
            if got is not None:
                results[t] = (got[0], time.perf_counter())
                live.discard(t)

    nw = min(args.serve_warm, len(reqs))
    warm, rest = reqs[:nw], reqs[nw:]
    # closed loop: all warm requests at once
    t0 = time.perf_counter()
    live, res_w = {submit(r) for r in warm}, {}
    while live:
        drain(live, res_w)
        time.sleep(0.002)
    t_warm = time.perf_counter() - t0
    capacity = nw / t_warm
    rate = 0.8 * capacity
    arr = W.poisson_arrivals(len(rest), rate, args.serve_seed + 1)
    res, live, tick = {}, set(), {}
    t0 = time.perf_counter()
    with ClockSampler(0) as clk:
        i = 0
        while i < len(rest) or live:
            now = time.perf_counter() - t0
            while i < len(rest) and arr[i] <= now:
                t = submit(rest[i])
                tick[t] = rest[i]
                live.add(t)
                i += 1
            drain(live, res)
            time.sleep(0.001)
    t_all = time.perf_counter() - t0
    info = srv.info()
    srv.close()
    lat = np.array([r[0]["latency_ms"] for r in res.values()])
    qms = np.array([r[0]["queue_ms"] for r in res.values()])
    st = [r[0]["status"] for r in res.values()]
    its = np.array([r[0]["iters"] for r in res.values()])
    by = {}
    for t, (r0, _) in res.items():
        q = tick[t]
        k = f"nside{q['nside']}_tol{q['tol']:g}"
        by.setdefault(k, []).append(r0["latency_ms"])
    ok = sum(1 for x in st if x == 0)
    line = {"metric": "WF solves/s (serving)", "value": len(res) / t_all, "unit": "solves/s", "n_gpus": 1,
            "steps": len(res), "warmup": nw, "ms_per_step": t_all * 1e3 / max(1, len(res)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 mixed pools (tol 1e-5), float-float pools (tol 1e-8)", "data": "synthetic",
            "config": {"workload": f"serving mix sample: {len(reqs)} requests, nside in {nsides}, lmax = 2 nside, "
                                   f"70 % WF / 30 % CR, tol 1e-5 or 1e-8, Poisson arrivals at 0.8 x capacity",
                       "slots_per_pool": args.serve_slots, "max_iter": args.serve_max_iter,
                       "hbm_budget_gb": args.serve_budget_gb},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "queue_ms": {"p50": float(np.percentile(qms, 50)), "p99": float(np.percentile(qms, 99))},
            "latency_p50_ms_by_class": {k: float(np.percentile(v, 50)) for k, v in sorted(by.items())},
            "capacity_closed_loop": capacity, "arrival_rate": rate,
            "status": {"ok": ok, "not_converged": sum(1 for x in st if x == 4), "other": len(st) - ok -
                       sum(1 for x in st if x == 4)},
            "iterations": {"mean": float(its.mean()), "max": int(its.max())},
            "server": info, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.solve_tol is not None:
        return run_solves(args)
    if args.serve:
        return run_serve(args)
    if args.flat:
        return run_flat(args)
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

    plan, wl, d = bench_inputs(dmwf, torch, dev, nside, lmax, B)
    nalm = plan.nalm
    prec = dmwf.DM_MIXED_FP32 if args.precision == "mixed" else dmwf.DM_FP64
    if args.ring_radix is not None:
        plan.set_ring_radix(args.ring_radix)
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
        fms = timed_single_steps(plan, d, nf, torch)
        fp64_line = {"value": B / (fms * 1e-3), "unit": "DM iterations/s", "steps": nf,
                     "ms_per_step": fms, "note": f"median of {nf} single timed iterations"}
    # ---- the float-float Legendre path (FP64-class results on the FP32 pipe) ----
    ff_line = None
    if args.fp64_steps > 0 and prec != dmwf.DM_FP64:
        nf = args.fp64_steps
        plan.set_precision(dmwf.DM_FLOAT_FLOAT)
        real_schedule(nf)
        fms = timed_single_steps(plan, d, nf, torch)
        ff_line = {"value": B / (fms * 1e-3), "unit": "DM iterations/s", "steps": nf,
                   "ms_per_step": fms, "precision": "DM_FLOAT_FLOAT",
                   "note": f"median of {nf} single timed iterations"}
    plan.set_tc_tiles({"auto": None, "stored": False, "generated": True}[args.tc_tiles])
    plan.set_precision(prec)
    tuning = None
    if args.tuning:
        plan.set_tuning(json.loads(open(args.tuning).read() if os.path.exists(args.tuning) else args.tuning))
        tuning = plan.tuning()
        tuning["source"] = "applied (--tuning)"
    elif args.ring_radix is None and not args.no_autotune:
        t0 = time.perf_counter()
        tuning = plan.autotune()
        tuning["seconds"] = time.perf_counter() - t0

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
    # the K steps run as up to 16 equal chunks with an event pair each, for
    # the median over chunks beside the total
    nch = max(1, min(16, K))
    sizes = [K // nch + (1 if j < K % nch else 0) for j in range(nch)]
    cev = [torch.cuda.Event(enable_timing=True) for _ in range(nch + 1)]
    with ClockSampler(local) as clk:
        e0.record(stream)
        cev[0].record(stream)
        for j, n in enumerate(sizes):
            plan.solve_iterate(n)
            cev[j + 1].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    chunk_ms = [cev[j].elapsed_time(cev[j + 1]) / sizes[j] for j in range(nch)]
    prof = plan.profile_read()
    plan.profile_enable(False)
    st, stats = plan.solve_end(s_out)
    iters = prof["iterations"]
    assert iters == K, f"timed {iters} iterations, expected {K}"
    assert stats[0]["iters_total"] == Wu + K, stats[0]["iters_total"]
    ams, every, local_whole = 0.0, ANCHOR_EVERY, ms
    if prec != dmwf.DM_FP64:
        n_anch = warm_prof["anchors"] + prof["anchors"]
        ams = (warm_prof["ms_anchor"] + prof["ms_anchor"]) / max(1, n_anch)
        local_whole = ms - prof["ms_anchor"] + ams * K / every
    ms_max, whole_ms = max_over_ranks([ms, local_whole], dev, ws)
    raw_value = whole_job_value(B, K, ws, ms_max)
    value = whole_job_value(B, K, ws, whole_ms)
    anchor = None
    if prec != dmwf.DM_FP64:
        anchor = {"ms_per_anchor": ams, "anchor_every": every, "anchors_in_timed_window": prof["anchors"],
                  "timed_window_value": raw_value,
                  "steady_value_between_anchors": B * K * ws / ((ms_max - prof["ms_anchor"]) * 1e-3),
                  "note": "value = K iterations plus K/anchor_every of a measured anchor; with the default "
                          "K = anchor_every the window holds exactly one anchor and value = timed_window_value"}

    # ---- rooflines of the four stages; the dominant one is reported ----
    npairs = 2 * nside
    nrings = 4 * nside - 1
    mmax = lmax
    triples = nalm * npairs
    its = max(1, prof["iterations"])
    stage = {k: prof[k] / its for k in ["ms_analysis", "ms_reduce", "ms_synthesis", "ms_ring", "ms_control"]}
    workload_name = f"nside{nside}_lmax{lmax}_B{B}"
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s (of fallback)"
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    bf16_src = ("MEASURED_PEAKS.json bf16_tflops_sustained (of measured; timed inside a long step)"
                if "bf16_tflops_sustained" in peaks else "fallback 1700 TFLOP/s sustained (of fallback)")
    mixed = prec != dmwf.DM_FP64
    use_tc = mixed and B in (8, 16, 32, 64)
    # the tensor-core operand: generated tiles when asked, or by the library's size rule (stored tiles and
    # their FP32 tables within 40 GiB; nside 1024 and above generate them)
    gen_tiles = args.tc_tiles == "generated" or (args.tc_tiles == "auto" and nside >= 1024)
    # ring stage (k_ring<RING_ITER>, one launch per FFT-size class).
    # Algorithmic bytes (the map bytes of the hot-path scope): per pixel and
    # RHS-field w d (the anchor map in the mixed mode), s_prev and s, in the
    # map precision, with w shared by the batch.  What the kernel must also
    # move, the ring coefficients (read + write per ring, m and RHS-field)
    # and w per RHS, is implementation traffic, reported beside it.
    px_alg = 12.0 if mixed else 24.0
    ring_bytes = 3.0 * B * px_alg * npix
    px_b, rc_b = (16.0, 16.0) if mixed else (32.0, 32.0)
    ring_impl_bytes = 3.0 * B * (px_b * npix + rc_b * nrings * (mmax + 1))
    # Legendre contractions: 20 flops per (l, m, ring pair) triple per RHS
    # (T: lambda x 2 re/im; Q, U: lam+ and lam- x 4) -- executed on the tensor
    # cores as three BF16 products (hi*hi + hi*lo + lo*hi) in the mixed mode
    leg_flops = 20.0 * triples * B
    # filtered step: per alm and RHS-field the analysis partial sums, then
    # mixed: FP32 state e read + write and its FP32 anchor term c read;
    # FP64: a read + write
    nparts = 1 if use_tc else (npairs + 63) // 64
    red_bytes = 3.0 * B * nalm * ((8.0 * nparts + 24.0) if mixed else (16.0 * nparts + 32.0))

    def hbm_line(kernel, nbytes, ms, traffic_key, impl_bytes=None):
        ach = nbytes / (ms * 1e-3) / 1e9
        tr = traffic_for(traffic_key, workload_name)
        out = {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
               "peak_source": hbm_src, "algorithmic_bytes": nbytes, "ms_per_launch": ms, "traffic": tr,
               "traffic_over_algorithmic": (tr / nbytes) if tr else None}
        if impl_bytes is not None:
            out["implementation_bytes"] = impl_bytes
            out["implementation_frac"] = impl_bytes / (ms * 1e-3) / 1e9 / hbm
        return out

    def leg_line(kernel, ms, traffic_key):
        if use_tc:
            ach = leg_flops / (ms * 1e-3) / 1e12
            return {"bound": "tensor", "kernel": kernel, "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                    "frac": ach / bf16, "peak_source": bf16_src, "algorithmic_flops": leg_flops,
                    "executed_tensor_flops_factor": 3, "ms_per_launch": ms,
                    "traffic": traffic_for(traffic_key, workload_name)}
        peak = fp32_peak if mixed else fp64_peak
        flops = leg_flops if mixed else FLOPS_PER_TRIPLE * triples * B
        ach = flops / (ms * 1e-3) / 1e12
        return {"bound": "alu", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "peak_source": "FMA-chain probe measured live on this GPU (dm_measure_alu_peaks)",
                "algorithmic_flops": flops, "ms_per_launch": ms, "traffic": traffic_for(traffic_key, workload_name)}

    stages = {
        "ring": hbm_line("k_ring<RING_ITER> (one launch per FFT-size class)", ring_bytes, stage["ms_ring"],
                         "k_ring_iter", ring_impl_bytes),
        "synthesis": leg_line(("k_syn_b + k_syn_gen<0,1>" if gen_tiles else "k_syn_b + k_syn_tc<0,1>") if use_tc else ("k_leg_syn32" if mixed else "k_leg_syn64"),
                              stage["ms_synthesis"], "k_syn_tc" if use_tc else "k_leg_syn64"),
        "analysis": leg_line(("k_ana_gen<0,1>" if gen_tiles else "k_ana_tc<0,1>") if use_tc else ("k_leg_ana32" if mixed else "k_leg_ana64"),
                             stage["ms_analysis"], "k_ana_tc" if use_tc else "k_leg_ana64"),
        "reduce": hbm_line("k_ana_step_e32" if mixed else "k_ana_reduce", red_bytes, stage["ms_reduce"], "k_reduce"),
    }
    dom = max(stages, key=lambda k: stages[k]["ms_per_launch"])
    roofline = dict(stages[dom])
    roofline.update({"stage": dom, "stage_ms_per_iter": stage, "stages": stages,
                     "fp64_peak_tflops": fp64_peak, "fp32_peak_tflops": fp32_peak})

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    if not args.no_e2e:
        plan.set_schedule(lambda0=1000.0, n_levels=10, iters_per_level=1, check_every=max(1, K))
        plan.set_forced_iters(iters_split(K))
        d_host = d.cpu().pin_memory()
        s_host = torch.empty_like(d_host).pin_memory()
        plan.set_diagnostics(False)  # a throughput call: no end-of-solve residual and chi^2
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        plan.wiener_filter_host(d_host, s_host)
        h1.record(stream)
        torch.cuda.synchronize()
        plan.set_diagnostics(True)
        wall = time.perf_counter() - t0
        ems = max(h0.elapsed_time(h1), wall * 1e3)
        nbytes = d_host.numel() * 8
        e2e = {"value": B * K / (ems * 1e-3), "unit": "DM iterations/s",
               "h2d_bytes_per_step": nbytes / K, "d2h_bytes_per_step": nbytes / K,
               "note": f"one dm_wiener_filter_host call of {K} iterations (a whole solve: begin, {K} "
                       f"iterations, end); d in and s out once per call; end-of-solve diagnostics off"}

    # ---- whole solves of the same batch (the metric's WF solves/s) ----
    solves = None
    if not args.no_solve and prec == dmwf.DM_MIXED_FP32:
        tol = args.solve_leg_tol
        plan.set_forced_iters(None)
        plan.set_schedule(lambda0=1000.0, n_levels=10, iters_per_level=0, eps0=1e-4, eps_final=tol, eta=0.0,
                          max_iter=100000, check_every=64)
        plan.set_progressive(0.25, 8)
        s_sol = torch.zeros_like(d)
        torch.cuda.synchronize()
        with ClockSampler(0) as sclk:
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            _, sstats = plan.wiener_filter(d, s_sol)
            g1.record(stream)
            torch.cuda.synchronize()
        sms = g0.elapsed_time(g1)
        slev = plan.progressive_levels(10)
        plan.set_progressive(0.0, 8)
        its = np.array([x["iters_total"] for x in sstats])
        solves = {"value": B / (sms * 1e-3), "unit": "WF solves/s", "seconds": sms * 1e-3,
                  "rhs": B, "tol": tol, "converged_rhs": int(sum(1 for x in sstats if x["iters_total"] < 100000)),
                  "iterations_per_rhs": {"mean": float(its.mean()), "min": int(its.min()), "max": int(its.max())},
                  "true_resid": {"mean": float(np.mean([x["true_resid"] for x in sstats])),
                                 "max": float(np.max([x["true_resid"] for x in sstats]))},
                  "schedule": f"lambda 1000 -> 1 in 10 levels, Cauchy 1e-4 -> {tol:g}, progressive working "
                              f"resolution (margin 0.25): {slev}",
                  "fp64_gpu_derived": None, "clocks": sclk.summary(),
                  "note": "one dm_wiener_filter call on the bench's batch (every RHS is a Wiener-filter solve; "
                          "the constrained realisations' fluctuation RHS included)"}
        if fp64_line is not None and (nside, lmax, B, tol) == (512, 1024, 64, 1e-5):
            # plain FP64: its measured iterations/s over the full-resolution iteration count of the same
            # schedule (FP64 solves take the oracle's counts; measured at nside 512 / 1e-5: 7378 per RHS)
            solves["fp64_gpu_derived"] = {"value": fp64_line["value"] / 7378.0, "unit": "WF solves/s",
                                          "iterations_per_rhs": 7378,
                                          "note": "derived: plain FP64 DM iterations/s / 7378, the mean count of "
                                                  "the full-resolution mixed solve of this batch to 1e-5"}

    # ---- CPU baseline (oracle), rank 0 at N = 1 only ----
    cpu, err = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        d0 = oracle_data(O, nside, lmax, wl)
        cpu, ref0 = cpu_baseline(nside, lmax, wl, d0)
        err = error_vs_oracle(plan, d, d0, ref0, prec, torch)

    if rank == 0:
        line = {"metric": "DM iterations/s", "value": value, "unit": "DM iterations/s", "n_gpus": ws,
                "steps": K, "warmup": Wu, "ms_per_step": B * ws / value * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == dmwf.DM_FP64 else "f32 (bf16x3 tensor-core Legendre, f64 harmonic state)",
                "data": "synthetic",
                "config": {"workload": f"batched constrained realisations nside {nside} lmax {lmax}: "
                                       f"{nwf} WF + {B - nwf} fluctuation RHS per launch (seeds 100..{99 + B})",
                           "nside": nside, "lmax": lmax, "batch": B, "precision": args.precision,
                           "ring_radix": ("autotuned" if tuning else "plan default") if args.ring_radix is None
                           else args.ring_radix,
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                           "tc_tiles": args.tc_tiles,
                           "l2": "inputs larger than L2 (maps and ring coefficients exceed 129 MB)"},
                "ms_per_step_median": float(np.median(chunk_ms)),
                "timing": {"chunks": nch, "chunk_ms_per_step": chunk_ms,
                           "median_ms_per_step": float(np.median(chunk_ms))},
                "error_vs_oracle": err,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": prof["launches"],
                "fp64_gpu": fp64_line, "ff64_gpu": ff_line, "solves": solves, "refinement": anchor,
                "autotune": tuning,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
