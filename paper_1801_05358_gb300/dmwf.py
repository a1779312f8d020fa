"""Thin Python binding of libdmwf (include/dmwf.h): argument marshalling only.

Every step of the dual messenger path runs in the CUDA library; this module
passes torch device pointers and CUDA streams through ctypes and converts the
host-side arrays (spectra, noise, mask, schedule).  Importing it fails loudly
when the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdmwf.so")

DM_OK, DM_EINVAL, DM_ENOMEM, DM_ECUDA, DM_ENOTCONV, DM_ETIMEOUT, DM_EAGAIN, DM_EBUSY = range(8)
DM_FP64, DM_MIXED_FP32, DM_FLOAT_FLOAT = 0, 1, 2
DM_MAX_LEVELS = 64

EXPORTS = [
    "dm_plan_create", "dm_plan_destroy", "dm_last_error", "dm_plan_info", "dm_set_precision", "dm_set_spectra",
    "dm_set_noise_mask", "dm_set_schedule", "dm_set_forced_iters", "dm_wiener_filter", "dm_wiener_filter_host",
    "dm_constrained_realization", "dm_draw_cr_inputs", "dm_alm2map", "dm_map2alm", "dm_ring_fft_forward",
    "dm_ring_fft_inverse", "dm_legendre_synthesis", "dm_legendre_analysis", "dm_apply_filter", "dm_noise_info",
    "dm_profile_enable", "dm_profile_read", "dm_measure_alu_peaks", "dm_solve_begin", "dm_solve_iterate",
    "dm_solve_end", "dm_set_refinement", "dm_set_noise_mask_rhs", "dm_server_create", "dm_serve_submit",
    "dm_serve_poll", "dm_serve_cancel", "dm_server_info", "dm_server_destroy", "dm_set_tensor_cores", "dm_set_tc_tiles", "dm_set_ff_slab_bytes", "dm_set_analysis_slots", "dm_set_ring_radix",
    "dm_set_anchor_precision", "dm_set_noise_cov",
    "dm_legendre_analysis_noalloc", "dm_set_diagnostics", "dm_autotune", "dm_get_tuning", "dm_set_tuning",
    "dm_jacobi_refine", "dm_test_tc_withhold", "dm_plan_create_flat", "dm_set_spectra_flat", "dm_set_noise_flat",
    "dm_set_progressive", "dm_get_progressive_levels",
]
DM_REQ_WF, DM_REQ_CR = 0, 1


class DmSchedule(ctypes.Structure):
    _fields_ = [("lambda0", ctypes.c_double), ("n_levels", ctypes.c_int), ("iters_per_level", ctypes.c_int),
                ("eps0", ctypes.c_double), ("eps_final", ctypes.c_double), ("eta", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int)]


class DmStats(ctypes.Structure):
    _fields_ = [("iters_total", ctypes.c_int), ("levels_done", ctypes.c_int),
                ("iters_per_level", ctypes.c_int * DM_MAX_LEVELS), ("cauchy_final", ctypes.c_double),
                ("true_resid", ctypes.c_double), ("chi2", ctypes.c_double), ("ms_total", ctypes.c_float)]


class DmProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("iterations", ctypes.c_int64), ("ms_analysis", ctypes.c_double),
                ("ms_reduce", ctypes.c_double), ("ms_synthesis", ctypes.c_double), ("ms_ring", ctypes.c_double),
                ("ms_control", ctypes.c_double), ("anchors", ctypes.c_int64), ("ms_anchor", ctypes.c_double)]


DM_TUNE_MAX_CLASSES = 12


class DmTuning(ctypes.Structure):
    _fields_ = [("n_ring_classes", ctypes.c_int), ("ring_radix_lr", ctypes.c_int * DM_TUNE_MAX_CLASSES),
                ("ring_lanes", ctypes.c_int * DM_TUNE_MAX_CLASSES),
                ("ring_fused", ctypes.c_int * DM_TUNE_MAX_CLASSES), ("syn_stages", ctypes.c_int * 2),
                ("ana_ltiles", ctypes.c_int * 2), ("ana_stages", ctypes.c_int * 2),
                ("ms_ring", ctypes.c_float), ("ms_ring_default", ctypes.c_float),
                ("ms_synthesis", ctypes.c_float), ("ms_synthesis_default", ctypes.c_float),
                ("ms_analysis", ctypes.c_float), ("ms_analysis_default", ctypes.c_float),
                ("from_cache", ctypes.c_int)]


class DmServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("slots_per_plan", ctypes.c_int),
                ("iters_per_round", ctypes.c_int), ("prec", ctypes.c_int), ("sched", DmSchedule),
                ("anchor_every", ctypes.c_int), ("max_pending", ctypes.c_int), ("strict_tol", ctypes.c_double),
                ("strict_prec", ctypes.c_int)]


class DmRequest(ctypes.Structure):
    _fields_ = [("nside", ctypes.c_int), ("lmax", ctypes.c_int), ("kind", ctypes.c_int), ("tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("cl", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("d", ctypes.c_void_p), ("s_out", ctypes.c_void_p)]


class DmResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("cauchy_final", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class DmServerInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ["pending", "busy_slots", "pools", "bytes_reserved", "rounds",
                                               "admitted", "retired"]]


class DmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dmwf status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libdmwf.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built: run `python -m paper_1801_05358_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.dm_plan_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
        L.dm_plan_destroy.argtypes = [vp]
        L.dm_plan_destroy.restype = None
        L.dm_last_error.argtypes = [vp]
        L.dm_last_error.restype = ctypes.c_char_p
        L.dm_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]
        L.dm_set_precision.argtypes = [vp, ctypes.c_int]
        L.dm_set_spectra.argtypes = [vp, vp]
        L.dm_set_noise_mask.argtypes = [vp, vp, vp]
        L.dm_set_noise_cov.argtypes = [vp, vp, vp, vp, vp]
        L.dm_set_schedule.argtypes = [vp, ctypes.POINTER(DmSchedule)]
        L.dm_set_forced_iters.argtypes = [vp, vp]
        L.dm_wiener_filter.argtypes = [vp, vp, vp, vp, vp, vp]
        L.dm_wiener_filter_host.argtypes = [vp, vp, vp, vp, vp, vp]
        L.dm_constrained_realization.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.dm_draw_cr_inputs.argtypes = [vp, vp, vp, vp, vp, vp]
        for name in ["dm_alm2map", "dm_map2alm", "dm_ring_fft_forward", "dm_ring_fft_inverse",
                     "dm_legendre_synthesis", "dm_legendre_analysis", "dm_legendre_analysis_noalloc"]:
            getattr(L, name).argtypes = [vp, vp, vp, vp]
        L.dm_apply_filter.argtypes = [vp, ctypes.c_double, vp, vp, vp]
        L.dm_noise_info.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.dm_profile_enable.argtypes = [vp, ctypes.c_int]
        L.dm_profile_read.argtypes = [vp, ctypes.POINTER(DmProfile)]
        L.dm_solve_begin.argtypes = [vp, vp, vp]
        L.dm_solve_iterate.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp]
        L.dm_solve_end.argtypes = [vp, vp, vp, vp, vp]
        L.dm_set_refinement.argtypes = [vp, ctypes.c_int]
        L.dm_set_anchor_precision.argtypes = [vp, ctypes.c_int]
        L.dm_set_tensor_cores.argtypes = [vp, ctypes.c_int]
        L.dm_set_tc_tiles.argtypes = [vp, ctypes.c_int]
        L.dm_set_ff_slab_bytes.argtypes = [vp, ctypes.c_int64]
        L.dm_set_analysis_slots.argtypes = [vp, ctypes.c_int]
        L.dm_set_diagnostics.argtypes = [vp, ctypes.c_int]
        L.dm_autotune.argtypes = [vp, ctypes.c_int, vp]
        L.dm_jacobi_refine.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp, vp]
        L.dm_test_tc_withhold.argtypes = [vp, ctypes.c_int]
        L.dm_set_progressive.argtypes = [vp, ctypes.c_double, ctypes.c_int]
        L.dm_get_progressive_levels.argtypes = [vp, vp, vp]
        L.dm_plan_create_flat.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(vp)]
        L.dm_set_spectra_flat.argtypes = [vp, vp]
        L.dm_set_noise_flat.argtypes = [vp, vp, vp, vp]
        L.dm_get_tuning.argtypes = [vp, ctypes.POINTER(DmTuning)]
        L.dm_set_tuning.argtypes = [vp, ctypes.POINTER(DmTuning)]
        L.dm_set_noise_mask_rhs.argtypes = [vp, ctypes.c_int, vp, vp]
        L.dm_server_create.argtypes = [ctypes.POINTER(DmServerConfig), ctypes.POINTER(vp)]
        L.dm_serve_submit.argtypes = [vp, ctypes.POINTER(DmRequest), ctypes.POINTER(ctypes.c_uint64)]
        L.dm_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(DmResult)]
        L.dm_serve_cancel.argtypes = [vp, ctypes.c_uint64]
        L.dm_server_info.argtypes = [vp, ctypes.POINTER(DmServerInfo)]
        L.dm_server_destroy.argtypes = [vp]
        L.dm_server_destroy.restype = None
        L.dm_measure_alu_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        _lib = L
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _np_ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def measure_alu_peaks():
    """(fp64, fp32) TFLOP/s of the current device from FMA chains."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = lib().dm_measure_alu_peaks(ctypes.byref(a), ctypes.byref(b))
    if st != DM_OK:
        raise DmError(st, "peak probe failed")
    return a.value, b.value


class Plan:
    """One dm_plan: geometry (nside, lmax), batch of right-hand sides."""

    def __init__(self, nside: int, lmax: int, batch: int = 1):
        h = ctypes.c_void_p()
        st = lib().dm_plan_create(nside, lmax, batch, ctypes.byref(h))
        if st != DM_OK:
            raise DmError(st, "dm_plan_create failed (nside, lmax, batch out of range or no memory)")
        self.h = h
        self.nside, self.lmax, self.batch = nside, lmax, batch
        self.npix = 12 * nside * nside
        self.nalm = (lmax + 1) * (lmax + 2) // 2
        self.nrings = 4 * nside - 1
        self._keep = []

    def close(self):
        if self.h:
            lib().dm_plan_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != DM_OK and st not in allow:
            raise DmError(st, lib().dm_last_error(self.h).decode())
        return st

    # ---- set-up ----
    def set_precision(self, prec):
        self._check(lib().dm_set_precision(self.h, prec))

    def set_spectra(self, cl):
        c = np.ascontiguousarray(cl, dtype=np.float64)
        self._check(lib().dm_set_spectra(self.h, _np_ptr(c)))

    def set_noise_mask(self, sigma, mask=None):
        s = np.ascontiguousarray(sigma, dtype=np.float64)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        self._check(lib().dm_set_noise_mask(self.h, _np_ptr(s), _np_ptr(m)))

    def set_noise_mask_rhs(self, b, sigma, mask=None):
        s = np.ascontiguousarray(sigma, dtype=np.float64)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        self._check(lib().dm_set_noise_mask_rhs(self.h, int(b), _np_ptr(s), _np_ptr(m)))

    def set_schedule(self, lambda0=1000.0, n_levels=10, iters_per_level=10, eps0=1e-4, eps_final=1e-6, eta=0.0,
                     max_iter=100000, check_every=8):
        sc = DmSchedule(lambda0, n_levels, iters_per_level, eps0, eps_final, eta, max_iter, check_every)
        self._check(lib().dm_set_schedule(self.h, ctypes.byref(sc)))

    def set_forced_iters(self, iters):
        if iters is None:
            self._check(lib().dm_set_forced_iters(self.h, None))
            return
        a = np.ascontiguousarray(iters, dtype=np.int32)
        self._check(lib().dm_set_forced_iters(self.h, _np_ptr(a)))

    def noise_info(self):
        a, t = ctypes.c_double(), ctypes.c_double()
        self._check(lib().dm_noise_info(self.h, ctypes.byref(a), ctypes.byref(t)))
        return a.value, t.value

    def profile_enable(self, on=True):
        self._check(lib().dm_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        pr = DmProfile()
        self._check(lib().dm_profile_read(self.h, ctypes.byref(pr)))
        return {k: getattr(pr, k) for k, _ in DmProfile._fields_}

    def info(self):
        a, b, c, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        self._check(lib().dm_plan_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        return dict(npix=a.value, nalm=b.value, nrings=c.value, workspace_bytes=d.value)

    # ---- hot path (torch CUDA tensors, float64 / complex128) ----
    @staticmethod
    def _stats_out(stats_arr):
        return [dict(iters_total=s.iters_total, levels_done=s.levels_done,
                     iters_per_level=list(s.iters_per_level), cauchy_final=s.cauchy_final,
                     true_resid=s.true_resid, chi2=s.chi2, ms_total=s.ms_total) for s in stats_arr]

    def wiener_filter(self, d, s_out, alm_out=None, stream=None):
        stats = (DmStats * self.batch)()
        st = lib().dm_wiener_filter(self.h, _ptr(d), _ptr(s_out), _ptr(alm_out), stats, _stream(stream))
        self._check(st, allow=(DM_ENOTCONV,))
        return st, self._stats_out(stats)

    def solve_begin(self, d, stream=None):
        self._check(lib().dm_solve_begin(self.h, _ptr(d), _stream(stream)))

    def solve_iterate(self, max_iters, stream=None):
        done = ctypes.c_int(0)
        self._check(lib().dm_solve_iterate(self.h, int(max_iters), ctypes.byref(done), _stream(stream)))
        return bool(done.value)

    def solve_end(self, s_out=None, alm_out=None, stream=None):
        stats = (DmStats * self.batch)()
        st = lib().dm_solve_end(self.h, _ptr(s_out), _ptr(alm_out), stats, _stream(stream))
        self._check(st, allow=(DM_ENOTCONV,))
        return st, self._stats_out(stats)

    def test_tc_withhold(self, on=True):
        """Failure-test hook: one withheld mbarrier arrival in the tensor-core analysis."""
        self._check(lib().dm_test_tc_withhold(self.h, 1 if on else 0))

    def set_progressive(self, margin=0.25, lmin=8):
        """Progressive working resolution per cooling level (0 turns it off)."""
        self._check(lib().dm_set_progressive(self.h, ctypes.c_double(margin), int(lmin)))

    def progressive_levels(self, n_levels):
        nk = np.zeros(n_levels, dtype=np.int32)
        lk = np.zeros(n_levels, dtype=np.int32)
        self._check(lib().dm_get_progressive_levels(self.h, _np_ptr(nk), _np_ptr(lk)))
        return list(zip(nk.tolist(), lk.tolist()))

    def set_diagnostics(self, on=True):
        """End-of-solve true residual and chi^2 in the stats (default on)."""
        self._check(lib().dm_set_diagnostics(self.h, 1 if on else 0))

    def autotune(self, force=False, stream=None):
        """Time the launch candidates on this plan (dm_autotune); returns the picks."""
        self._check(lib().dm_autotune(self.h, 1 if force else 0, _stream(stream)))
        return self.tuning()

    def tuning(self):
        t = DmTuning()
        self._check(lib().dm_get_tuning(self.h, ctypes.byref(t)))
        n = t.n_ring_classes
        out = {k: getattr(t, k) for k, _ in DmTuning._fields_ if not k.startswith(("ring_", "syn_", "ana_"))}
        out.update(ring_radix_lr=list(t.ring_radix_lr)[:n], ring_lanes=list(t.ring_lanes)[:n],
                   ring_fused=list(t.ring_fused)[:n],
                   syn_stages=list(t.syn_stages), ana_ltiles=list(t.ana_ltiles), ana_stages=list(t.ana_stages))
        return out

    def set_tuning(self, d):
        t = DmTuning()
        t.n_ring_classes = len(d.get("ring_lanes", []))
        for i, v in enumerate(d.get("ring_radix_lr", [])):
            t.ring_radix_lr[i] = v
        for i, v in enumerate(d.get("ring_lanes", [])):
            t.ring_lanes[i] = v
        for i in range(DM_TUNE_MAX_CLASSES):
            t.ring_fused[i] = -1
        for i, v in enumerate(d.get("ring_fused", [])):
            t.ring_fused[i] = v
        for k in ("syn_stages", "ana_ltiles", "ana_stages"):
            for i, v in enumerate(d.get(k, [0, 0])):
                getattr(t, k)[i] = v
        self._check(lib().dm_set_tuning(self.h, ctypes.byref(t)))

    def set_tensor_cores(self, on=True):
        self._check(lib().dm_set_tensor_cores(self.h, 1 if on else 0))

    def set_tc_tiles(self, generate=True):
        """Tensor-core Legendre operand generated in the kernels (True), streamed from stored
        tables (False) or chosen by size (None)."""
        self._check(lib().dm_set_tc_tiles(self.h, -1 if generate is None else (1 if generate else 0)))

    def set_analysis_slots(self, slots):
        """Chunk slots of the FP64-class analysis partial sums per RHS (fewer than chunks: waves)."""
        self._check(lib().dm_set_analysis_slots(self.h, int(slots)))

    def set_ff_slab_bytes(self, nbytes):
        """Largest per-slab table of the float-float stages when the plan keeps no full FP32 tables."""
        self._check(lib().dm_set_ff_slab_bytes(self.h, int(nbytes)))

    def set_ring_radix(self, lr):
        """Fixed-size ring transforms of radix 2^lr (3 or 4), or 0 for the generic kernels."""
        self._check(lib().dm_set_ring_radix(self.h, int(lr)))

    def set_noise_cov(self, sigma, rho, mask_t=None, mask_p=None):
        """Correlated 3x3 noise per pixel with distinct T / P masks (dm_set_noise_cov)."""
        sg = np.ascontiguousarray(sigma, dtype=np.float64)
        rh = np.ascontiguousarray(rho, dtype=np.float64)
        mt = None if mask_t is None else np.ascontiguousarray(mask_t, dtype=np.uint8)
        mp = None if mask_p is None else np.ascontiguousarray(mask_p, dtype=np.uint8)
        self._check(lib().dm_set_noise_cov(self.h, sg.ctypes.data, rh.ctypes.data,
                                           None if mt is None else mt.ctypes.data,
                                           None if mp is None else mp.ctypes.data))

    def set_refinement(self, anchor_every):
        self._check(lib().dm_set_refinement(self.h, int(anchor_every)))

    def set_anchor_precision(self, prec):
        self._check(lib().dm_set_anchor_precision(self.h, int(prec)))

    def jacobi_refine(self, d, n_refine, s_out, alm_out=None, stream=None):
        """Wiener filter plus n_refine modified Jacobi steps (Appendix A)."""
        stats = (DmStats * self.batch)()
        st = lib().dm_jacobi_refine(self.h, _ptr(d), int(n_refine), _ptr(s_out), _ptr(alm_out), stats,
                                    _stream(stream))
        self._check(st, allow=(DM_ENOTCONV,))
        return st, self._stats_out(stats)

    def wiener_filter_host(self, d_host, s_host, alm_host=None, stream=None):
        stats = (DmStats * self.batch)()
        st = lib().dm_wiener_filter_host(self.h, _ptr(d_host), _ptr(s_host), _ptr(alm_host), stats,
                                         _stream(stream))
        self._check(st, allow=(DM_ENOTCONV,))
        return st, self._stats_out(stats)

    def constrained_realization(self, d, seeds, s_out, alm_out=None, stream=None):
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        stats = (DmStats * self.batch)()
        st = lib().dm_constrained_realization(self.h, _ptr(d), _np_ptr(sd), _ptr(s_out), _ptr(alm_out), stats,
                                              _stream(stream))
        self._check(st, allow=(DM_ENOTCONV,))
        return st, self._stats_out(stats)

    def draw_cr_inputs(self, seeds, ahat=None, shat=None, dhat=None, stream=None):
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        self._check(lib().dm_draw_cr_inputs(self.h, _np_ptr(sd), _ptr(ahat), _ptr(shat), _ptr(dhat),
                                            _stream(stream)))

    def alm2map(self, alm, out, stream=None):
        self._check(lib().dm_alm2map(self.h, _ptr(alm), _ptr(out), _stream(stream)))

    def map2alm(self, maps, out, stream=None):
        self._check(lib().dm_map2alm(self.h, _ptr(maps), _ptr(out), _stream(stream)))

    def ring_fft_forward(self, maps, rc, stream=None):
        self._check(lib().dm_ring_fft_forward(self.h, _ptr(maps), _ptr(rc), _stream(stream)))

    def ring_fft_inverse(self, rc, maps, stream=None):
        self._check(lib().dm_ring_fft_inverse(self.h, _ptr(rc), _ptr(maps), _stream(stream)))

    def legendre_synthesis(self, alm, rc, stream=None):
        self._check(lib().dm_legendre_synthesis(self.h, _ptr(alm), _ptr(rc), _stream(stream)))

    def legendre_analysis(self, rc, alm, stream=None):
        self._check(lib().dm_legendre_analysis(self.h, _ptr(rc), _ptr(alm), _stream(stream)))

    def legendre_analysis_noalloc(self, rc, alm, stream=None):
        """dm_legendre_analysis without any device allocation in the call
        (scratch in a fixed file-scope device array)."""
        self._check(lib().dm_legendre_analysis_noalloc(self.h, _ptr(rc), _ptr(alm), _stream(stream)))

    def apply_filter(self, lam, alm_in, alm_out, stream=None):
        self._check(lib().dm_apply_filter(self.h, ctypes.c_double(lam), _ptr(alm_in), _ptr(alm_out),
                                          _stream(stream)))


class Server:
    """Continuous-batching server (dm_server_*).  Requests carry host arrays;
    the result map is written into a host array owned by this object until the
    ticket completes.  Requests with tol < strict_tol are served by pools of
    strict_prec (DM_FP64 or DM_FLOAT_FLOAT), the others by pools of prec."""

    def __init__(self, hbm_budget_bytes, slots_per_plan=8, iters_per_round=16, prec=DM_FP64, lambda0=1000.0,
                 n_levels=10, eps0=1e-4, max_iter=1000000, anchor_every=0, max_pending=0, strict_tol=0.0,
                 strict_prec=DM_FP64):
        sc = DmSchedule(lambda0, n_levels, 0, eps0, 1e-6, 0.0, max_iter, 8)
        cfg = DmServerConfig(int(hbm_budget_bytes), slots_per_plan, iters_per_round, prec, sc, anchor_every,
                             max_pending, float(strict_tol), strict_prec)
        h = ctypes.c_void_p()
        st = lib().dm_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != DM_OK:
            raise DmError(st, "dm_server_create failed")
        self.h = h
        self._live = {}

    def submit(self, nside, lmax, kind, tol, cl, sigma, d, mask=None, seed=0):
        arrs = dict(cl=np.ascontiguousarray(cl, dtype=np.float64), sigma=np.ascontiguousarray(sigma, dtype=np.float64),
                    d=np.ascontiguousarray(d, dtype=np.float64),
                    mask=None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8))
        out = np.zeros((3, 12 * nside * nside), dtype=np.float64)
        req = DmRequest(nside, lmax, kind, tol, seed, arrs["cl"].ctypes.data, arrs["sigma"].ctypes.data,
                        None if arrs["mask"] is None else arrs["mask"].ctypes.data, arrs["d"].ctypes.data,
                        out.ctypes.data)
        t = ctypes.c_uint64()
        st = lib().dm_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st != DM_OK:
            raise DmError(st, "dm_serve_submit")
        self._live[t.value] = out
        return t.value

    def poll(self, ticket):
        """None while pending, else (result dict, map)."""
        r = DmResult()
        st = lib().dm_serve_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r))
        if st == DM_EAGAIN:
            return None
        if st != DM_OK:
            raise DmError(st, "dm_serve_poll")
        out = self._live.pop(ticket)
        return dict(status=r.status, iters=r.iters, cauchy_final=r.cauchy_final, latency_ms=r.latency_ms,
                    queue_ms=r.queue_ms), out

    def cancel(self, ticket):
        return lib().dm_serve_cancel(self.h, ctypes.c_uint64(ticket))

    def info(self):
        i = DmServerInfo()
        lib().dm_server_info(self.h, ctypes.byref(i))
        return {k: getattr(i, k) for k, _ in DmServerInfo._fields_}

    def close(self):
        if self.h:
            lib().dm_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FlatPlan(Plan):
    """A flat-sky plan (dm_plan_create_flat): an N x N grid of side L radians.
    Maps [batch, 3, N * N] row-major; harmonic modes [batch, 3, N/2, N]
    complex (kx major, ky in FFT order)."""

    def __init__(self, N: int, L: float, batch: int = 1):
        h = ctypes.c_void_p()
        st = lib().dm_plan_create_flat(int(N), ctypes.c_double(L), int(batch), ctypes.byref(h))
        if st != DM_OK:
            raise DmError(st, "dm_plan_create_flat failed (N a power of two in [16, 2048], L > 0, batch)")
        self.h = h
        self.N, self.L, self.batch = N, L, batch
        self.nside, self.lmax = None, N // 2 - 1
        self.npix = N * N
        self.nalm = (N // 2) * N
        self.nrings = N
        self._keep = []

    def set_spectra(self, S):
        """Spectra per mode [4, N, N] (TT, EE, BB, TE) in numpy FFT order."""
        c = np.ascontiguousarray(S, dtype=np.float64)
        self._check(lib().dm_set_spectra_flat(self.h, _np_ptr(c)))

    def set_noise(self, sigma, mask_t=None, mask_p=None):
        s = np.ascontiguousarray(sigma, dtype=np.float64)
        mt = None if mask_t is None else np.ascontiguousarray(mask_t, dtype=np.uint8)
        mp = None if mask_p is None else np.ascontiguousarray(mask_p, dtype=np.uint8)
        self._check(lib().dm_set_noise_flat(self.h, _np_ptr(s), _np_ptr(mt), _np_ptr(mp)))
