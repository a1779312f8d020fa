"""ctypes wrapper around the FP64 CPU oracle (dm_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The CUDA product path never imports this module.

Every function follows the dual messenger method of Kodi Ramanah, Lavaux &
Wandelt (arXiv:1801.05358) on the HEALPix sphere; the C file cites the
section, equation or algorithm each routine implements.  Array layouts:

* maps ``[3, npix]`` (I, Q, U), RING order, float64;
* alm ``[3, nalm]`` complex128 (T, E, B), m-major index ``m(2lmax+1-m)/2 + l``;
* ring coefficients ``[3, nrings, lmax+1]`` complex128;
* spectra ``cl[4, lmax+1]`` = TT, EE, BB, TE.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_ip = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile dm_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FMA
    contraction so that x86 and Arm hosts round identically)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_npix.restype = ctypes.c_long
        L.orc_nalm.restype = ctypes.c_long
        L.orc_almidx.restype = ctypes.c_long
        L.orc_alpha.restype = ctypes.c_double
        L.orc_chi2.restype = ctypes.c_double
        L.orc_dm_solve.restype = ctypes.c_int
        L.orc_cov_alpha.restype = ctypes.c_double
        L.orc_dm_solve_cov.restype = ctypes.c_int
        L.orc_wf_residual.restype = ctypes.c_double
        L.orc_wf_residual_cov.restype = ctypes.c_double
        L.orc_chi2_cov.restype = ctypes.c_double
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def npix(nside):
    return 12 * nside * nside


def nrings(nside):
    return 4 * nside - 1


def nalm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def almidx(lmax, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def ring_info(nside, i):
    """(n_pix_in_ring, first_pixel, z, 1-z, 1+z, phi0) of ring i (1-based)."""
    nr, st = ctypes.c_long(), ctypes.c_long()
    z, omz, opz, p0 = (ctypes.c_double() for _ in range(4))
    lib().orc_ring_info(nside, i, ctypes.byref(nr), ctypes.byref(st), ctypes.byref(z),
                        ctypes.byref(omz), ctypes.byref(opz), ctypes.byref(p0))
    return nr.value, st.value, z.value, omz.value, opz.value, p0.value


def pix_centers(nside):
    z = np.zeros(npix(nside))
    phi = np.zeros(npix(nside))
    lib().orc_pix_centers(nside, _d(z), _d(phi))
    return z, phi


def lam_theta(lmax, m, theta):
    """lambda_lm, 2lambda_lm, -2lambda_lm (l = 0..lmax) at colatitude theta."""
    out = [np.zeros(lmax + 1) for _ in range(3)]
    lib().orc_lambda_theta(lmax, m, ctypes.c_double(theta), *map(_d, out))
    return out


def lam_ring(lmax, m, omz, opz):
    out = [np.zeros(lmax + 1) for _ in range(3)]
    lib().orc_lambda(lmax, m, ctypes.c_double(omz), ctypes.c_double(opz), *map(_d, out))
    return out


def ring_alm2map(nside, lmax, alm, i):
    """The three maps of Y a on ring i (1-based), shape (3, n_r): a sampled alm2map."""
    a = _c2r(alm)
    nr = ring_info(nside, i)[0]
    out = np.zeros((3, nr))
    lib().orc_ring_alm2map(nside, lmax, _d(a), i, _d(out))
    return out


def map2alm_m(nside, lmax, maps, m):
    """Column m of A f, shape (3, lmax + 1) complex (l < m zero): a sampled map2alm."""
    f = np.ascontiguousarray(maps, dtype=np.float64)
    out = np.zeros((3, lmax + 1), dtype=np.complex128)
    lib().orc_map2alm_m(nside, lmax, _d(f), m, _d(out.view(np.float64)))
    return out


def _c2r(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def ring_dft_forward(nside, mmax, ringmap):
    """Per-ring G_m = sum_j f_j e^{-i m phi_j}; returns [nrings, mmax+1] complex."""
    f = np.ascontiguousarray(ringmap, dtype=np.float64)
    rc = np.zeros((nrings(nside), mmax + 1), dtype=np.complex128)
    lib().orc_ring_dft_forward(nside, mmax, _d(f), _d(rc.view(np.float64)))
    return rc


def ring_dft_inverse(nside, mmax, rc):
    r = _c2r(rc)
    f = np.zeros(npix(nside))
    lib().orc_ring_dft_inverse(nside, mmax, _d(r), _d(f))
    return f


def legendre_synthesis(nside, lmax, alm):
    a = _c2r(alm)
    rc = np.zeros((3, nrings(nside), lmax + 1), dtype=np.complex128)
    lib().orc_legendre_synthesis(nside, lmax, _d(a), _d(rc.view(np.float64)))
    return rc


def legendre_analysis(nside, lmax, rc):
    r = _c2r(rc)
    alm = np.zeros((3, nalm(lmax)), dtype=np.complex128)
    lib().orc_legendre_analysis(nside, lmax, _d(r), _d(alm.view(np.float64)))
    return alm


def alm2map(nside, lmax, alm):
    """Synthesis Y: alm [3, nalm] (T, E, B) -> maps [3, npix] (I, Q, U)."""
    a = _c2r(alm)
    m = np.zeros((3, npix(nside)))
    lib().orc_alm2map(nside, lmax, _d(a), _d(m))
    return m


def map2alm(nside, lmax, maps):
    """Analysis A = Omega Y^dagger: maps [3, npix] -> alm [3, nalm]."""
    mp = np.ascontiguousarray(maps, dtype=np.float64)
    alm = np.zeros((3, nalm(lmax)), dtype=np.complex128)
    lib().orc_map2alm(nside, lmax, _d(mp), _d(alm.view(np.float64)))
    return alm


def filter_coefs(lmax, cl, mu, th):
    """Per-l (F_TT, F_TE, F_EE, F_BB) of the filter (Sbar+U)(Sbar+xi)^{-1}."""
    c = np.ascontiguousarray(cl, dtype=np.float64)
    coef = np.zeros((lmax + 1, 4))
    lib().orc_filter_coefs(lmax, _d(c), ctypes.c_double(mu), ctypes.c_double(th), _d(coef))
    return coef


def apply_filter(lmax, coef, alm):
    a = np.array(alm, dtype=np.complex128, copy=True)
    lib().orc_apply_filter(lmax, _d(np.ascontiguousarray(coef)), _d(a.view(np.float64)))
    return a


def _mask_ptr(mask):
    if mask is None:
        return None, ctypes.cast(None, _u8p)
    mk = np.ascontiguousarray(mask, dtype=np.uint8)
    return mk, mk.ctypes.data_as(_u8p)


def alpha(sigma, mask):
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    mk, mp = _mask_ptr(mask)
    return lib().orc_alpha(s.shape[1], _d(s), mp)


def weights(sigma, mask, alpha_):
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    mk, mp = _mask_ptr(mask)
    w = np.zeros_like(s)
    lib().orc_weights(s.shape[1], _d(s), mp, ctypes.c_double(alpha_), _d(w))
    return w


def messenger_update(w, d, s):
    w = np.ascontiguousarray(w, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    t = np.zeros_like(s)
    lib().orc_messenger_update(w.size, _d(w), _d(d), _d(s), _d(t))
    return t


def cov_ninv(sigma, rho, maskT, maskP):
    """Per-pixel N^{-1} [npix, 3, 3] of the correlated noise model (Appendix B)."""
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    mt, mtp = _mask_ptr(maskT)
    mp_, mpp = _mask_ptr(maskP)
    npix = sg.shape[1]
    out = np.zeros((npix, 3, 3))
    lib().orc_cov_ninv(npix, _d(sg), _d(rh), mtp, mpp, _d(out))
    return out


def cov_alpha(ninv):
    n = np.ascontiguousarray(ninv, dtype=np.float64)
    return lib().orc_cov_alpha(n.shape[0], _d(n))


def messenger_update_cov(alpha_, ninv, d, s):
    n = np.ascontiguousarray(ninv, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    t = np.zeros_like(s)
    lib().orc_messenger_update_cov(n.shape[0], ctypes.c_double(alpha_), _d(n), _d(d), _d(s), _d(t))
    return t


def dm_solve_cov(nside, lmax, cl, sigma, rho, maskT, maskP, d, lambdas, eps=None, forced_iters=None,
                 max_iter=100000):
    """Algorithm 1 with the correlated noise model and distinct T/P masks.
    Returns dict(s, alm, iters_per_level, cauchy, iters)."""
    lambdas = np.ascontiguousarray(lambdas, dtype=np.float64)
    nlev = lambdas.size
    eps = np.ascontiguousarray(np.zeros(nlev) if eps is None else eps, dtype=np.float64)
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    mt, mtp = _mask_ptr(maskT)
    mp_, mpp = _mask_ptr(maskP)
    s = np.zeros((3, npix(nside)))
    alm = np.zeros((3, nalm(lmax)), dtype=np.complex128)
    iters = np.zeros(nlev, dtype=np.int32)
    if forced_iters is not None:
        fi = np.ascontiguousarray(forced_iters, dtype=np.int32)
        fptr = fi.ctypes.data_as(_ip)
        max_iter = int(fi.sum())
    else:
        fi = None
        fptr = ctypes.cast(None, _ip)
    cauchy = np.zeros(max(max_iter, 1))
    n = lib().orc_dm_solve_cov(nside, lmax, _d(c), _d(sg), _d(rh), mtp, mpp, _d(dd), nlev, _d(lambdas), _d(eps),
                               fptr, max_iter, _d(s), _d(alm.view(np.float64)), iters.ctypes.data_as(_ip),
                               _d(cauchy))
    return dict(s=s, alm=alm, iters_per_level=iters, cauchy=cauchy[:n], iters=n)


def dm_solve(nside, lmax, cl, sigma, mask, d, lambdas, eps=None, forced_iters=None, max_iter=100000):
    """Algorithm 1 on the sphere.  Returns dict(s, alm, iters_per_level, cauchy, iters)."""
    lambdas = np.ascontiguousarray(lambdas, dtype=np.float64)
    nlev = lambdas.size
    if eps is None:
        eps = np.zeros(nlev)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    mk, mp = _mask_ptr(mask)
    s = np.zeros((3, npix(nside)))
    alm = np.zeros((3, nalm(lmax)), dtype=np.complex128)
    iters = np.zeros(nlev, dtype=np.int32)
    if forced_iters is not None:
        fi = np.ascontiguousarray(forced_iters, dtype=np.int32)
        fptr = fi.ctypes.data_as(_ip)
        max_iter = int(fi.sum())
    else:
        fi = None
        fptr = ctypes.cast(None, _ip)
    cauchy = np.zeros(max(max_iter, 1))
    n = lib().orc_dm_solve(nside, lmax, _d(c), _d(sg), mp, _d(dd), nlev, _d(lambdas), _d(eps), fptr,
                           max_iter, _d(s), _d(alm.view(np.float64)), iters.ctypes.data_as(_ip),
                           _d(cauchy))
    return dict(s=s, alm=alm, iters_per_level=iters, cauchy=cauchy[:n], iters=n)


def chi2(nside, lmax, cl, sigma, mask, d, s, alm):
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    mk, mp = _mask_ptr(mask)
    return lib().orc_chi2(nside, lmax, _d(c), _d(sg), mp, _d(np.ascontiguousarray(d, dtype=np.float64)),
                          _d(np.ascontiguousarray(s, dtype=np.float64)), _d(_c2r(alm)))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def gauss_pair(seed, c0, c1, c2):
    z0, z1 = ctypes.c_double(), ctypes.c_double()
    lib().orc_gauss_pair(ctypes.c_uint64(seed), ctypes.c_uint32(c0), ctypes.c_uint32(c1),
                         ctypes.c_uint32(c2), ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def draw_signal_alm(lmax, cl, seed):
    c = np.ascontiguousarray(cl, dtype=np.float64)
    alm = np.zeros((3, nalm(lmax)), dtype=np.complex128)
    lib().orc_draw_signal_alm(lmax, _d(c), ctypes.c_uint64(seed), _d(alm.view(np.float64)))
    return alm


def draw_noise(nside, sigma, mask, seed):
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    mk, mp = _mask_ptr(mask)
    n = np.zeros((3, npix(nside)))
    lib().orc_draw_noise(nside, _d(sg), mp, ctypes.c_uint64(seed), _d(n))
    return n


def cr_inputs(nside, lmax, cl, sigma, mask, seed):
    """(ahat, shat, dhat) of the constrained realisation (Section 2.2)."""
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    mk, mp = _mask_ptr(mask)
    ahat = np.zeros((3, nalm(lmax)), dtype=np.complex128)
    shat = np.zeros((3, npix(nside)))
    dhat = np.zeros((3, npix(nside)))
    lib().orc_cr_inputs(nside, lmax, _d(c), _d(sg), mp, ctypes.c_uint64(seed),
                        _d(ahat.view(np.float64)), _d(shat), _d(dhat))
    return ahat, shat, dhat


def constrained_realization(nside, lmax, cl, sigma, mask, d, seed, lambdas, eps=None, forced_iters=None,
                            max_iter=100000):
    """s_CR = W(d - dhat) + shat (Eq. 19).  Returns dict like dm_solve plus s_cr."""
    ahat, shat, dhat = cr_inputs(nside, lmax, cl, sigma, mask, seed)
    r = dm_solve(nside, lmax, cl, sigma, mask, np.asarray(d) - dhat, lambdas, eps, forced_iters, max_iter)
    r["s_cr"] = r["s"] + shat
    r["alm_cr"] = r["alm"] + ahat
    r["shat"], r["dhat"], r["ahat"] = shat, dhat, ahat
    return r


def draw_noise_cov(nside, sigma, rho, maskT, maskP, seed):
    """nhat ~ N of the correlated noise model (Sigma L z with the Philox normals)."""
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    mt, mtp = _mask_ptr(maskT)
    mp_, mpp = _mask_ptr(maskP)
    n = np.zeros((3, npix(nside)))
    lib().orc_draw_noise_cov(nside, _d(sg), _d(rh), mtp, mpp, ctypes.c_uint64(seed), _d(n))
    return n


def cr_inputs_cov(nside, lmax, cl, sigma, rho, maskT, maskP, seed):
    """(ahat, shat, dhat) of a constrained realisation under the correlated noise model."""
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    mt, mtp = _mask_ptr(maskT)
    mp_, mpp = _mask_ptr(maskP)
    ahat = np.zeros((3, nalm(lmax)), dtype=np.complex128)
    shat = np.zeros((3, npix(nside)))
    dhat = np.zeros((3, npix(nside)))
    lib().orc_cr_inputs_cov(nside, lmax, _d(c), _d(sg), _d(rh), mtp, mpp, ctypes.c_uint64(seed),
                            _d(ahat.view(np.float64)), _d(shat), _d(dhat))
    return ahat, shat, dhat


def constrained_realization_cov(nside, lmax, cl, sigma, rho, maskT, maskP, d, seed, lambdas, eps=None,
                                forced_iters=None, max_iter=100000):
    """s_CR = W(d - dhat) + shat (Eq. 19) under the correlated noise model."""
    ahat, shat, dhat = cr_inputs_cov(nside, lmax, cl, sigma, rho, maskT, maskP, seed)
    r = dm_solve_cov(nside, lmax, cl, sigma, rho, maskT, maskP, np.asarray(d) - dhat, lambdas, eps, forced_iters,
                     max_iter)
    r["s_cr"] = r["s"] + shat
    r["alm_cr"] = r["alm"] + ahat
    r["shat"], r["dhat"], r["ahat"] = shat, dhat, ahat
    return r


def cl_pinv(lmax, cl):
    """(C^+, range projector) per l in the filter-coefficient layout [lmax+1, 4]."""
    c = np.ascontiguousarray(cl, dtype=np.float64)
    pinv = np.zeros((lmax + 1, 4))
    proj = np.zeros((lmax + 1, 4))
    lib().orc_cl_pinv(lmax, _d(c), _d(pinv), _d(proj))
    return pinv, proj


def wf_residual(nside, lmax, cl, sigma, mask, d, alm):
    """||A x - y|| / ||y|| of the Wiener-filter equation at the iterate alm."""
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    a = np.ascontiguousarray(alm, dtype=np.complex128)
    m, mp = _mask_ptr(mask)
    return lib().orc_wf_residual(nside, lmax, _d(c), _d(sg), mp, _d(dd), _d(a.view(np.float64)))


def chi2_cov(nside, lmax, cl, sigma, rho, maskT, maskP, d, s, alm):
    """chi^2 of Eq. 3 with the correlated noise model (block N^-1)."""
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    ss = np.ascontiguousarray(s, dtype=np.float64)
    a = np.ascontiguousarray(alm, dtype=np.complex128)
    mt, mtp = _mask_ptr(maskT)
    mp_, mpp = _mask_ptr(maskP)
    return lib().orc_chi2_cov(nside, lmax, _d(c), _d(sg), _d(rh), mtp, mpp, _d(dd), _d(ss), _d(a.view(np.float64)))


def wf_residual_cov(nside, lmax, cl, sigma, rho, maskT, maskP, d, alm):
    """||A x - y|| / ||y|| with the correlated noise model (block N^-1)."""
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    a = np.ascontiguousarray(alm, dtype=np.complex128)
    mt, mtp = _mask_ptr(maskT)
    mp_, mpp = _mask_ptr(maskP)
    return lib().orc_wf_residual_cov(nside, lmax, _d(c), _d(sg), _d(rh), mtp, mpp, _d(dd), _d(a.view(np.float64)))


def jacobi_source(nside, lmax, cl, sigma, mask, d, alm):
    """P [A(w (d - Y a)) - alpha Omega C^+ a] (Appendix A, harmonic form)."""
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    a = np.ascontiguousarray(alm, dtype=np.complex128)
    m, mp = _mask_ptr(mask)
    g = np.zeros((3, nalm(lmax)), dtype=np.complex128)
    lib().orc_jacobi_source(nside, lmax, _d(c), _d(sg), mp, _d(dd), _d(a.view(np.float64)), _d(g.view(np.float64)))
    return g


def dm_frozen(nside, lmax, cl, sigma, mask, g, lambdas, counts):
    """W~(g): the dual messenger iteration at fixed per-level counts, driven by
    the harmonic source g, from a = 0."""
    c = np.ascontiguousarray(cl, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    gg = np.ascontiguousarray(g, dtype=np.complex128)
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    cnt = np.ascontiguousarray(counts, dtype=np.int32)
    m, mp = _mask_ptr(mask)
    a = np.zeros((3, nalm(lmax)), dtype=np.complex128)
    lib().orc_dm_frozen(nside, lmax, _d(c), _d(sg), mp, _d(gg.view(np.float64)), len(lam), _d(lam),
                        cnt.ctypes.data_as(_ip), _d(a.view(np.float64)))
    return a


def jacobi_refine(nside, lmax, cl, sigma, mask, d, lambdas, eps=None, forced_iters=None, n_refine=1,
                  max_iter=100000):
    """Appendix A: the usual solve (recording its per-level counts), then
    n_refine steps a <- a + W~(P g(a)) at those counts."""
    r = dm_solve(nside, lmax, cl, sigma, mask, d, lambdas, eps, forced_iters, max_iter)
    counts = np.asarray(r["iters_per_level"], dtype=np.int32)
    a = r["alm"]
    steps = [a]
    for _ in range(n_refine):
        a = a + dm_frozen(nside, lmax, cl, sigma, mask, jacobi_source(nside, lmax, cl, sigma, mask, d, a),
                          lambdas, counts)
        steps.append(a)
    return {"alm": a, "s": alm2map(nside, lmax, a), "counts": counts, "steps": steps, "solve": r}


def level_lambdas(lambda0, nlev):
    """Geometric cooling lambda_k = lambda0^(1 - k/(nlev-1)), last level exactly 1."""
    if nlev == 1:
        return np.array([1.0])
    lam = np.array([lambda0 ** (1.0 - k / (nlev - 1)) for k in range(nlev)])
    lam[-1] = 1.0
    return lam
