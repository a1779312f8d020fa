"""Synthetic workloads shaped like the paper's (Section 3.1), carried onto the
HEALPix sphere.

The paper simulates flat-sky T/Q/U maps from CAMB spectra with a Cholesky draw
of (T, E, B) harmonic coefficients, adds correlated noise and applies T and P
masks (Section 3.1).  None of those data exist here, so this module stands in
for them with analytic spectra, an inhomogeneous diagonal noise model and
band-plus-disk masks.  Nothing here is part of the method: the transforms, the
filter and the messenger loop live in the CUDA library (product) and in the
oracle (test infrastructure).  Both receive these arrays as plain data.

Recipe (all seeded through numpy's PCG64 via SeedSequence):

* spectra: C_l^TT = exp(-(l/40)^2) / (l(l+1)) for l >= 1, C_0^TT = 0;
  C^EE = 0.05 C^TT, C^BB = 0.01 C^EE, C^TE = 0.3 sqrt(C^TT C^EE), polarisation
  only from l = 2;
* signal: a_lm drawn from the per-l 2x2 TE block by Cholesky, B independent;
  m = 0 real, m > 0 with re and im at half variance;
* noise: sigma_T = s0 (1 + 2|cos theta|)(0.5 + U(0,1)) per pixel with s0 = 10 %
  of the analytic T rms sqrt(sum (2l+1) C_l^TT / 4pi); sigma_Q = sigma_U =
  sqrt(2) sigma_T; an optional (1 + cos^2 theta) scan-depth factor;
* mask: |z| < band removed, plus disks (centres uniform on the sphere), a pixel
  is masked when its centre lies inside a disk.

The flat-sky section at the end keeps the paper's own geometry (a 10 degree
patch on a 1024^2 grid, T and P masks of f_sky 0.78 and 0.82) with the same
stand-in spectra evaluated at each Fourier mode's |l|.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ARCMIN = np.pi / (180.0 * 60.0)
DEG = np.pi / 180.0


def cl_analytic(lmax: int, lscale: float = 40.0) -> np.ndarray:
    """[4, lmax+1] = TT, EE, BB, TE."""
    ell = np.arange(lmax + 1, dtype=np.float64)
    tt = np.zeros(lmax + 1)
    tt[1:] = np.exp(-(ell[1:] / lscale) ** 2) / (ell[1:] * (ell[1:] + 1.0))
    ee = 0.05 * tt
    bb = 0.01 * ee
    te = 0.3 * np.sqrt(tt * ee)
    ee[:2] = 0.0
    bb[:2] = 0.0
    te[:2] = 0.0
    return np.stack([tt, ee, bb, te])


def signal_rms(cl: np.ndarray) -> float:
    ell = np.arange(cl.shape[1])
    return float(np.sqrt(np.sum((2 * ell + 1) * cl[0]) / (4 * np.pi)))


def pixel_centers(nside: int):
    """(z, phi) of every HEALPix pixel in RING order (Gorski et al. 2005)."""
    ns = nside
    npix = 12 * ns * ns
    p = np.arange(npix, dtype=np.int64)
    z = np.empty(npix)
    phi = np.empty(npix)
    ncap = 2 * ns * (ns - 1)
    # north cap
    north = p < ncap
    pn = p[north]
    i = ((1 + np.sqrt(1 + 2 * pn)) / 2).astype(np.int64)
    i = np.where(2 * i * (i - 1) > pn, i - 1, i)
    i = np.where(2 * (i + 1) * i <= pn, i + 1, i)
    j = pn - 2 * i * (i - 1)
    z[north] = 1 - i * i / (3.0 * ns * ns)
    phi[north] = (j + 0.5) * np.pi / (2.0 * i)
    # equatorial belt
    eq = (p >= ncap) & (p < npix - ncap)
    pe = p[eq] - ncap
    i = pe // (4 * ns) + ns
    j = pe % (4 * ns)
    shift = ((i - ns + 1) % 2 == 1).astype(np.float64) * 0.5
    z[eq] = 4.0 / 3.0 - 2.0 * i / (3.0 * ns)
    phi[eq] = (j + shift) * np.pi / (2.0 * ns)
    # south cap (mirror)
    south = p >= npix - ncap
    ps = npix - 1 - p[south]
    i = ((1 + np.sqrt(1 + 2 * ps)) / 2).astype(np.int64)
    i = np.where(2 * i * (i - 1) > ps, i - 1, i)
    i = np.where(2 * (i + 1) * i <= ps, i + 1, i)
    jr = ps - 2 * i * (i - 1)  # counted from the end of the ring
    j = 4 * i - 1 - jr
    z[south] = -(1 - i * i / (3.0 * ns * ns))
    phi[south] = (j + 0.5) * np.pi / (2.0 * i)
    return z, phi


def noise_sigma(nside: int, cl: np.ndarray, rng: np.random.Generator, scan_depth: bool = False,
                level: float = 0.1) -> np.ndarray:
    """[3, npix] per-pixel noise std-dev (I, Q, U)."""
    z, _ = pixel_centers(nside)
    s0 = level * signal_rms(cl)
    st = s0 * (1.0 + 2.0 * np.abs(z)) * (0.5 + rng.random(z.size))
    if scan_depth:
        st = st * (1.0 + z * z)
    return np.stack([st, np.sqrt(2.0) * st, np.sqrt(2.0) * st])


def mask_band_disks(nside: int, rng: np.random.Generator, band: float, disks) -> np.ndarray:
    """uint8 [npix], 1 = observed.  disks: list of (count, radius_rad) or
    (count, (rmin, rmax)) with radii uniform in [rmin, rmax]."""
    z, phi = pixel_centers(nside)
    obs = np.abs(z) >= band
    sth = np.sqrt(np.maximum(0.0, 1 - z * z))
    vx, vy, vz = sth * np.cos(phi), sth * np.sin(phi), z
    for count, rad in disks:
        cz = rng.uniform(-1.0, 1.0, count)
        cphi = rng.uniform(0.0, 2 * np.pi, count)
        if np.isscalar(rad):
            radii = np.full(count, float(rad))
        else:
            radii = rng.uniform(rad[0], rad[1], count)
        cs = np.sqrt(1 - cz * cz)
        cx, cy = cs * np.cos(cphi), cs * np.sin(cphi)
        # a pixel within angle r of the centre has |z - z_c| < r (|d cos / d theta| <= 1);
        # z does not increase along RING order, so the candidates are one index range
        negz = -z
        for k in range(count):
            lo = np.searchsorted(negz, -(cz[k] + radii[k]) - 1e-12, side="left")
            hi = np.searchsorted(negz, -(cz[k] - radii[k]) + 1e-12, side="right")
            sl = slice(lo, hi)
            cosd = vx[sl] * cx[k] + vy[sl] * cy[k] + vz[sl] * cz[k]
            obs[sl] &= cosd < np.cos(radii[k])
    return obs.astype(np.uint8)


def draw_alm(lmax: int, cl: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Gaussian (T, E, B) harmonic coefficients [3, nalm] complex128, m-major."""
    tt, ee, bb, te = cl
    nalm = (lmax + 1) * (lmax + 2) // 2
    ls = np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])
    ms = np.concatenate([np.full(lmax + 1 - m, m) for m in range(lmax + 1)])
    zr = rng.standard_normal((3, nalm))
    zi = rng.standard_normal((3, nalm))
    l11 = np.sqrt(np.maximum(tt, 0.0))
    l21 = np.where(l11 > 0, te / np.where(l11 > 0, l11, 1.0), 0.0)
    l22 = np.sqrt(np.maximum(ee - l21 ** 2, 0.0))
    lbb = np.sqrt(np.maximum(bb, 0.0))
    scale = np.where(ms == 0, 1.0, np.sqrt(0.5))
    zc = zr + 1j * np.where(ms == 0, 0.0, zi)
    alm = np.empty((3, nalm), dtype=np.complex128)
    alm[0] = scale * l11[ls] * zc[0]
    alm[1] = scale * (l21[ls] * zc[0] + l22[ls] * zc[1])
    alm[2] = scale * lbb[ls] * zc[2]
    return alm


def draw_noise(sigma: np.ndarray, mask: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    return sigma * rng.standard_normal(sigma.shape) * mask[None, :]


@dataclass
class Workload:
    """One synthetic problem: spectra, noise, mask and the true signal alm."""
    name: str
    nside: int
    lmax: int
    cl: np.ndarray
    sigma: np.ndarray
    mask: np.ndarray
    alm_true: list = field(default_factory=list)   # per RHS [3, nalm]
    noise: list = field(default_factory=list)      # per RHS [3, npix]
    seeds: list = field(default_factory=list)

    @property
    def npix(self):
        return 12 * self.nside * self.nside

    def data(self, signal_maps):
        """d = s + n on observed pixels, 0 on masked ones (Eq. 1)."""
        return [(s + n) * self.mask[None, :] for s, n in zip(signal_maps, self.noise)]


def _streams(seed: int, n: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(n)]


# Workload recipes.  Sizes follow the five benchmark configurations: nside 16 /
# 256 / 512 / 2048 and the serving mix.
CONFIGS = {
    "nside16": dict(nside=16, lmax=47, band=0.2, disks=[(10, 3.0 * DEG)], scan=False),
    "nside256": dict(nside=256, lmax=512, band=0.2, disks=[(10, 3.0 * DEG), (50, 0.5 * DEG)], scan=False),
    "nside512": dict(nside=512, lmax=1024, band=0.2, disks=[(10, 3.0 * DEG), (50, 0.5 * DEG)], scan=False),
    "nside2048": dict(nside=2048, lmax=4096, band=0.3, disks=[(2000, (5 * ARCMIN, 30 * ARCMIN))], scan=True),
}


def make_workload(name: str, seeds, nside: int | None = None, lmax: int | None = None,
                  with_signal: bool = True) -> Workload:
    """Spectra, noise sigma and mask from the first seed; per-RHS signal alm and
    noise realisation from each seed."""
    cfg = dict(CONFIGS[name])
    if nside is not None:
        cfg["nside"] = nside
        cfg["lmax"] = lmax if lmax is not None else 2 * nside
    ns, lm = cfg["nside"], cfg["lmax"]
    seeds = list(seeds)
    cl = cl_analytic(lm)
    r_sigma, r_mask = _streams(seeds[0] * 7919 + 1, 2)
    sigma = noise_sigma(ns, cl, r_sigma, scan_depth=cfg["scan"])
    mask = mask_band_disks(ns, r_mask, cfg["band"], cfg["disks"])
    wl = Workload(name=name, nside=ns, lmax=lm, cl=cl, sigma=sigma, mask=mask, seeds=seeds)
    for sd in seeds:
        r_sig, r_noise = _streams(sd, 2)
        wl.alm_true.append(draw_alm(lm, cl, r_sig) if with_signal else None)
        wl.noise.append(draw_noise(sigma, mask, r_noise))
    return wl


def lambda_schedule(lambda0: float = 1000.0, nlev: int = 10) -> np.ndarray:
    """Geometric cooling 1000 -> 1 over nlev levels (last exactly 1)."""
    lam = np.array([lambda0 ** (1.0 - k / (nlev - 1)) for k in range(nlev)])
    lam[-1] = 1.0
    return lam


def eps_schedule(nlev: int, eps0: float = 1e-4, eps_final: float = 1e-6) -> np.ndarray:
    """Cauchy thresholds cooled geometrically from eps0 to eps_final."""
    return np.array([eps0 * (eps_final / eps0) ** (k / (nlev - 1)) for k in range(nlev)])


def random_maps(nside: int, nmaps: int, seed: int) -> np.ndarray:
    """Unstructured N(0,1) test maps [nmaps, 3, npix] (transform parity inputs)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nmaps, 3, 12 * nside * nside))


def random_alm(lmax: int, nalm_sets: int, seed: int, cl: np.ndarray | None = None) -> np.ndarray:
    """Random harmonic coefficients [n, 3, nalm] (real-field valid: m = 0 real,
    E/B zero for l < 2).  White unless cl is given."""
    rng = np.random.default_rng(seed)
    if cl is None:
        cl = np.ones((4, lmax + 1))
        cl[3] = 0.0
        cl[1:3, :2] = 0.0
    return np.stack([draw_alm(lmax, cl, rng) for _ in range(nalm_sets)])


def serving_stream(n: int, seed: int, nsides=(64, 128, 256, 512, 1024), p_wf: float = 0.7,
                   tols=(1e-5, 1e-8)) -> list:
    """The serving mix: n requests with nside drawn uniformly from nsides,
    lmax = 2 nside, Wiener filter with probability p_wf (else constrained
    realisation), tolerance drawn uniformly from tols, and a per-request seed
    (its mask, noise and signal come from make_workload with that seed).
    Arrival times are drawn separately (poisson_arrivals), so the same mix
    can be replayed at any rate."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        ns = int(rng.choice(nsides))
        out.append(dict(nside=ns, lmax=2 * ns, kind=0 if rng.random() < p_wf else 1,
                        tol=float(rng.choice(tols)), seed=int(seed) * 100000 + i))
    return out


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate (1/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


# Correlated noise with distinct temperature and polarisation masks (the 3x3
# per-pixel noise covariance of the paper's Section 2.1 and Appendix B).

def noise_correlations(nside: int, rng: np.random.Generator, rho_max: float = 0.3) -> np.ndarray:
    """[3, npix] correlation coefficients (rho_IQ, rho_IU, rho_QU), uniform in
    [-rho_max, rho_max]; with rho_max <= 0.3 every correlation matrix is
    diagonally dominant, hence positive definite."""
    return rng.uniform(-rho_max, rho_max, size=(3, 12 * nside * nside))


def draw_noise_cov(sigma: np.ndarray, rho: np.ndarray, mask_t: np.ndarray, mask_p: np.ndarray,
                   rng: np.random.Generator) -> np.ndarray:
    """[3, npix] noise n = Sigma L z per pixel (C = L L^T, z ~ N(0, 1)), zero on
    masked components (the temperature mask for I, the polarisation mask for Q
    and U)."""
    npix = sigma.shape[1]
    C = np.empty((npix, 3, 3))
    C[:, 0, 0] = C[:, 1, 1] = C[:, 2, 2] = 1.0
    C[:, 0, 1] = C[:, 1, 0] = rho[0]
    C[:, 0, 2] = C[:, 2, 0] = rho[1]
    C[:, 1, 2] = C[:, 2, 1] = rho[2]
    L = np.linalg.cholesky(C)
    z = rng.standard_normal((npix, 3))
    n = sigma.T * np.einsum("pij,pj->pi", L, z)
    obs = np.stack([mask_t, mask_p, mask_p], axis=1)
    return (n * obs).T.copy()


@dataclass
class CovWorkload(Workload):
    """A Workload with correlated noise: mask is the temperature mask,
    mask_p the polarisation mask, rho the per-pixel correlations."""
    rho: np.ndarray = None
    mask_p: np.ndarray = None

    def data(self, signal_maps):
        """d = s + n on observed components, 0 on masked ones."""
        obs = np.stack([self.mask, self.mask_p, self.mask_p])
        return [(s + n) * obs for s, n in zip(signal_maps, self.noise)]


def make_cov_workload(seeds, nside: int, lmax: int | None = None, band_t: float = 0.215, band_p: float = 0.175,
                      rho_max: float = 0.3) -> CovWorkload:
    """The nside 16 recipe with correlated noise and distinct masks: a |z| <
    band_t band plus 10 disks of 3 degrees masks temperature, a |z| < band_p
    band plus 10 other 3-degree disks masks polarisation (sky fractions near
    0.78 and 0.82, as in the paper's run); spectra, sigma, masks and rho from
    the first seed, signal and noise per seed."""
    lm = lmax if lmax is not None else 2 * nside
    seeds = list(seeds)
    cl = cl_analytic(lm)
    r_sigma, r_mask_t, r_mask_p, r_rho = _streams(seeds[0] * 7919 + 3, 4)
    sigma = noise_sigma(nside, cl, r_sigma)
    mask_t = mask_band_disks(nside, r_mask_t, band_t, [(10, 3.0 * DEG)])
    mask_p = mask_band_disks(nside, r_mask_p, band_p, [(10, 3.0 * DEG)])
    rho = noise_correlations(nside, r_rho, rho_max)
    wl = CovWorkload(name="cov", nside=nside, lmax=lm, cl=cl, sigma=sigma, mask=mask_t, seeds=seeds, rho=rho,
                     mask_p=mask_p)
    for sd in seeds:
        r_sig, r_noise = _streams(sd, 2)
        wl.alm_true.append(draw_alm(lm, cl, r_sig))
        wl.noise.append(draw_noise_cov(sigma, rho, mask_t, mask_p, r_noise))
    return wl


# ----------------------------------------------------------------- flat sky
# The paper's own setting (Section 3.1): a square patch of side L = 10 degrees
# on an N x N grid (N = 1024), T and P masks covering f_sky = 0.78 and 0.82,
# noise of a few uK.  Stand-ins, as on the sphere: the analytic spectra
# evaluated at the real |l| of each Fourier mode, with a damping scale that
# reaches the patch's multipoles (l from 2 pi / L = 36 to the Nyquist l =
# pi N / L); inhomogeneous diagonal noise; masks made of a strip and disks.
#
# Fourier convention shared with the consumers of these arrays: a mode of
# integer wavenumber (k_x, k_y), numpy FFT order, axis 0 = y and axis 1 = x,
# has l = 2 pi k / L and <|a_l|^2> = L^2 C_|l|.  Modes on the Nyquist row or
# column (k = -N/2) carry no signal.

FLAT_L = 10.0 * DEG
FLAT_N = 1024
FLAT_LSCALE = 1500.0


def flat_ell(N: int, L: float) -> np.ndarray:
    """|l| of every mode of an N x N grid of side L (numpy FFT order)."""
    k = np.fft.fftfreq(N, d=1.0 / N)
    return 2.0 * np.pi / L * np.hypot(k[:, None], k[None, :])


def flat_nyquist(N: int) -> np.ndarray:
    """True on the Nyquist row and column of an even N (no such modes for odd N)."""
    k = np.fft.fftfreq(N, d=1.0 / N)
    ny = (k == -(N // 2)) if N % 2 == 0 else np.zeros(N, bool)
    return ny[:, None] | ny[None, :]


def cl_flat(ell: np.ndarray, lscale: float = FLAT_LSCALE) -> np.ndarray:
    """[4, ...] = TT, EE, BB, TE at real multipoles ell: the sphere recipe's
    formulas with damping scale lscale; 0 at l = 0 and polarisation only
    from l = 2."""
    ell = np.asarray(ell, dtype=np.float64)
    pos = ell > 0
    safe = np.where(pos, ell, 1.0)
    tt = np.where(pos, np.exp(-(safe / lscale) ** 2) / (safe * (safe + 1.0)), 0.0)
    pol = ell >= 2
    ee = np.where(pol, 0.05 * tt, 0.0)
    bb = 0.01 * ee
    te = np.where(pol, 0.3 * np.sqrt(tt * ee), 0.0)
    return np.stack([tt, ee, bb, te])


def flat_spectra(N: int, L: float, lscale: float = FLAT_LSCALE) -> np.ndarray:
    """[4, N, N] spectra per Fourier mode, 0 on the Nyquist row and column."""
    return cl_flat(flat_ell(N, L), lscale) * ~flat_nyquist(N)


def draw_flat_alm(S: np.ndarray, L: float, rng: np.random.Generator) -> np.ndarray:
    """Gaussian (T, E, B) Fourier coefficients [3, N, N] complex128 with
    <|a_l|^2> = L^2 C_l and the Hermitian symmetry of real fields, from the
    per-mode 2x2 TE Cholesky factor (B independent): unit white-noise maps,
    Fourier transformed and scaled by L / N per mode."""
    tt, ee, bb, te = S
    N = S.shape[-1]
    z = np.fft.fft2(rng.standard_normal((3, N, N)), axes=(-2, -1)) * (L / N)
    l11 = np.sqrt(np.maximum(tt, 0.0))
    l21 = np.where(l11 > 0, te / np.where(l11 > 0, l11, 1.0), 0.0)
    l22 = np.sqrt(np.maximum(ee - l21 ** 2, 0.0))
    lbb = np.sqrt(np.maximum(bb, 0.0))
    return np.stack([l11 * z[0], l21 * z[0] + l22 * z[1], lbb * z[2]])


def flat_noise_sigma(N: int, L: float, S: np.ndarray, rng: np.random.Generator, level: float = 0.04):
    """sigma_T = s0 (0.75 + 0.5 U(0,1)) per pixel with s0 = level x the analytic
    T rms of the patch, sqrt(sum_l C_l^TT) / L; sigma_Q = sigma_U = sqrt(2) sigma_T."""
    s0 = level * np.sqrt(S[0].sum()) / L
    st = s0 * (0.75 + 0.5 * rng.random((N, N)))
    return np.stack([st, np.sqrt(2.0) * st, np.sqrt(2.0) * st])


def flat_mask(N: int, rng: np.random.Generator, fsky: float, strip: float = 0.1) -> np.ndarray:
    """uint8 [N, N], 1 = observed: a horizontal strip of height strip x N through
    the middle, then disks of radius 1 to 4 % of N at uniform centres until
    the observed fraction drops to fsky."""
    y, x = np.mgrid[0:N, 0:N]
    m = np.ones((N, N), np.uint8)
    h = int(round(strip * N))
    m[(N - h) // 2:(N - h) // 2 + h, :] = 0
    while m.mean() > fsky:
        cy, cx = rng.random(2) * N
        r = N * (0.01 + 0.03 * rng.random())
        m[(y - cy) ** 2 + (x - cx) ** 2 < r * r] = 0
    return m


@dataclass
class FlatWorkload:
    """One flat-sky problem: spectra per mode, noise, T and P masks, the true
    (T, E, B) Fourier coefficients per RHS and their noise realisations."""
    N: int
    L: float
    S: np.ndarray                 # [4, N, N] TT, EE, BB, TE per mode
    sigma: np.ndarray             # [3, N, N]
    mask_t: np.ndarray            # [N, N]
    mask_p: np.ndarray            # [N, N]
    alm_true: list = field(default_factory=list)
    noise: list = field(default_factory=list)
    seeds: list = field(default_factory=list)
    rho: np.ndarray | None = None  # [3, N, N] (rho_IQ, rho_IU, rho_QU) when the noise is correlated

    def data(self, signal_maps):
        """d = s + n on observed components, 0 on masked ones."""
        obs = np.stack([self.mask_t, self.mask_p, self.mask_p])
        return [(s + n) * obs for s, n in zip(signal_maps, self.noise)]


def make_flat_workload(seeds, N: int = FLAT_N, L: float = FLAT_L, lscale: float = FLAT_LSCALE,
                       fsky_t: float = 0.78, fsky_p: float = 0.82, level: float = 0.04,
                       rho_max: float = 0.0) -> FlatWorkload:
    """Spectra, noise sigma and masks from the first seed; per-RHS signal and
    noise draws from each seed.  With rho_max > 0 the noise is correlated
    across I, Q and U as in the paper's run: per-pixel correlations uniform in
    [-rho_max, rho_max] and n = Sigma L z (draw_noise_cov)."""
    seeds = list(seeds)
    S = flat_spectra(N, L, lscale)
    r_sigma, r_mt, r_mp = _streams(seeds[0] * 7919 + 3, 3)
    sigma = flat_noise_sigma(N, L, S, r_sigma, level)
    mask_t = flat_mask(N, r_mt, fsky_t)
    mask_p = flat_mask(N, r_mp, fsky_p)
    wl = FlatWorkload(N=N, L=L, S=S, sigma=sigma, mask_t=mask_t, mask_p=mask_p, seeds=seeds)
    if rho_max > 0:
        wl.rho = _streams(seeds[0] * 7919 + 5, 1)[0].uniform(-rho_max, rho_max, (3, N, N))
    for sd in seeds:
        r_sig, r_noise = _streams(sd + 104729, 2)
        wl.alm_true.append(draw_flat_alm(S, L, r_sig))
        if wl.rho is None:
            wl.noise.append(sigma * r_noise.standard_normal(sigma.shape))
        else:
            n = draw_noise_cov(sigma.reshape(3, -1), wl.rho.reshape(3, -1), mask_t.ravel(), mask_p.ravel(), r_noise)
            wl.noise.append(n.reshape(3, N, N))
    return wl
