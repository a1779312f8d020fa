"""Flat-sky dual messenger oracle: the paper's own setting (Section 2.1,
Eqs. 12-16, Algorithm 1) on a square patch of side L with N x N pixels.

TEST INFRASTRUCTURE ONLY: tests/ call it, and the CUDA product path never
imports it.  Plain numpy in float64; numpy's FFT is the only library step.

Conventions:

* pixel (row i, column j) sits at x = j L / N, y = i L / N (axis 0 is y,
  axis 1 is x) and has area Omega_p = (L / N)^2;
* a mode of integer wavenumber (k_x, k_y) in numpy FFT order has
  l = 2 pi k / L; phi_l is the angle between l and the l_x axis;
* F^dagger (analysis): a_l = Omega_p sum_x m(x) e^{-i l.x}; F (synthesis):
  m(x) = L^-2 sum_l a_l e^{i l.x}.  F^dagger F is the identity on the harmonic
  space, the exact inverse that Algorithm 1 writes as sigma^-1 F^dagger;
* temperature a^T = F^dagger I; polarisation by the rotation of Eqs. 13-16,
  Q = E cos 2phi - B sin 2phi and U = E sin 2phi + B cos 2phi per mode, and its
  inverse E = Q cos 2phi + U sin 2phi, B = -Q sin 2phi + U cos 2phi;
* the Nyquist row and column of an even N (k_x or k_y = -N/2) are not part of
  the harmonic space: a mode there is its own conjugate partner, so the
  rotation by the angle of l could not keep real fields real.  Analysis
  drops them;
* <|a_l|^2> = L^2 C_|l| for a patch of area L^2, and the noise of a pixel
  with variance alpha has Fourier power L^2 Omega_p alpha.  So the per-mode
  filter takes C_l and T_h = alpha Omega_p, as on the sphere.

Because F^dagger F = 1 here, the iteration is Algorithm 1 as printed:
a = (S-bar + U)(S-bar + xi)^-1 F^dagger t, s = F a, t = (1 - w) s + w d with
w = alpha / N per pixel-component (0 where masked).
"""
from __future__ import annotations

import numpy as np


def geometry(N: int, L: float):
    """(l_x, l_y, phi, keep) per mode of an N x N grid of side L; keep is False
    on the Nyquist row and column of an even N."""
    k = np.fft.fftfreq(N, d=1.0 / N)
    ky, kx = np.meshgrid(k, k, indexing="ij")
    lx, ly = 2.0 * np.pi * kx / L, 2.0 * np.pi * ky / L
    phi = np.arctan2(ly, lx)
    keep = np.ones((N, N), bool)
    if N % 2 == 0:
        keep &= (kx != -(N // 2)) & (ky != -(N // 2))
    return lx, ly, phi, keep


def analysis(maps: np.ndarray, L: float) -> np.ndarray:
    """(I, Q, U) maps [3, N, N] -> (T, E, B) Fourier coefficients [3, N, N]."""
    N = maps.shape[-1]
    _, _, phi, keep = geometry(N, L)
    h = (L / N) ** 2 * np.fft.fft2(maps, axes=(-2, -1))
    c, s = np.cos(2.0 * phi), np.sin(2.0 * phi)
    t = h[0]
    e = h[1] * c + h[2] * s
    b = -h[1] * s + h[2] * c
    return np.stack([t, e, b]) * keep


def synthesis(alm: np.ndarray, L: float) -> np.ndarray:
    """(T, E, B) Fourier coefficients [3, N, N] -> real (I, Q, U) maps.  The
    coefficients of real fields are Hermitian; the imaginary part the inverse
    FFT leaves is rounding and is dropped."""
    N = alm.shape[-1]
    _, _, phi, keep = geometry(N, L)
    a = alm * keep
    c, s = np.cos(2.0 * phi), np.sin(2.0 * phi)
    h = np.stack([a[0], a[1] * c - a[2] * s, a[1] * s + a[2] * c])
    return (np.fft.ifft2(h, axes=(-2, -1)) * (N * N / L ** 2)).real


def filter_coefs(S: np.ndarray, mu: float, th: float) -> np.ndarray:
    """Per-mode filter (S-bar + U)(S-bar + xi)^-1 of Algorithm 1 with
    S-bar = max(S_e - mu, 0) on the eigenvalues S_e of the mode's 3x3 block
    (Eq. 10), so that S-bar + U = max(S_e, mu) and S-bar + xi = that + T_h.
    Returns [4, N, N]: the symmetric TE block (f_TT, f_TE, f_EE) and f_BB."""
    tt, ee, bb, te = S
    blk = np.stack([np.stack([tt, te], -1), np.stack([te, ee], -1)], -2)  # [N, N, 2, 2]
    e, v = np.linalg.eigh(blk)
    sp = np.maximum(np.maximum(e, 0.0), mu)
    f = sp / (sp + th)
    F = np.einsum("...ik,...k,...jk->...ij", v, f, v)
    sb = np.maximum(np.maximum(bb, 0.0), mu)
    return np.stack([F[..., 0, 0], F[..., 0, 1], F[..., 1, 1], sb / (sb + th)])


def apply_filter(coef: np.ndarray, a: np.ndarray) -> np.ndarray:
    return np.stack([coef[0] * a[0] + coef[1] * a[1], coef[1] * a[0] + coef[2] * a[1], coef[3] * a[2]])


def weights(sigma: np.ndarray, mask_t: np.ndarray, mask_p: np.ndarray):
    """(alpha, w): alpha = min N over observed pixel-components (T = alpha 1,
    Section 2), w = alpha / N there and 0 where masked (N^-1 = 0)."""
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    var = sigma ** 2
    alpha = var[obs].min()
    return alpha, np.where(obs, alpha / np.where(obs, var, 1.0), 0.0)


def dm_solve(d, sigma, mask_t, mask_p, S, L, lambdas, eps=None, forced_iters=None, max_iter=100000):
    """Algorithm 1 on the flat patch.  d, sigma [3, N, N]; masks [N, N] (1 =
    observed); S [4, N, N] spectra per mode; lambdas the cooling levels
    (lambda = xi / T_h, mu = (lambda - 1) T_h); per level either a Cauchy
    threshold eps[k] on ||s_i - s_{i-1}|| / ||s_i|| or a fixed count
    forced_iters[k].  Returns s, alm and the iteration record."""
    d = np.asarray(d, dtype=np.float64)
    N = d.shape[-1]
    alpha, w = weights(sigma, mask_t, mask_p)
    th = alpha * (L / N) ** 2
    obs = w > 0
    s = np.zeros_like(d)
    t = np.where(obs, d, 0.0)
    a = np.zeros((3, N, N), np.complex128)
    iters_per_level, cauchy = [], []
    it = 0
    for k, lam in enumerate(lambdas):
        coef = filter_coefs(S, (lam - 1.0) * th, th)
        nk = 0
        while True:
            if forced_iters is not None and nk >= forced_iters[k]:
                break
            if forced_iters is None and it >= max_iter:
                break
            a = apply_filter(coef, analysis(t, L))
            sn = synthesis(a, L)
            ss = np.sum(sn * sn)
            c = np.sqrt(np.sum((sn - s) ** 2) / ss) if ss > 0 else 0.0
            s = sn
            t = (1.0 - w) * s + w * d
            cauchy.append(c)
            it += 1
            nk += 1
            if forced_iters is None and c < eps[k]:
                break
        iters_per_level.append(nk)
    return {"s": s, "alm": a, "iters": it, "iters_per_level": np.array(iters_per_level),
            "cauchy": np.array(cauchy), "alpha": alpha}


def _block_pow(S: np.ndarray, p: float):
    """Per-mode powers of the signal covariance block for the parameters it
    constrains: [4, N, N] (TE block entries and BB) of V diag(S_e^p) V^T over
    the eigenvalues S_e > 0, 0 on the null directions (a pseudo-inverse)."""
    tt, ee, bb, te = S
    blk = np.stack([np.stack([tt, te], -1), np.stack([te, ee], -1)], -2)
    e, v = np.linalg.eigh(blk)
    tiny = 1e-300
    ep = np.where(e > tiny, np.where(e > tiny, e, 1.0) ** p, 0.0)
    M = np.einsum("...ik,...k,...jk->...ij", v, ep, v)
    bp = np.where(bb > tiny, np.where(bb > tiny, bb, 1.0) ** p, 0.0)
    return np.stack([M[..., 0, 0], M[..., 0, 1], M[..., 1, 1], bp])


def wf_residual(alm, d, sigma, mask_t, mask_p, S, L):
    """||A x - y|| / ||y|| of the Wiener filter in the form A x = y with
    A = 1 + S^1/2 F^H N^-1 F S^1/2, x = S^-1/2 a and y = S^1/2 F^H N^-1 d,
    where F is the synthesis and F^H its adjoint (the diagnostic the paper
    reports beside its solutions, Section 3.2 and Appendix C).  Here <a a^H> = L^2 C per mode,
    the adjoint of F (synthesis) is analysis / (Omega_p L^2), and N^-1 = 0 on
    masked pixel-components."""
    N = d.shape[-1]
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    ninv = np.where(obs, 1.0 / np.where(obs, sigma ** 2, 1.0), 0.0)
    adj = lambda m: analysis(m, L) / ((L / N) ** 2 * L ** 2)
    Sa = S * L ** 2
    half, mhalf = _block_pow(Sa, 0.5), _block_pow(Sa, -0.5)
    y = apply_filter(half, adj(ninv * d))
    r = apply_filter(mhalf, alm) - apply_filter(half, adj(ninv * (d - synthesis(alm, L))))
    return float(np.sqrt(np.sum(np.abs(r) ** 2) / np.sum(np.abs(y) ** 2)))


def chi2(alm, d, sigma, mask_t, mask_p, S, L):
    """(d - s)^T N^-1 (d - s) over observed pixel-components plus
    sum over modes a^H S^-1 a with <a a^H> = L^2 C (Eq. 3), S^-1 taken on the
    non-zero eigenvalues of each mode's block."""
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    s = synthesis(alm, L)
    r = (d - s)[obs]
    noise = np.sum(r * r / (sigma[obs] ** 2))
    inv = _block_pow(S * L ** 2, -1.0)
    prior = np.sum(np.real(np.conj(alm) * apply_filter(inv, alm)))
    return float(noise + prior)


# ------------------------------------------------- correlated noise (App. B)
# The paper's own noise model: per pixel N = Sigma C Sigma with C the
# unit-diagonal correlation matrix of (rho_IQ, rho_IU, rho_QU).  Masks enter
# as Sigma^-1 = 0 on masked components (I on the temperature mask, Q and U on
# the polarisation mask), so N^-1 = Sigma^-1 C^-1 Sigma^-1 with zero rows and
# columns there.  T = alpha 1 with alpha the smallest eigenvalue of N over the
# observed components, alpha = min over pixels of 1 / lambda_max(N^-1).  The
# messenger equation of Appendix B then reads t = s + alpha N^-1 (d - s).


def cov_ninv(sigma, rho, mask_t, mask_p):
    """[3, 3, N, N] per-pixel N^-1 with masked components' rows and columns 0."""
    r01, r02, r12 = rho
    one = np.ones_like(r01)
    C = np.stack([np.stack([one, r01, r02]), np.stack([r01, one, r12]), np.stack([r02, r12, one])])
    Ci = np.moveaxis(np.linalg.inv(np.moveaxis(C, (0, 1), (-2, -1))), (-2, -1), (0, 1))
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    si = np.where(obs, 1.0 / np.where(obs, sigma, 1.0), 0.0)
    return si[:, None] * Ci * si[None, :]


def cov_alpha(ninv):
    lam = np.linalg.eigvalsh(np.moveaxis(ninv, (0, 1), (-2, -1)))[..., -1]
    return float(1.0 / lam[lam > 0].max())


def dm_solve_cov(d, sigma, rho, mask_t, mask_p, S, L, lambdas, eps=None, forced_iters=None, max_iter=100000):
    """Algorithm 1 on the flat patch with the correlated noise model: as
    dm_solve, with the messenger update t = s + alpha N^-1 (d - s)."""
    d = np.asarray(d, dtype=np.float64)
    N = d.shape[-1]
    ninv = cov_ninv(sigma, rho, mask_t, mask_p)
    alpha = cov_alpha(ninv)
    th = alpha * (L / N) ** 2
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    s = np.zeros_like(d)
    t = np.where(obs, d, 0.0)
    a = np.zeros((3, N, N), np.complex128)
    iters_per_level, cauchy = [], []
    it = 0
    for k, lam in enumerate(lambdas):
        coef = filter_coefs(S, (lam - 1.0) * th, th)
        nk = 0
        while True:
            if forced_iters is not None and nk >= forced_iters[k]:
                break
            if forced_iters is None and it >= max_iter:
                break
            a = apply_filter(coef, analysis(t, L))
            sn = synthesis(a, L)
            ss = np.sum(sn * sn)
            c = np.sqrt(np.sum((sn - s) ** 2) / ss) if ss > 0 else 0.0
            s = sn
            t = s + alpha * np.einsum("ij...,j...->i...", ninv, np.where(obs, d, 0.0) - s)
            cauchy.append(c)
            it += 1
            nk += 1
            if forced_iters is None and c < eps[k]:
                break
        iters_per_level.append(nk)
    return {"s": s, "alm": a, "iters": it, "iters_per_level": np.array(iters_per_level),
            "cauchy": np.array(cauchy), "alpha": alpha}


# ------------------------------------------ constrained realisations (Eq. 19)
# s_CR = W(d - dhat) + shat with shat a signal draw from the prior and
# dhat = shat + nhat, nhat a noise draw whose covariance is the inverse of the
# precision the solve uses (Eq. 18).  The random numbers are inputs: unit
# white-noise maps z_s (signal) and z_n (noise), [3, N, N] each.


def draw_signal(z_s, S, L):
    """Fourier coefficients [3, N, N] with <a a^H> = L^2 C per mode and the
    Hermitian symmetry of real fields: the per-mode Cholesky factor of the
    TE block (and sqrt C^BB) applied to (L / N) FFT(z_s)."""
    N = z_s.shape[-1]
    tt, ee, bb, te = S
    h = (L / N) * np.fft.fft2(z_s, axes=(-2, -1))
    l11 = np.sqrt(np.maximum(tt, 0.0))
    l21 = np.where(l11 > 0, te / np.where(l11 > 0, l11, 1.0), 0.0)
    l22 = np.sqrt(np.maximum(ee - l21 ** 2, 0.0))
    _, _, _, keep = geometry(N, L)
    return np.stack([l11 * h[0], l21 * h[0] + l22 * h[1], np.sqrt(np.maximum(bb, 0.0)) * h[2]]) * keep


def draw_noise(z_n, sigma, mask_t, mask_p, rho=None):
    """Noise draw on observed components, 0 on masked ones.  Diagonal model:
    sigma z.  Correlated model: Sigma x with x = L z (C = L L^T) on a fully
    observed pixel; where some components are masked (Sigma^-1 = 0 there) the
    observed block of the precision inverts to the covariance of x_o given
    x_m = 0, drawn as x_o - C_om C_mm^-1 x_m."""
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    if rho is None:
        return np.where(obs, sigma * z_n, 0.0)
    r01, r02, r12 = rho
    l11 = np.sqrt(1.0 - r01 ** 2)
    l21 = (r12 - r02 * r01) / l11
    l22 = np.sqrt(1.0 - r02 ** 2 - l21 ** 2)
    x0 = z_n[0]
    x1 = r01 * z_n[0] + l11 * z_n[1]
    x2 = r02 * z_n[0] + l21 * z_n[1] + l22 * z_n[2]
    ot, op = obs[0], obs[1]
    t_only = ot & ~op  # Q, U masked: condition I on x_Q = x_U = 0
    p_only = op & ~ot  # I masked: condition Q, U on x_I = 0
    y1 = (x1 - r12 * x2) / (1.0 - r12 ** 2)
    y2 = (x2 - r12 * x1) / (1.0 - r12 ** 2)
    x0 = np.where(t_only, x0 - (r01 * y1 + r02 * y2), x0)
    x1 = np.where(p_only, x1 - r01 * z_n[0], x1)
    x2 = np.where(p_only, x2 - r02 * z_n[0], x2)
    return np.where(obs, sigma * np.stack([x0, x1, x2]), 0.0)


def constrained_realization(d, z_s, z_n, sigma, mask_t, mask_p, S, L, lambdas, rho=None, **solve_args):
    """s_CR = W(d - dhat) + shat (Eq. 19) with W the dual messenger solve
    (dm_solve, or dm_solve_cov when rho is given)."""
    a_hat = draw_signal(z_s, S, L)
    s_hat = synthesis(a_hat, L)
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    d_hat = np.where(obs, s_hat + draw_noise(z_n, sigma, mask_t, mask_p, rho), 0.0)
    if rho is None:
        r = dm_solve(np.asarray(d) - d_hat, sigma, mask_t, mask_p, S, L, lambdas, **solve_args)
    else:
        r = dm_solve_cov(np.asarray(d) - d_hat, sigma, rho, mask_t, mask_p, S, L, lambdas, **solve_args)
    r["s_cr"] = r["s"] + s_hat
    r["alm_cr"] = r["alm"] + a_hat
    r["s_hat"], r["d_hat"], r["a_hat"] = s_hat, d_hat, a_hat
    return r


# ---------------------------------------------------------------- Appendix A
# Jacobi refinement s^{n+1} = s^n + W~(d - W^+ s^n).  W~ is the dual messenger
# operator run with the per-level iteration counts of the usual solve, kept
# fixed so that W~ is one linear operator.  Data enter the messenger update
# t = (Nbar^-1 + T^-1)^-1 (T^-1 s + Nbar^-1 d) only through its data term,
# h = w d on observed components.  For the correction the data are
# W^+ s = N (S^-1 + N^-1) s, whose data term is T Z = alpha (S^+ + N^-1) s with
# S^+ the pixel-space pseudo-inverse of the signal covariance: w s on observed
# components plus alpha S^+ s on every pixel, masked ones included (the limit
# N -> infinity of w W^+ s there).  This is Appendix A's rewriting of the
# messenger equation in terms of Z, free of N on masked pixels.  Every run of
# W~ starts from t_0 = h, the update applied to s = 0, so that W~ sees h only
# through F^dagger h.  The Wiener-filter equation holds on the directions
# S spans; along its null directions (the T monopole and E, B at l = 0 on the
# patch) the data carry no equation, yet W~ at levels with mu > 0 would pass
# them.  So the correction's data term is projected onto the range of S in
# harmonic space before W~ runs; the exact Wiener filter is then a fixed point
# of the refinement whatever the counts.


def dm_frozen(h, w, S, L, lambdas, counts, th):
    """W~ applied to a messenger data term h [3, N, N]: t_0 = h, then for each
    level k, counts[k] times a = filter_k(F^dagger t), s = F a,
    t = (1 - w) s + h.  Returns (s, a)."""
    t = np.array(h, dtype=np.float64)
    s = np.zeros_like(t)
    a = np.zeros(t.shape, np.complex128)
    for lam, n in zip(lambdas, counts):
        coef = filter_coefs(S, (lam - 1.0) * th, th)
        for _ in range(int(n)):
            a = apply_filter(coef, analysis(t, L))
            s = synthesis(a, L)
            t = (1.0 - w) * s + h
    return s, a


def jacobi_data_term(s, w, alpha, S, L):
    """T Z of Appendix A for the signal map s: w s + alpha S^+ s, where
    S^+ s = Omega_p L^2 F S_a^+ F^dagger s and S_a = L^2 C per mode."""
    N = s.shape[-1]
    sinv = _block_pow(S * L ** 2, -1.0)
    return w * s + alpha * (L / N) ** 2 * L ** 2 * synthesis(apply_filter(sinv, analysis(s, L)), L)


def range_projected(x, S, L):
    """x minus the synthesis of the part of F^dagger x along the null
    directions of each mode's signal block, so that F^dagger of the result is
    the projection of F^dagger x onto the range of S."""
    g = analysis(x, L)
    keep = apply_filter(_block_pow(S, 0.0), g)
    return x - synthesis(g - keep, L)


def jacobi_refine(d, sigma, mask_t, mask_p, S, L, lambdas, eps=None, forced_iters=None, n_refine=1,
                  max_iter=100000):
    """The usual solve (recording its per-level counts), then n_refine steps
    s <- s + W~(P(w d - T Z(s))) with W~ run at those counts (Appendix A) and
    P the projection onto the range of S.
    Returns the final s, alm, the counts and the map after each step."""
    r = dm_solve(d, sigma, mask_t, mask_p, S, L, lambdas, eps=eps, forced_iters=forced_iters, max_iter=max_iter)
    N = d.shape[-1]
    alpha, w = weights(sigma, mask_t, mask_p)
    th = alpha * (L / N) ** 2
    counts = r["iters_per_level"]
    hd = w * np.asarray(d, dtype=np.float64)
    s = r["s"]
    steps = [s]
    for _ in range(n_refine):
        x = range_projected(hd - jacobi_data_term(s, w, alpha, S, L), S, L)
        c, _ = dm_frozen(x, w, S, L, lambdas, counts, th)
        s = s + c
        steps.append(s)
    return {"s": s, "alm": analysis(s, L), "counts": counts, "steps": steps, "solve": r}
