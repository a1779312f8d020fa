"""Pins for the oracle's per-l filter, messenger update, level loop, chi^2 and
constrained realisations (Sections 2, 2.1, 2.2; Algorithm 1; Eqs. 2, 3, 8, 9,
10, 18, 19)."""
import numpy as np
import pytest

import workloads as W
from tests.harmonics_ref import alm_to_params, dense_synthesis, params_to_alm, real_param_index


def _sblock(cl, l):
    tt, ee, bb, te = cl[:, l]
    return np.array([[tt, te, 0.0], [te, ee, 0.0], [0.0, 0.0, bb]])


def test_filter_is_truncated_wiener_gain(orc):
    """F_l = (Sbar + U)(Sbar + xi)^{-1} with Sbar = max(S_e - mu, 0) on the
    eigenvalues of the 3x3 block of Eq. 10, checked with numpy's eigh."""
    lmax = 60
    cl = W.cl_analytic(lmax)
    th = 3e-5
    for mu in [0.0, 10 * th, 1e-3, 0.5]:
        coef = orc.filter_coefs(lmax, cl, mu, th)
        for l in range(lmax + 1):
            e, v = np.linalg.eigh(_sblock(cl, l))
            e = np.maximum(e, 0.0)
            sp = np.maximum(e, mu)
            F = (v * (sp / (sp + th))) @ v.T
            got = np.array([[coef[l, 0], coef[l, 1], 0], [coef[l, 1], coef[l, 2], 0], [0, 0, coef[l, 3]]])
            assert np.max(np.abs(got - F)) < 1e-13


def test_homogeneous_full_sky_first_step_is_closed_form(orc):
    """Unmasked homogeneous noise N = alpha: w = 1 and t = d, so the first
    iteration at lambda = 1 is a = S (S + alpha Omega)^{-1} A d per l (the
    harmonic Wiener filter, Eq. 2), computed here with numpy.linalg.solve."""
    nside, lmax = 8, 16
    cl = W.cl_analytic(lmax, lscale=8.0)
    npix = 12 * nside * nside
    sigma = np.full((3, npix), 0.03)
    d = W.random_maps(nside, 1, 21)[0]
    r = orc.dm_solve(nside, lmax, cl, sigma, None, d, [1.0], forced_iters=[1])
    Ad = orc.map2alm(nside, lmax, d)
    th = 0.03 ** 2 * 4 * np.pi / npix
    ref = np.zeros_like(Ad)
    for m in range(lmax + 1):
        for l in range(m, lmax + 1):
            ix = orc.almidx(lmax, l, m)
            S = _sblock(cl, l)
            ref[:, ix] = S @ np.linalg.solve(S + th * np.eye(3), Ad[:, ix])
    assert np.max(np.abs(r["alm"] - ref)) < 1e-13 * np.max(np.abs(ref))


def test_messenger_update_corner_cases(orc):
    """t = (Nbar^{-1} + T^{-1})^{-1}(T^{-1} s + Nbar^{-1} d) (Eq. 9) with
    T = alpha: w = alpha/N; N = alpha gives t = d (the Nbar = 0 corner case of
    Section 2.1), a masked pixel (N^{-1} = 0) gives t = s."""
    rng = np.random.default_rng(1)
    N = rng.uniform(1.0, 5.0, 50)
    alpha = N.min()
    N[3] = alpha
    w = alpha / N
    w[7] = 0.0
    d, s = rng.standard_normal(50), rng.standard_normal(50)
    t = orc.messenger_update(w, d, s)
    for i in range(50):
        if i == 7:
            assert t[i] == s[i]
        elif N[i] == alpha:
            assert t[i] == pytest.approx(d[i], abs=1e-15)
        else:
            nb = N[i] - alpha
            ref = (s[i] / alpha + d[i] / nb) / (1 / nb + 1 / alpha)
            assert t[i] == pytest.approx(ref, rel=1e-12)


def _dense_problem(nside, lmax, seed, mu=0.0, th=None):
    """Dense real-parameter form of the Wiener filter at nside 4."""
    z, phi = W.pixel_centers(nside)
    cl = W.cl_analytic(lmax, lscale=6.0)
    params_all = real_param_index(lmax)
    rng = np.random.default_rng(seed)
    npix = z.size
    sig_t = 0.02 * (0.7 + 0.6 * rng.random(npix))
    sigma = np.stack([sig_t, 1.4 * sig_t, 1.4 * sig_t])
    mask = (np.abs(z) > 0.25).astype(np.uint8)
    return cl, params_all, sigma, mask, z, phi


def _prior_precision(cl, params, mu):
    """Block precision of the real parameters under S' = V max(S_e, mu) V^T,
    inverted on the parameters that exist (no E/B below l = 2)."""
    n = len(params)
    P = np.zeros((n, n))
    idx = {p: j for j, p in enumerate(params)}
    done = set()
    for (f, l, m, part) in params:
        if (l, m, part) in done:
            continue
        done.add((l, m, part))
        e, v = np.linalg.eigh(_sblock(cl, l))
        Sp = (v * np.maximum(np.maximum(e, 0.0), mu)) @ v.T
        ids = [(k, idx[(k, l, m, part)]) for k in range(3) if (k, l, m, part) in idx]
        sub = np.array([[Sp[a, b] for b, _ in ids] for a, _ in ids])
        Sinv = np.linalg.inv(sub)
        fac = 1.0 if m == 0 else 2.0
        for i1, (_, j1) in enumerate(ids):
            for i2, (_, j2) in enumerate(ids):
                P[j1, j2] = fac * Sinv[i1, i2]
    return P


@pytest.mark.parametrize("level_lambda,lmax", [(1.0, 8), (40.0, 8), (1.0, 11), (40.0, 11)])
def test_dm_fixed_point_is_dense_wiener_filter(orc, level_lambda, lmax):
    """At a fixed level the dual messenger iteration converges to the Wiener
    filter with signal covariance Sbar + U (Eq. 8 at mu = 0 is Eq. 2):
    (S'^{-1} + Y^T N^{-1} Y) x = Y^T N^{-1} d, solved densely at nside 4 with
    harmonics from scipy and Goldberg et al. (1967).  At lmax 11 = 3 nside - 1
    the quadrature is poor (AY spans 0.53 to 1.48) and the level contracts at
    0.996 an iteration, yet the fixed point is still the exact Wiener filter."""
    nside = 4
    cl, params_all, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    npix = z.size
    alpha = np.min((sigma ** 2)[:, mask > 0])
    th = alpha * 4 * np.pi / npix
    mu = (level_lambda - 1.0) * th
    # parameters with zero prior variance are fixed at zero (T l = 0 at mu = 0)
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0 and mu == 0.0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Ninv = (mask[None, :] / sigma ** 2).reshape(-1)
    d = W.random_maps(nside, 1, 8)[0] * 0.05
    d = d * mask[None, :]
    P = _prior_precision(cl, params, mu)
    Amat = P + Y.T @ (Ninv[:, None] * Y)
    x = np.linalg.solve(Amat, Y.T @ (Ninv * d.reshape(-1)))
    r = orc.dm_solve(nside, lmax, cl, sigma, mask, d, [level_lambda], eps=[1e-15], max_iter=60000)
    xo = alm_to_params(r["alm"], params, lmax)
    assert np.linalg.norm(xo - x) / np.linalg.norm(x) < 1e-9
    s_ref = (Y @ x).reshape(3, -1)
    assert np.linalg.norm(r["s"] - s_ref) / np.linalg.norm(s_ref) < 1e-9


def test_linearity_of_fixed_schedule(orc):
    wl = W.make_workload("nside16", [0], nside=8, lmax=16)
    d1 = W.random_maps(8, 1, 1)[0] * wl.mask
    d2 = W.random_maps(8, 1, 2)[0] * wl.mask
    lam = W.lambda_schedule(100.0, 3)
    f = lambda d: orc.dm_solve(8, 16, wl.cl, wl.sigma, wl.mask, d, lam, forced_iters=[4, 4, 4])["s"]
    a, b, c = f(d1), f(d2), f(d1 + 2 * d2)
    assert np.linalg.norm(c - a - 2 * b) / np.linalg.norm(c) < 1e-12


def test_level_loop_accounting(orc):
    wl = W.make_workload("nside16", [0], nside=8, lmax=16)
    s = orc.alm2map(8, 16, wl.alm_true[0])
    d = wl.data([s])[0]
    lam = W.lambda_schedule(1000.0, 5)
    eps = W.eps_schedule(5, 1e-3, 1e-5)
    r = orc.dm_solve(8, 16, wl.cl, wl.sigma, wl.mask, d, lam, eps=eps)
    ipl = r["iters_per_level"]
    assert ipl.sum() == r["iters"] and np.all(ipl >= 1)
    ends = np.cumsum(ipl) - 1
    assert np.all(r["cauchy"][ends] < eps)
    starts = np.concatenate([[0], ends[:-1] + 1])
    for st, en, e in zip(starts, ends, eps):
        assert np.all(r["cauchy"][st:en] >= e)


@pytest.mark.slow
def test_chi2_matches_degrees_of_freedom(orc):
    """At the Wiener filter chi^2_min = d^T (S + N)^{-1} d, whose expectation is
    the number of observed pixel-components (Section 3.4)."""
    nside, lmax = 8, 16
    wl = W.make_workload("nside16", [4], nside=nside, lmax=lmax)
    s = orc.alm2map(nside, lmax, wl.alm_true[0])
    d = wl.data([s])[0]
    lam = W.lambda_schedule(1000.0, 6)
    r = orc.dm_solve(nside, lmax, wl.cl, wl.sigma, wl.mask, d, lam, eps=W.eps_schedule(6, 1e-5, 1e-9))
    chi = orc.chi2(nside, lmax, wl.cl, wl.sigma, wl.mask, d, r["s"], r["alm"])
    ndof = 3 * int(wl.mask.sum())
    assert abs(chi - ndof) < 5 * np.sqrt(2 * ndof)


# --------------------------------------------------------------------------
# Constrained realisations (Section 2.2)
# --------------------------------------------------------------------------

def test_philox_known_answers(orc):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        assert orc.philox4x32_10(v[:4], v[4:6]) == v[6:]


def test_gaussian_draws_are_standard(orc):
    z = np.array([orc.gauss_pair(12345, i, 0, 0) for i in range(20000)]).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 0.15


def test_signal_draw_covariance(orc):
    """ahat ~ S: empirical per-l T/E/B covariances over draws match Eq. 10."""
    lmax = 6
    cl = W.cl_analytic(lmax, lscale=4.0)
    K = 3000
    acc = np.zeros((lmax + 1, 3, 3))
    cnt = np.zeros(lmax + 1)
    for seed in range(K):
        a = orc.draw_signal_alm(lmax, cl, seed)
        for m in range(lmax + 1):
            for l in range(m, lmax + 1):
                v = a[:, orc.almidx(lmax, l, m)]
                # m = 0 real at full variance, m > 0 re and im at half: E|a|^2 = C
                acc[l] += np.real(np.outer(v, np.conj(v)))
                cnt[l] += 1
    for l in range(2, lmax + 1):
        emp = acc[l] / cnt[l]
        S = _sblock(cl, l)
        n_eff = cnt[l]
        for i in range(3):
            assert abs(emp[i, i] - S[i, i]) < 6 * S[i, i] * np.sqrt(2.0 / n_eff)
        assert abs(emp[0, 1] - S[0, 1]) < 6 * np.sqrt(S[0, 0] * S[1, 1] / n_eff)


@pytest.mark.slow
def test_fluctuation_covariance_is_posterior(orc):
    """f = shat - W dhat has <f f^T> = (S^{-1} + N^{-1})^{-1} (Eq. 18): the mean
    Mahalanobis norm of f under that covariance equals the dimension."""
    nside, lmax = 4, 8
    cl, params_all, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Ninv = (mask[None, :] / sigma ** 2).reshape(-1)
    P = _prior_precision(cl, params, 0.0)
    H = P + Y.T @ (Ninv[:, None] * Y)
    Wmat = np.linalg.solve(H, Y.T * Ninv[None, :])
    K = 400
    q = []
    for seed in range(K):
        ahat, shat, dhat = orc.cr_inputs(nside, lmax, cl, sigma, mask, 1000 + seed)
        f = alm_to_params(ahat, params, lmax) - Wmat @ dhat.reshape(-1)
        q.append(f @ H @ f)
    n = len(params)
    assert abs(np.mean(q) - n) < 5 * np.sqrt(2.0 * n / K)


def test_cr_inputs_consistent(orc):
    nside, lmax = 4, 8
    cl = W.cl_analytic(lmax)
    wl = W.make_workload("nside16", [0], nside=nside, lmax=lmax)
    ahat, shat, dhat = orc.cr_inputs(nside, lmax, cl, wl.sigma, wl.mask, 77)
    assert np.allclose(shat, orc.alm2map(nside, lmax, ahat), atol=1e-14)
    n = orc.draw_noise(nside, wl.sigma, wl.mask, 77)
    assert np.allclose(dhat, (shat + n) * wl.mask, atol=1e-14)
    assert np.all(dhat[:, wl.mask == 0] == 0)


def test_filter_is_scalar_where_spectra_underflow(orc):
    """Where both eigenvalues of the TE block lie far below mu the filter of
    Eq. 10 is f 1 exactly (any rotation R), even where the analytic spectra
    (around 1e-160 near l = 750) have subnormal squares and products."""
    lmax = 4096
    cl = W.cl_analytic(lmax)
    th, mu = 1.06e-9, 999.0 * 1.06e-9
    coef = orc.filter_coefs(lmax, cl, mu, th)
    f = mu / (mu + th)
    for l in [700, 740, 750, 753, 756, 760, 800, 1100, 4096]:
        assert coef[l, 0] == pytest.approx(f, rel=1e-14)
        assert coef[l, 2] == pytest.approx(f, rel=1e-14)
        assert abs(coef[l, 1]) <= 1e-14 * f


@pytest.mark.slow
def test_cr_power_spectrum_is_unbiased(orc):
    """Constrained realisations through the oracle's own converged solve
    (Eq. 19), over true signals drawn from the prior and their data: the mean
    power of a_CR per field pair, pooled over l, equals the input spectrum
    (Section 3.2: CRs restore the power the Wiener filter suppresses)."""
    nside, lmax = 4, 8
    cl, _, sigma, mask, _, _ = _dense_problem(nside, lmax, 3)
    rng = np.random.default_rng(50)
    K = 150
    pw = np.zeros((4, lmax + 1))  # TT, EE, BB, TE
    for k in range(K):
        a = W.draw_alm(lmax, cl, rng)
        d = (orc.alm2map(nside, lmax, a) + sigma * rng.standard_normal(sigma.shape)) * mask[None, :]
        r = orc.constrained_realization(nside, lmax, cl, sigma, mask, d, 7000 + k, [1.0], eps=[1e-10],
                                        max_iter=20000)
        acr = r["alm_cr"]
        for m in range(lmax + 1):
            fac = 1.0 if m == 0 else 2.0
            for l in range(m, lmax + 1):
                ix = orc.almidx(lmax, l, m)
                t, e, b = acr[:, ix]
                pw[0, l] += fac * abs(t) ** 2
                pw[1, l] += fac * abs(e) ** 2
                pw[2, l] += fac * abs(b) ** 2
                pw[3, l] += fac * (t * np.conj(e)).real
    ells = np.arange(lmax + 1)
    pw /= K * (2 * ells + 1)[None, :]
    for row, lmin in [(0, 1), (1, 2), (2, 2)]:
        sel = slice(lmin, lmax + 1)
        ratio = pw[row, sel] / cl[row, sel]
        se = np.sqrt(np.sum(2.0 / (K * (2 * ells[sel] + 1)))) / len(ratio)  # standard error of the mean ratio
        assert abs(np.mean(ratio) - 1.0) < 5 * se
    # TE: the cross power against C^TE, as z-scores pooled over l
    sel = slice(2, lmax + 1)
    ref = cl[3, sel]
    sd = np.sqrt((cl[0, sel] * cl[1, sel] + ref ** 2) / (K * (2 * ells[sel] + 1)))
    assert abs(np.mean((pw[3, sel] - ref) / sd)) < 5.0 / np.sqrt(len(ref))


def test_chi2_minimum_is_the_dense_identity(orc):
    """At the Wiener filter x* = H^-1 b (H = P + Y^T N^-1 Y, b = Y^T N^-1 d),
    chi^2 of Eq. 3 takes its minimum d^T N^-1 d - b^T H^-1 b: an exact check of
    both terms of orc_chi2 at nside 4; away from x* it is larger."""
    nside, lmax = 4, 8
    cl, params_all, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Ninv = (mask[None, :] / sigma ** 2).reshape(-1)
    d = W.random_maps(nside, 1, 72)[0] * 0.05 * mask[None, :]
    H = _prior_precision(cl, params, 0.0) + Y.T @ (Ninv[:, None] * Y)
    b = Y.T @ (Ninv * d.reshape(-1))
    x = np.linalg.solve(H, b)
    ref = d.reshape(-1) @ (Ninv * d.reshape(-1)) - b @ x
    a = params_to_alm(x, params, lmax)
    got = orc.chi2(nside, lmax, cl, sigma, mask, d, orc.alm2map(nside, lmax, a), a)
    assert got == pytest.approx(ref, rel=1e-10)
    a2 = params_to_alm(x + 1e-2 * np.abs(x).max() * np.random.default_rng(73).standard_normal(len(x)), params, lmax)
    assert orc.chi2(nside, lmax, cl, sigma, mask, d, orc.alm2map(nside, lmax, a2), a2) > got
