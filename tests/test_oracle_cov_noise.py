"""Pins of the oracle's correlated-noise model (3x3 noise covariance per
pixel, distinct temperature and polarisation masks; Section 2.1 and
Appendix B).

- N^{-1} against numpy's inverse of Sigma C Sigma, with masked components
  (Sigma^{-1} = 0) zeroed;
- alpha against numpy's eigenvalues of N;
- the update t = s + alpha N^{-1} (d - s) against the literal messenger
  equation of Appendix B, t = (Nbar^{-1} + T^{-1})^{-1}(T^{-1} s + Nbar^{-1} d)
  with Nbar^{-1} = Sigma^{-1} P^T (Delta - alpha P Sigma^{-2} P^T)^{-1} P Sigma^{-1};
- the corner case Nbar = 0 of Section 2.1 (t = d along that direction);
- masked components: t = s there, and their data never enter;
- uncorrelated noise with one mask: the same solve as the diagonal oracle;
- the converged loop against a dense Wiener-filter solve with the
  block-diagonal N^{-1} at nside 4;
- constrained-realisation noise draws (Eq. 18): uncorrelated with one mask
  they are the diagonal draws; their sample covariance is the inverse of the
  observed block of N^{-1} (Sigma C Sigma on fully observed pixels, the
  conditional covariance on partially masked ones); the CR inputs are the
  signal draw plus that noise on observed components; the fluctuation
  shat - W dhat has the posterior covariance at nside 4."""
import numpy as np
import pytest

import workloads as W
from tests.harmonics_ref import alm_to_params, dense_synthesis, params_to_alm
from tests.test_oracle_dm import _dense_problem, _prior_precision


def _corr(rho):
    """[npix, 3, 3] correlation matrices from [3, npix] (rho_IQ, rho_IU, rho_QU)."""
    npix = rho.shape[1]
    C = np.empty((npix, 3, 3))
    C[:, 0, 0] = C[:, 1, 1] = C[:, 2, 2] = 1.0
    C[:, 0, 1] = C[:, 1, 0] = rho[0]
    C[:, 0, 2] = C[:, 2, 0] = rho[1]
    C[:, 1, 2] = C[:, 2, 1] = rho[2]
    return C


def _random_model(npix, seed, masked=True):
    rng = np.random.default_rng(seed)
    sigma = rng.uniform(0.5, 2.0, (3, npix))
    rho = rng.uniform(-0.3, 0.3, (3, npix))
    mt = (rng.random(npix) > 0.3).astype(np.uint8) if masked else np.ones(npix, np.uint8)
    mp = (rng.random(npix) > 0.3).astype(np.uint8) if masked else np.ones(npix, np.uint8)
    return sigma, rho, mt, mp


def test_ninv_is_masked_inverse_of_sigma_c_sigma(orc):
    sigma, rho, mt, mp = _random_model(200, 1)
    ninv = orc.cov_ninv(sigma, rho, mt, mp)
    C = _corr(rho)
    for p in range(200):
        si = np.array([mt[p] / sigma[0, p], mp[p] / sigma[1, p], mp[p] / sigma[2, p]])
        ref = si[:, None] * np.linalg.inv(C[p]) * si[None, :]
        assert np.allclose(ninv[p], ref, rtol=1e-13, atol=1e-15)
        if mt[p] and mp[p]:
            N = np.diag(sigma[:, p]) @ C[p] @ np.diag(sigma[:, p])
            assert np.allclose(ninv[p], np.linalg.inv(N), rtol=1e-12)


def test_alpha_is_smallest_eigenvalue_of_n(orc):
    sigma, rho, mt, mp = _random_model(300, 2, masked=False)
    ninv = orc.cov_ninv(sigma, rho, mt, mp)
    C = _corr(rho)
    lam = min(np.linalg.eigvalsh(np.diag(sigma[:, p]) @ C[p] @ np.diag(sigma[:, p])).min() for p in range(300))
    assert orc.cov_alpha(ninv) == pytest.approx(lam, rel=1e-13)
    # with masks: the smallest eigenvalue over the observed components
    sigma, rho, mt, mp = _random_model(300, 3)
    ninv = orc.cov_ninv(sigma, rho, mt, mp)
    ref = min(1.0 / np.linalg.eigvalsh(ninv[p]).max() for p in range(300) if np.abs(ninv[p]).max() > 0)
    assert orc.cov_alpha(ninv) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("masked", [False, True])
def test_update_equals_appendix_b_messenger_equation(orc, masked):
    """The literal Appendix B formula with C = P^T Delta P (numpy eigh) and
    T = alpha 1, at pixels where Nbar is invertible."""
    npix = 120
    sigma, rho, mt, mp = _random_model(npix, 4, masked)
    ninv = orc.cov_ninv(sigma, rho, mt, mp)
    alpha = orc.cov_alpha(ninv)
    rng = np.random.default_rng(5)
    d, s = rng.standard_normal((3, npix)), rng.standard_normal((3, npix))
    t = orc.messenger_update_cov(alpha, ninv, d, s)
    C = _corr(rho)
    checked = 0
    for p in range(npix):
        si = np.diag([mt[p] / sigma[0, p], mp[p] / sigma[1, p], mp[p] / sigma[2, p]])
        ev, V = np.linalg.eigh(C[p])
        P, Delta = V.T, np.diag(ev)
        M = Delta - alpha * P @ si @ si @ P.T
        if np.linalg.eigvalsh(M).min() < 1e-6:
            continue  # the corner case, checked below
        nbinv = si @ P.T @ np.linalg.inv(M) @ P @ si
        lhs = nbinv + np.eye(3) / alpha
        ref = np.linalg.solve(lhs, s[:, p] / alpha + nbinv @ d[:, p])
        assert np.allclose(t[:, p], ref, rtol=1e-11, atol=1e-12)
        checked += 1
    assert checked >= npix - 2


def test_corner_case_keeps_the_data(orc):
    """At the pixel where alpha is attained (Nbar = 0 along one direction v of
    Section 2.1) the update keeps the data there: v . t = v . d."""
    npix = 80
    sigma, rho, mt, mp = _random_model(npix, 6, masked=False)
    ninv = orc.cov_ninv(sigma, rho, mt, mp)
    alpha = orc.cov_alpha(ninv)
    C = _corr(rho)
    N = [np.diag(sigma[:, p]) @ C[p] @ np.diag(sigma[:, p]) for p in range(npix)]
    p0 = int(np.argmin([np.linalg.eigvalsh(n).min() for n in N]))
    ev, V = np.linalg.eigh(N[p0])
    v = V[:, 0]
    assert ev[0] == pytest.approx(alpha, rel=1e-13)
    rng = np.random.default_rng(7)
    d, s = rng.standard_normal((3, npix)), rng.standard_normal((3, npix))
    t = orc.messenger_update_cov(alpha, ninv, d, s)
    assert v @ t[:, p0] == pytest.approx(v @ d[:, p0], abs=1e-13)


def test_masked_components_keep_s_and_ignore_d(orc):
    npix = 150
    sigma, rho, mt, mp = _random_model(npix, 8)
    ninv = orc.cov_ninv(sigma, rho, mt, mp)
    alpha = orc.cov_alpha(ninv)
    rng = np.random.default_rng(9)
    d, s = rng.standard_normal((3, npix)), rng.standard_normal((3, npix))
    t = orc.messenger_update_cov(alpha, ninv, d, s)
    obs = np.stack([mt, mp, mp]).astype(bool)
    assert np.array_equal(t[~obs], s[~obs])
    d2 = d.copy()
    d2[~obs] = 1e6 * rng.standard_normal((~obs).sum())
    assert np.array_equal(orc.messenger_update_cov(alpha, ninv, d2, s), t)


def test_uncorrelated_common_mask_is_the_diagonal_solve(orc):
    """rho = 0 and one mask for I, Q and U: the correlated-noise solve is the
    diagonal one (alpha = min sigma^2, W = alpha / sigma^2) up to rounding."""
    wl = W.make_workload("nside16", [11], nside=8, lmax=16)
    d = wl.data([orc.alm2map(8, 16, wl.alm_true[0])])[0]
    rho = np.zeros_like(wl.sigma)
    lam = W.lambda_schedule(1000.0, 4)
    ref = orc.dm_solve(8, 16, wl.cl, wl.sigma, wl.mask, d, lam, forced_iters=[3, 3, 3, 3])
    got = orc.dm_solve_cov(8, 16, wl.cl, wl.sigma, rho, wl.mask, wl.mask, d, lam, forced_iters=[3, 3, 3, 3])
    assert got["iters"] == 12
    assert np.linalg.norm(got["s"] - ref["s"]) / np.linalg.norm(ref["s"]) < 1e-13
    assert np.linalg.norm(got["alm"] - ref["alm"]) / np.linalg.norm(ref["alm"]) < 1e-13


@pytest.mark.parametrize("level_lambda", [1.0, 40.0])
def test_cov_fixed_point_is_dense_wiener_filter(orc, level_lambda):
    """At a fixed level the loop converges to (S'^{-1} + Y^T N^{-1} Y) x =
    Y^T N^{-1} d with the block-diagonal N^{-1} (I, Q, U of a pixel coupled)
    and distinct temperature and polarisation masks, solved densely at
    nside 4."""
    nside, lmax = 4, 8
    cl, params_all, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    npix = z.size
    rng = np.random.default_rng(12)
    rho = rng.uniform(-0.3, 0.3, (3, npix))
    mask_t = (np.abs(z) > 0.25).astype(np.uint8)
    mask_p = (np.abs(z - 0.1) > 0.2).astype(np.uint8)
    ninv = orc.cov_ninv(sigma, rho, mask_t, mask_p)
    alpha = orc.cov_alpha(ninv)
    th = alpha * 4 * np.pi / npix
    mu = (level_lambda - 1.0) * th
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0 and mu == 0.0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Nd = np.zeros((3 * npix, 3 * npix))
    for p in range(npix):
        for i in range(3):
            for j in range(3):
                Nd[i * npix + p, j * npix + p] = ninv[p, i, j]
    obs = np.stack([mask_t, mask_p, mask_p])
    d = W.random_maps(nside, 1, 8)[0] * 0.05 * obs
    P = _prior_precision(cl, params, mu)
    x = np.linalg.solve(P + Y.T @ Nd @ Y, Y.T @ Nd @ d.reshape(-1))
    r = orc.dm_solve_cov(nside, lmax, cl, sigma, rho, mask_t, mask_p, d, [level_lambda], eps=[1e-15],
                         max_iter=60000)
    xo = alm_to_params(r["alm"], params, lmax)
    assert np.linalg.norm(xo - x) / np.linalg.norm(x) < 1e-9
    s_ref = (Y @ x).reshape(3, -1)
    assert np.linalg.norm(r["s"] - s_ref) / np.linalg.norm(s_ref) < 1e-9


def test_correlated_noise_draws_have_the_model_covariance():
    """draw_noise_cov: the sample covariance of many draws of one pixel model
    is Sigma C Sigma (to the sampling error), and masked components are 0."""
    n = 200000
    sigma = np.tile(np.array([[1.0], [1.5], [0.7]]), (1, n))
    rho = np.tile(np.array([[0.25], [-0.2], [0.1]]), (1, n))
    ones = np.ones(n, np.uint8)
    x = W.draw_noise_cov(sigma, rho, ones, ones, np.random.default_rng(13))
    C = _corr(rho[:, :1])[0]
    ref = np.diag(sigma[:, 0]) @ C @ np.diag(sigma[:, 0])
    assert np.allclose(np.cov(x), ref, atol=0.02)
    mt = np.zeros(n, np.uint8)
    y = W.draw_noise_cov(sigma, rho, mt, ones, np.random.default_rng(14))
    assert not y[0].any() and y[1].any()


def test_masked_data_never_enter_the_solve(orc):
    """Arbitrary values on masked components of d change nothing, from the
    first iteration on (t_0 is d on observed components only)."""
    wl = W.make_cov_workload([15], 8, 16)
    d = wl.data([orc.alm2map(8, 16, wl.alm_true[0])])[0]
    obs = np.stack([wl.mask, wl.mask_p, wl.mask_p]).astype(bool)
    d2 = d.copy()
    d2[~obs] = np.random.default_rng(16).standard_normal((~obs).sum())
    lam = W.lambda_schedule(1000.0, 2)
    a = orc.dm_solve_cov(8, 16, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, d, lam, forced_iters=[2, 2])
    b = orc.dm_solve_cov(8, 16, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, d2, lam, forced_iters=[2, 2])
    assert np.array_equal(a["s"], b["s"]) and np.array_equal(a["alm"], b["alm"])


def test_cov_cr_draw_reduces_to_the_diagonal_draw(orc):
    """rho = 0 and one mask: the correlated CR noise draw is the diagonal one,
    value for value (same Philox normals, L = 1)."""
    wl = W.make_workload("nside16", [0], nside=16, lmax=32)
    rho = np.zeros_like(wl.sigma)
    a = orc.draw_noise_cov(16, wl.sigma, rho, wl.mask, wl.mask, 91)
    b = orc.draw_noise(16, wl.sigma, wl.mask, 91)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["observed", "t_masked", "p_masked"])
def test_cov_cr_draw_covariance_is_inverse_observed_precision(orc, case):
    """Over 786432 pixels of one noise model the sample covariance of the
    observed components is ((Sigma^{-1} C^{-1} Sigma^{-1})_oo)^{-1}, from
    numpy's inverses; it differs from the marginal Sigma_o C_oo Sigma_o on
    partially masked pixels by far more than the sampling error."""
    nside = 256
    n = 12 * nside * nside
    sd = np.array([1.0, 1.5, 0.7])
    r = np.array([0.5, -0.4, 0.3])
    sigma = np.tile(sd[:, None], (1, n))
    rho = np.tile(r[:, None], (1, n))
    mt = np.full(n, case != "t_masked", np.uint8)
    mp = np.full(n, case != "p_masked", np.uint8)
    x = orc.draw_noise_cov(nside, sigma, rho, mt, mp, 17)
    o = {"observed": [0, 1, 2], "t_masked": [1, 2], "p_masked": [0]}[case]
    m = [i for i in range(3) if i not in o]
    assert not x[m].any()
    C = _corr(rho[:, :1])[0]
    N = np.diag(sd) @ C @ np.diag(sd)
    ref = np.linalg.inv(np.linalg.inv(N)[np.ix_(o, o)])
    emp = np.atleast_2d(np.cov(x[o]))
    tol = 6 * np.sqrt((np.outer(np.diag(ref), np.diag(ref)) + ref ** 2) / n)
    assert np.all(np.abs(emp - ref) < tol)
    assert np.all(np.abs(x[o].mean(axis=1)) < 6 * np.sqrt(np.diag(ref) / n))
    if m:
        marginal = N[np.ix_(o, o)]
        assert np.max(np.abs(marginal - ref) - tol) > 0


def test_cov_cr_inputs_consistent(orc):
    """ahat and shat are the signal draw of the diagonal CR inputs (the same
    seed); dhat = shat + nhat on observed components and 0 on masked ones."""
    wl = W.make_cov_workload([5], 4, 8)
    ahat, shat, dhat = orc.cr_inputs_cov(4, 8, wl.cl, wl.sigma, wl.rho, wl.mask, wl.mask_p, 77)
    a0, s0, _ = orc.cr_inputs(4, 8, wl.cl, wl.sigma[0:1].repeat(3, 0), wl.mask, 77)
    assert np.array_equal(ahat, a0) and np.array_equal(shat, s0)
    assert np.allclose(shat, orc.alm2map(4, 8, ahat), atol=1e-14)
    nh = orc.draw_noise_cov(4, wl.sigma, wl.rho, wl.mask, wl.mask_p, 77)
    obs = np.stack([wl.mask, wl.mask_p, wl.mask_p]).astype(bool)
    assert np.allclose(dhat, np.where(obs, shat + nh, 0.0), atol=1e-14)
    assert np.all(dhat[~obs] == 0)


@pytest.mark.slow
def test_cov_fluctuation_covariance_is_posterior(orc):
    """f = ahat - W dhat has <f f^T> = (S^{-1} + Y^T N^{-1} Y)^{-1} (Eq. 18)
    with the block-diagonal N^{-1} and distinct masks: the mean Mahalanobis
    norm of f under that covariance equals the dimension."""
    nside, lmax = 4, 8
    cl, params_all, sigma, _, z, phi = _dense_problem(nside, lmax, 3)
    npix = z.size
    rng = np.random.default_rng(21)
    rho = rng.uniform(-0.3, 0.3, (3, npix))
    mask_t = (np.abs(z) > 0.25).astype(np.uint8)
    mask_p = (np.abs(z - 0.1) > 0.2).astype(np.uint8)
    ninv = orc.cov_ninv(sigma, rho, mask_t, mask_p)
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Nd = np.zeros((3 * npix, 3 * npix))
    for i in range(3):
        for j in range(3):
            Nd[i * npix + np.arange(npix), j * npix + np.arange(npix)] = ninv[:, i, j]
    H = _prior_precision(cl, params, 0.0) + Y.T @ Nd @ Y
    Wmat = np.linalg.solve(H, Y.T @ Nd)
    K = 400
    q = []
    for seed in range(K):
        ahat, _, dhat = orc.cr_inputs_cov(nside, lmax, cl, sigma, rho, mask_t, mask_p, 2000 + seed)
        f = alm_to_params(ahat, params, lmax) - Wmat @ dhat.reshape(-1)
        q.append(f @ H @ f)
    n = len(params)
    assert abs(np.mean(q) - n) < 5 * np.sqrt(2.0 * n / K)


def test_cov_true_residual_against_the_dense_normal_equations(orc):
    """||A x - y|| / ||y|| with the block-diagonal N^-1 and distinct masks at
    nside 4 (P the prior precision, Y from scipy and Goldberg): the oracle's
    value equals the dense one at random iterates and vanishes at the dense
    Wiener filter."""
    nside, lmax = 4, 8
    cl, params_all, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    npix = z.size
    rng = np.random.default_rng(70)
    rho = rng.uniform(-0.3, 0.3, (3, npix))
    mask_t = (np.abs(z) > 0.25).astype(np.uint8)
    mask_p = (np.abs(z - 0.1) > 0.2).astype(np.uint8)
    ninv = orc.cov_ninv(sigma, rho, mask_t, mask_p)
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Nd = np.zeros((3 * npix, 3 * npix))
    for i in range(3):
        for j in range(3):
            Nd[i * npix + np.arange(npix), j * npix + np.arange(npix)] = ninv[:, i, j]
    obs = np.stack([mask_t, mask_p, mask_p])
    d = W.random_maps(nside, 1, 71)[0] * 0.05 * obs
    P = _prior_precision(cl, params, 0.0)
    e, v = np.linalg.eigh(P)
    Pmh = (v / np.sqrt(e)) @ v.T
    H = P + Y.T @ Nd @ Y
    rhs = Y.T @ Nd @ d.reshape(-1)
    dense = lambda x: np.linalg.norm(Pmh @ (H @ x - rhs)) / np.linalg.norm(Pmh @ rhs)
    res = lambda x: orc.wf_residual_cov(nside, lmax, cl, sigma, rho, mask_t, mask_p, d,
                                        params_to_alm(x, params, lmax))
    x_wf = np.linalg.solve(H, rhs)
    assert res(x_wf) < 1e-10
    for scale in [1e-3, 1e-1, 1.0]:
        x = x_wf + scale * np.linalg.norm(x_wf) / np.sqrt(len(x_wf)) * rng.standard_normal(len(x_wf))
        assert res(x) == pytest.approx(dense(x), rel=1e-9)


def test_cov_chi2_minimum_is_the_dense_identity(orc):
    """chi^2 with the block N^-1 at the dense Wiener filter equals
    d^T N^-1 d - b^T H^-1 b (b = Y^T N^-1 d, H = P + Y^T N^-1 Y) at nside 4,
    with distinct masks; at rho = 0 and one mask it is the diagonal chi^2."""
    nside, lmax = 4, 8
    cl, params_all, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    npix = z.size
    rng = np.random.default_rng(74)
    rho = rng.uniform(-0.3, 0.3, (3, npix))
    mask_t = (np.abs(z) > 0.25).astype(np.uint8)
    mask_p = (np.abs(z - 0.1) > 0.2).astype(np.uint8)
    ninv = orc.cov_ninv(sigma, rho, mask_t, mask_p)
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Nd = np.zeros((3 * npix, 3 * npix))
    for i in range(3):
        for j in range(3):
            Nd[i * npix + np.arange(npix), j * npix + np.arange(npix)] = ninv[:, i, j]
    d = W.random_maps(nside, 1, 75)[0] * 0.05 * np.stack([mask_t, mask_p, mask_p])
    H = _prior_precision(cl, params, 0.0) + Y.T @ Nd @ Y
    b = Y.T @ Nd @ d.reshape(-1)
    x = np.linalg.solve(H, b)
    a = params_to_alm(x, params, lmax)
    s = orc.alm2map(nside, lmax, a)
    got = orc.chi2_cov(nside, lmax, cl, sigma, rho, mask_t, mask_p, d, s, a)
    assert got == pytest.approx(d.reshape(-1) @ Nd @ d.reshape(-1) - b @ x, rel=1e-10)
    zero = np.zeros_like(rho)
    assert orc.chi2_cov(nside, lmax, cl, sigma, zero, mask, mask, d, s, a) == pytest.approx(
        orc.chi2(nside, lmax, cl, sigma, mask, d, s, a), rel=1e-13)
