"""Pins of the flat-sky oracle (oracle/flat.py; Section 2.1, Eqs. 12-16,
Algorithm 1), the paper's own setting on a square patch.

- analysis against the direct sums a_l = Omega_p sum_x m(x) e^{-i l.x} at
  N = 6 (brute force), its polarisation part in the spin-2 form
  E + iB = e^{-2i phi}(Q + iU) of the rotation of Eqs. 15-16, and the Nyquist
  row and column dropped;
- synthesis is the exact inverse of analysis on the harmonic space, and
  synthesis after analysis is a projection;
- E and B as gradient and curl modes: Q = (dx^2 - dy^2) psi, U = 2 dx dy psi
  is pure E with E = F^dagger[laplacian psi], and Q = -2 dx dy chi,
  U = (dx^2 - dy^2) chi is pure B with B = F^dagger[laplacian chi]
  (derivatives taken spectrally, x along axis 1);
- parity: under the mirror x -> -x, (Q, U) -> (Q, -U), E is even and B odd;
- the first iteration is the per-mode filter of F^dagger d, and with
  homogeneous unmasked noise (w = 1) it is already the fixed point;
- the converged loop against the textbook pixel-space Wiener filter
  S (S + N)^-1 d on the observed components, with S built densely from plane
  waves, at N = 8 with distinct T and P masks, at lambda = 1 and 40."""
import numpy as np
import pytest

import workloads as W
from oracle import flat as F

L = 10.0 * W.DEG


def _random_maps(N, seed):
    return np.random.default_rng(seed).standard_normal((3, N, N))


def test_analysis_is_the_direct_sum():
    N = 6
    m = _random_maps(N, 1)
    got = F.analysis(m, L)
    om = (L / N) ** 2
    k = np.fft.fftfreq(N, d=1.0 / N)
    iy, ix = np.mgrid[0:N, 0:N]
    x, y = ix * L / N, iy * L / N
    for a in range(N):
        for b in range(N):
            ly, lx = 2 * np.pi * k[a] / L, 2 * np.pi * k[b] / L
            if k[a] == -N // 2 or k[b] == -N // 2:
                assert np.all(got[:, a, b] == 0)
                continue
            ph = np.exp(-1j * (lx * x + ly * y))
            h = om * np.array([np.sum(m[f] * ph) for f in range(3)])
            assert abs(got[0, a, b] - h[0]) < 1e-13
            phi = np.arctan2(ly, lx)
            eb = np.exp(-2j * phi) * (h[1] + 1j * h[2])  # E + iB for real coefficients E, B
            # E and B are complex here; split E + iB = e^{-2i phi}(Q + iU) into its
            # two linear parts with the conjugate relation E - iB = e^{2i phi}(Q - iU)
            ebc = np.exp(2j * phi) * (h[1] - 1j * h[2])
            e, bb = (eb + ebc) / 2, (eb - ebc) / 2j
            assert abs(got[1, a, b] - e) < 1e-13 and abs(got[2, a, b] - bb) < 1e-13


def test_synthesis_inverts_analysis():
    N = 32
    a = F.analysis(_random_maps(N, 2), L)
    m = F.synthesis(a, L)
    assert np.max(np.abs(F.analysis(m, L) - a)) < 1e-13 * np.max(np.abs(a))
    m2 = F.synthesis(F.analysis(m, L), L)
    assert np.max(np.abs(m2 - m)) < 1e-13 * np.max(np.abs(m))
    # a map with Nyquist content is changed by the projection, but only there
    r = _random_maps(N, 3)
    pr = F.synthesis(F.analysis(r, L), L)
    resid = F.analysis(r - pr, L)
    assert np.max(np.abs(resid)) < 1e-13 * np.max(np.abs(F.analysis(r, L)))


def _spectral_derivs(psi, N):
    k = 2 * np.pi * np.fft.fftfreq(N, d=1.0 / N) / L
    ky, kx = np.meshgrid(k, k, indexing="ij")
    h = np.fft.fft2(psi)
    d = lambda f: np.fft.ifft2(f * h).real
    return d(-kx * kx), d(-ky * ky), d(-kx * ky)  # dxx, dyy, dxy


def _smooth_field(N, seed):
    """A real field without Nyquist content."""
    r = np.random.default_rng(seed).standard_normal((N, N))
    h = np.fft.fft2(r) * ~W.flat_nyquist(N)
    return np.fft.ifft2(h).real


@pytest.mark.parametrize("N", [16, 33])
def test_gradient_and_curl_fields_are_pure_e_and_b(N):
    psi, chi = _smooth_field(N, 4), _smooth_field(N, 5)
    pxx, pyy, pxy = _spectral_derivs(psi, N)
    cxx, cyy, cxy = _spectral_derivs(chi, N)
    lap = lambda f: F.analysis(np.stack([f, 0 * f, 0 * f]), L)[0]
    zero = np.zeros((N, N))
    ae = F.analysis(np.stack([zero, pxx - pyy, 2 * pxy]), L)
    ab = F.analysis(np.stack([zero, -2 * cxy, cxx - cyy]), L)
    ref_e, ref_b = lap(pxx + pyy), lap(cxx + cyy)
    scale = np.max(np.abs(ref_e))
    assert np.max(np.abs(ae[1] - ref_e)) < 1e-12 * scale
    assert np.max(np.abs(ae[2])) < 1e-12 * scale
    assert np.max(np.abs(ab[2] - ref_b)) < 1e-12 * np.max(np.abs(ref_b))
    assert np.max(np.abs(ab[1])) < 1e-12 * np.max(np.abs(ref_b))


def test_mirror_parity_of_e_and_b():
    N = 24
    m = _random_maps(N, 6)
    flip = lambda f: np.roll(f[..., ::-1], 1, axis=-1)  # x_j -> -x_j (mod L), also k_x -> -k_x
    mm = np.stack([flip(m[0]), flip(m[1]), -flip(m[2])])
    a, am = F.analysis(m, L), F.analysis(mm, L)
    assert np.max(np.abs(am[0] - flip(a[0]))) < 1e-13
    assert np.max(np.abs(am[1] - flip(a[1]))) < 1e-13
    assert np.max(np.abs(am[2] + flip(a[2]))) < 1e-13


def test_first_iteration_and_homogeneous_fixed_point():
    N = 32
    S = W.flat_spectra(N, L, lscale=300.0)
    sigma = np.full((3, N, N), 2e-3)
    ones = np.ones((N, N), np.uint8)
    d = _random_maps(N, 7) * 1e-3
    r = F.dm_solve(d, sigma, ones, ones, S, L, [1.0], forced_iters=[2])
    th = 4e-6 * (L / N) ** 2
    ad = F.analysis(d, L)
    ref = np.zeros_like(ad)
    for i in range(N):
        for j in range(N):
            tt, ee, bb, te = S[:, i, j]
            blk = np.array([[tt, te, 0], [te, ee, 0], [0, 0, bb]])
            ref[:, i, j] = blk @ np.linalg.solve(blk + th * np.eye(3), ad[:, i, j])
    assert np.max(np.abs(r["alm"] - ref)) < 1e-12 * np.max(np.abs(ref))
    assert r["cauchy"][1] < 1e-13  # w = 1: t = d after every step, so step 2 repeats step 1


def _dense_signal(S, N, mu):
    """Pixel covariance [3 N^2, 3 N^2] of the signal S' = V max(S_e, mu) V^T per
    mode, summed over the harmonic space as plane waves:
    Cov[X(x), Y(x')] = L^-2 sum_l (R S' R^T)_XY cos(l.(x - x'))."""
    k = np.fft.fftfreq(N, d=1.0 / N)
    iy, ix = np.mgrid[0:N, 0:N]
    x, y = (ix * L / N).ravel(), (iy * L / N).ravel()
    dx, dy = x[:, None] - x[None, :], y[:, None] - y[None, :]
    C = np.zeros((3, 3, N * N, N * N))
    for a in range(N):
        for b in range(N):
            if k[a] == -N // 2 or k[b] == -N // 2:
                continue
            ly, lx = 2 * np.pi * k[a] / L, 2 * np.pi * k[b] / L
            tt, ee, bb, te = S[:, a, b]
            e, v = np.linalg.eigh(np.array([[tt, te], [te, ee]]))
            te_blk = (v * np.maximum(np.maximum(e, 0.0), mu)) @ v.T
            sp = np.zeros((3, 3))
            sp[:2, :2] = te_blk
            sp[2, 2] = max(bb, mu)
            phi = np.arctan2(ly, lx)
            c, s = np.cos(2 * phi), np.sin(2 * phi)
            R = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
            M = R @ sp @ R.T
            cw = np.cos(lx * dx + ly * dy)
            C += M[:, :, None, None] * cw[None, None]
    C /= L ** 2
    return C.transpose(0, 2, 1, 3).reshape(3 * N * N, 3 * N * N)


@pytest.mark.parametrize("lam", [1.0, 40.0])
def test_fixed_point_is_the_pixel_space_wiener_filter(lam):
    N = 8
    S = W.flat_spectra(N, L, lscale=300.0)
    rng = np.random.default_rng(8)
    st = 0.1 * (0.75 + 0.5 * rng.random((N, N)))  # S / T_h up to about 100: the level converges fast
    sigma = np.stack([st, np.sqrt(2) * st, np.sqrt(2) * st])
    mask_t = (rng.random((N, N)) > 0.25).astype(np.uint8)
    mask_p = (rng.random((N, N)) > 0.2).astype(np.uint8)
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    d = _random_maps(N, 9) * 0.1 * obs
    r = F.dm_solve(d, sigma, mask_t, mask_p, S, L, [lam], eps=[1e-15], max_iter=20000)
    assert r["iters"] < 20000
    alpha = (sigma ** 2)[obs].min()
    mu = (lam - 1.0) * alpha * (L / N) ** 2
    Sp = _dense_signal(S, N, mu)
    o = obs.ravel()
    nv = (sigma ** 2).ravel()[o]
    x = np.linalg.solve(Sp[np.ix_(o, o)] + np.diag(nv), d.ravel()[o])
    s_ref = (Sp[:, o] @ x).reshape(3, N, N)
    assert np.linalg.norm(r["s"] - s_ref) / np.linalg.norm(s_ref) < 1e-9


def test_residual_and_chi2_at_the_wiener_filter():
    """At the dense Wiener filter of the N = 8 problem the residual
    ||A x - y|| / ||y|| vanishes and chi^2 takes its minimum
    d_o^T (S_oo + N_oo)^-1 d_o (observed components o); a perturbed solution
    has a finite residual and a larger chi^2."""
    N = 8
    S = W.flat_spectra(N, L, lscale=300.0)
    rng = np.random.default_rng(10)
    st = 0.1 * (0.75 + 0.5 * rng.random((N, N)))
    sigma = np.stack([st, np.sqrt(2) * st, np.sqrt(2) * st])
    mask_t = (rng.random((N, N)) > 0.25).astype(np.uint8)
    mask_p = (rng.random((N, N)) > 0.2).astype(np.uint8)
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    d = _random_maps(N, 11) * 0.1 * obs
    Sp = _dense_signal(S, N, 0.0)
    o = obs.ravel()
    x = np.linalg.solve(Sp[np.ix_(o, o)] + np.diag((sigma ** 2).ravel()[o]), d.ravel()[o])
    s_wf = (Sp[:, o] @ x).reshape(3, N, N)
    a_wf = F.analysis(s_wf, L)
    assert F.wf_residual(a_wf, d, sigma, mask_t, mask_p, S, L) < 1e-10
    c2 = F.chi2(a_wf, d, sigma, mask_t, mask_p, S, L)
    assert c2 == pytest.approx(float(d.ravel()[o] @ x), rel=1e-9)
    pert = a_wf + 0.01 * F.analysis(_random_maps(N, 12) * 0.1, L) * (S[[0, 1, 2]] > 0)
    assert F.wf_residual(pert, d, sigma, mask_t, mask_p, S, L) > 1e-4
    assert F.chi2(pert, d, sigma, mask_t, mask_p, S, L) > c2


def _n8_problem(seed):
    N = 8
    S = W.flat_spectra(N, L, lscale=300.0)
    rng = np.random.default_rng(seed)
    st = 0.1 * (0.75 + 0.5 * rng.random((N, N)))
    sigma = np.stack([st, np.sqrt(2) * st, np.sqrt(2) * st])
    mask_t = (rng.random((N, N)) > 0.25).astype(np.uint8)
    mask_p = (rng.random((N, N)) > 0.2).astype(np.uint8)
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    d = _random_maps(N, seed + 1) * 0.1 * obs
    Sp = _dense_signal(S, N, 0.0)
    o = obs.ravel()
    x = np.linalg.solve(Sp[np.ix_(o, o)] + np.diag((sigma ** 2).ravel()[o]), d.ravel()[o])
    return N, S, sigma, mask_t, mask_p, d, (Sp[:, o] @ x).reshape(3, N, N)


def test_jacobi_data_term_vanishes_against_the_data_at_the_wiener_filter():
    """On the range of S, F^dagger (w d - T Z(s_WF)) = 0: the Wiener-filter
    equation itself, so the Wiener filter is a fixed point of the refinement
    whatever the counts of W~ (Appendix A).  Along the null directions of S
    (l = 0 here) the data term is not zero, which is why the correction is
    projected; away from the Wiener filter the projected term is not zero."""
    N, S, sigma, mask_t, mask_p, d, s_wf = _n8_problem(20)
    alpha, w = F.weights(sigma, mask_t, mask_p)
    x = w * d - F.jacobi_data_term(s_wf, w, alpha, S, L)
    ref = np.max(np.abs(F.analysis(w * d, L)))
    g = F.analysis(F.range_projected(x, S, L), L)
    assert np.max(np.abs(g)) < 1e-10 * ref
    assert np.max(np.abs(F.analysis(x, L)[:, 0, 0])) > 1e-3 * ref  # the l = 0 mode
    s_off = s_wf + 0.01 * F.synthesis(F.analysis(_random_maps(N, 21), L), L)
    g2 = F.analysis(F.range_projected(w * d - F.jacobi_data_term(s_off, w, alpha, S, L), S, L), L)
    assert np.max(np.abs(g2)) > 1e-4 * ref


def test_jacobi_refinement_converges_to_the_wiener_filter():
    """A deliberately short usual solve (3 levels of 15 iterations, relative
    error 7e-2), then refinement steps with W~ at those counts: the distance
    to the dense Wiener filter falls at every step until rounding, and is
    below 1e-12 after 20 steps."""
    N, S, sigma, mask_t, mask_p, d, s_wf = _n8_problem(22)
    r = F.jacobi_refine(d, sigma, mask_t, mask_p, S, L, [20.0, 4.0, 1.0], forced_iters=[15, 15, 15],
                        n_refine=20)
    err = [np.linalg.norm(s - s_wf) / np.linalg.norm(s_wf) for s in r["steps"]]
    assert err[0] > 1e-2
    assert all(b < a for a, b in zip(err[:12], err[1:13]))
    assert err[-1] < 1e-12


def _cov_model(N, seed, rho_max=0.3):
    rng = np.random.default_rng(seed)
    st = 0.1 * (0.75 + 0.5 * rng.random((N, N)))
    sigma = np.stack([st, np.sqrt(2) * st, np.sqrt(2) * st])
    rho = rng.uniform(-rho_max, rho_max, (3, N, N))
    mask_t = (rng.random((N, N)) > 0.25).astype(np.uint8)
    mask_p = (rng.random((N, N)) > 0.2).astype(np.uint8)
    return sigma, rho, mask_t, mask_p


def test_cov_ninv_and_alpha_against_numpy():
    N = 6
    sigma, rho, mask_t, mask_p = _cov_model(N, 30)
    ninv = F.cov_ninv(sigma, rho, mask_t, mask_p)
    lam_max = 0.0
    for i in range(N):
        for j in range(N):
            C = np.array([[1, rho[0, i, j], rho[1, i, j]], [rho[0, i, j], 1, rho[2, i, j]],
                          [rho[1, i, j], rho[2, i, j], 1]])
            Sg = np.diag(sigma[:, i, j])
            ref = np.linalg.inv(Sg @ C @ Sg)
            o = np.array([mask_t[i, j], mask_p[i, j], mask_p[i, j]], bool)
            # Sigma^-1 = 0 on masked components: rows and columns of C^-1 scaled away
            ref = ref * np.outer(o, o)
            assert np.max(np.abs(ninv[:, :, i, j] - ref)) < 1e-12 * np.max(np.abs(ref) + 1e-300)
            if o.any():
                lam_max = max(lam_max, np.linalg.eigvalsh(ninv[:, :, i, j]).max())
    assert F.cov_alpha(ninv) == pytest.approx(1.0 / lam_max, rel=1e-13)


def test_cov_solve_at_zero_correlation_is_the_diagonal_solve():
    N = 16
    S = W.flat_spectra(N, L, lscale=300.0)
    sigma, _, mask_t, mask_p = _cov_model(N, 31)
    d = _random_maps(N, 32) * 0.1
    lam = [40.0, 4.0, 1.0]
    a = F.dm_solve(d, sigma, mask_t, mask_p, S, L, lam, forced_iters=[5, 5, 5])
    b = F.dm_solve_cov(d, sigma, np.zeros_like(sigma), mask_t, mask_p, S, L, lam, forced_iters=[5, 5, 5])
    assert np.linalg.norm(b["s"] - a["s"]) / np.linalg.norm(a["s"]) < 1e-13


@pytest.mark.parametrize("lam", [1.0, 40.0])
def test_cov_fixed_point_is_the_wiener_filter(lam):
    """(S'^-1 + N^-1)^-1 N^-1 d = S' (1 + N^-1 S')^-1 N^-1 d with the block
    per-pixel N^-1 (singular where masked), S' the dense plane-wave signal
    covariance of the level, at N = 8."""
    N = 8
    S = W.flat_spectra(N, L, lscale=300.0)
    sigma, rho, mask_t, mask_p = _cov_model(N, 33)
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    d = _random_maps(N, 34) * 0.1 * obs
    r = F.dm_solve_cov(d, sigma, rho, mask_t, mask_p, S, L, [lam], eps=[1e-15], max_iter=20000)
    assert r["iters"] < 20000
    ninv = F.cov_ninv(sigma, rho, mask_t, mask_p)
    n = 3 * N * N
    Nd = np.zeros((n, n))
    pix = np.arange(N * N)
    for i in range(3):
        for j in range(3):
            Nd[i * N * N + pix, j * N * N + pix] = ninv[i, j].ravel()
    mu = (lam - 1.0) * r["alpha"] * (L / N) ** 2
    Sp = _dense_signal(S, N, mu)
    s_ref = Sp @ np.linalg.solve(np.eye(n) + Nd @ Sp, Nd @ d.ravel())
    assert np.linalg.norm(r["s"].ravel() - s_ref) / np.linalg.norm(s_ref) < 1e-9


def test_cr_draws_reduce_and_condition():
    """The signal draw has the stated per-mode covariance; the correlated
    noise draw at rho = 0 is the diagonal one, and on a fully observed pixel
    its covariance is Sigma C Sigma while a pixel with Q, U masked has the
    conditional variance sigma_I^2 / (C^-1)_II."""
    N = 64
    S = W.flat_spectra(N, L)
    rng = np.random.default_rng(40)
    acc = np.zeros((3, N, N))
    K = 300
    for _ in range(K):
        a = F.draw_signal(rng.standard_normal((3, N, N)), S, L)
        acc += np.abs(a) ** 2
    sel = S[0] > 0
    assert np.mean(acc[0][sel] / K / L ** 2 / S[0][sel]) == pytest.approx(1.0, abs=0.02)
    sigma = np.full((3, N, N), 2.0)
    ones = np.ones((N, N), np.uint8)
    z = rng.standard_normal((3, N, N))
    assert np.array_equal(F.draw_noise(z, sigma, ones, ones, np.zeros((3, N, N))), F.draw_noise(z, sigma, ones, ones))
    r = np.array([0.5, -0.4, 0.3])
    rho = np.broadcast_to(r[:, None, None], (3, N, N)).copy()
    C = np.array([[1, r[0], r[1]], [r[0], 1, r[2]], [r[1], r[2], 1]])
    zeros = np.zeros((N, N), np.uint8)
    full, t_only = [], []
    for _ in range(40):
        z = rng.standard_normal((3, N, N))
        full.append(F.draw_noise(z, sigma, ones, ones, rho).reshape(3, -1))
        t_only.append(F.draw_noise(z, sigma, ones, zeros, rho).reshape(3, -1))
    full, t_only = np.concatenate(full, 1), np.concatenate(t_only, 1)
    n = full.shape[1]
    assert np.allclose(np.cov(full), 4.0 * C, atol=6 * 4.0 * np.sqrt(2.0 / n))
    assert not t_only[1:].any()
    assert np.var(t_only[0]) == pytest.approx(4.0 / np.linalg.inv(C)[0, 0], rel=6 * np.sqrt(2.0 / n))


@pytest.mark.parametrize("correlated", [False, True])
def test_cr_fluctuation_has_the_posterior_covariance(correlated):
    """f = shat - W dhat (Eq. 18) with the dense Wiener filter W at N = 8:
    f^T P^+ f averages the rank of P, the posterior covariance
    P = S (1 + N^-1 S)^-1, over 400 draws."""
    N = 8
    S = W.flat_spectra(N, L, lscale=300.0)
    sigma, rho, mask_t, mask_p = _cov_model(N, 41)
    if not correlated:
        rho = None
    ninv = F.cov_ninv(sigma, np.zeros_like(sigma) if rho is None else rho, mask_t, mask_p)
    n = 3 * N * N
    Nd = np.zeros((n, n))
    pix = np.arange(N * N)
    for i in range(3):
        for j in range(3):
            Nd[i * N * N + pix, j * N * N + pix] = ninv[i, j].ravel()
    Sp = _dense_signal(S, N, 0.0)
    Wd = Sp @ np.linalg.solve(np.eye(n) + Nd @ Sp, Nd)
    P = Sp @ np.linalg.inv(np.eye(n) + Nd @ Sp)
    P = 0.5 * (P + P.T)
    Pp = np.linalg.pinv(P, rcond=1e-10, hermitian=True)
    rank = np.linalg.matrix_rank(P, tol=1e-10 * np.abs(P).max(), hermitian=True)
    rng = np.random.default_rng(42)
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    q = []
    K = 400
    for _ in range(K):
        s_hat = F.synthesis(F.draw_signal(rng.standard_normal((3, N, N)), S, L), L)
        d_hat = np.where(obs, s_hat + F.draw_noise(rng.standard_normal((3, N, N)), sigma, mask_t, mask_p, rho), 0.0)
        f = s_hat.ravel() - Wd @ d_hat.ravel()
        q.append(f @ Pp @ f)
    assert abs(np.mean(q) - rank) < 5 * np.sqrt(2.0 * rank / K)


@pytest.mark.parametrize("correlated", [False, True])
def test_level_accounting_and_linearity(correlated):
    """Per-level counts add up to the total; each level ends at the first
    iteration whose Cauchy ratio is below its threshold; with fixed counts the
    solve is linear in the data."""
    N = 16
    S = W.flat_spectra(N, L, lscale=300.0)
    sigma, rho, mask_t, mask_p = _cov_model(N, 60)
    solve = (lambda *a, **k: F.dm_solve_cov(a[0], sigma, rho, mask_t, mask_p, *a[1:], **k)) if correlated else \
        (lambda *a, **k: F.dm_solve(a[0], sigma, mask_t, mask_p, *a[1:], **k))
    obs = np.stack([mask_t, mask_p, mask_p]).astype(bool)
    d1 = _random_maps(N, 61) * 0.1 * obs
    d2 = _random_maps(N, 62) * 0.1 * obs
    lam = [100.0, 10.0, 1.0]
    eps = [1e-3, 1e-4, 1e-5]
    r = solve(d1, S, L, lam, eps=eps)
    ipl = r["iters_per_level"]
    assert ipl.sum() == r["iters"] and np.all(ipl >= 1)
    ends = np.cumsum(ipl) - 1
    starts = np.concatenate([[0], ends[:-1] + 1])
    for st, en, e in zip(starts, ends, eps):
        assert r["cauchy"][en] < e and np.all(r["cauchy"][st:en] >= e)
    f = lambda d: solve(d, S, L, lam, forced_iters=[3, 3, 3])["s"]
    a, b, c = f(d1), f(d2), f(d1 + 2 * d2)
    assert np.linalg.norm(c - a - 2 * b) / np.linalg.norm(c) < 1e-12


@pytest.mark.slow
def test_chi2_at_the_wiener_filter_matches_degrees_of_freedom():
    """Section 3.2: at the converged Wiener filter chi^2 (Eq. 3) has the
    expectation n_dof, the number of observed pixel-components, with
    standard deviation sqrt(2 n_dof).  Signal and noise drawn from the
    model at N = 64 (the paper's patch, 4 % noise), one level at lambda = 1
    to a Cauchy ratio of 1e-5 (the distance to the exact Wiener filter then
    adds far less than one standard deviation to chi^2)."""
    wl = W.make_flat_workload([8], N=64)
    d = wl.data([F.synthesis(wl.alm_true[0], wl.L)])[0]
    r = F.dm_solve(d, wl.sigma, wl.mask_t, wl.mask_p, wl.S, wl.L, [1.0], eps=[1e-5], max_iter=100000)
    ndof = int(wl.mask_t.sum() + 2 * wl.mask_p.sum())
    c2 = F.chi2(r["alm"], d, wl.sigma, wl.mask_t, wl.mask_p, wl.S, wl.L)
    assert abs(c2 - ndof) < 5 * np.sqrt(2.0 * ndof)
