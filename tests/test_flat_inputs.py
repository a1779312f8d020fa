"""The flat-sky input recipe (workloads.make_flat_workload): the stated sky
fractions and noise level, spectra without Nyquist power, and Gaussian draws
with the Hermitian symmetry of real fields and <|a_l|^2> = L^2 C_l."""
import numpy as np
import pytest

import workloads as W


def test_masks_reach_the_paper_sky_fractions():
    wl = W.make_flat_workload([3], N=256)
    assert abs(wl.mask_t.mean() - 0.78) < 0.005
    assert abs(wl.mask_p.mean() - 0.82) < 0.005
    assert not np.array_equal(wl.mask_t, wl.mask_p)


def test_spectra_and_noise_level():
    N, L = 128, W.FLAT_L
    S = W.flat_spectra(N, L)
    assert np.all(S[:, W.flat_nyquist(N)] == 0)
    assert S[0, 0, 0] == 0 and np.all(S[1:, 0, 0] == 0)  # l = 0
    wl = W.make_flat_workload([4], N=N)
    s0 = 0.04 * np.sqrt(S[0].sum()) / L
    assert wl.sigma[0].min() >= 0.75 * s0 and wl.sigma[0].max() <= 1.25 * s0
    assert np.allclose(wl.sigma[1], np.sqrt(2) * wl.sigma[0]) and np.allclose(wl.sigma[2], wl.sigma[1])


def test_draws_are_hermitian_with_the_stated_variance():
    N, L = 64, W.FLAT_L
    S = W.flat_spectra(N, L)
    rng = np.random.default_rng(5)
    idx = (-np.arange(N)) % N
    acc = np.zeros((3, N, N))
    cross = np.zeros((N, N))
    K = 400
    for _ in range(K):
        a = W.draw_flat_alm(S, L, rng)
        assert np.max(np.abs(a - np.conj(a[:, idx][:, :, idx]))) < 1e-15 * np.max(np.abs(a))
        acc += np.abs(a) ** 2
        cross += np.real(a[0] * np.conj(a[1]))
    emp = acc / K / L ** 2
    for f, row in enumerate([0, 1, 2]):  # TT, EE, BB
        sel = S[row] > 0
        ratio = emp[f][sel] / S[row][sel]
        assert np.mean(ratio) == pytest.approx(1.0, abs=0.02)
    sel = S[3] > 0
    assert np.mean(cross[sel] / K / L ** 2 / S[3][sel]) == pytest.approx(1.0, abs=0.03)


def test_correlated_noise_option():
    N = 128
    wl = W.make_flat_workload([6, 7], N=N, rho_max=0.3)
    assert wl.rho is not None and np.abs(wl.rho).max() <= 0.3
    n = wl.noise[0]
    obs = np.stack([wl.mask_t, wl.mask_p, wl.mask_p]).astype(bool)
    assert not n[~obs].any()
    both = obs[0] & obs[1]
    # E[x y | rho] = rho_IQ for the normalised noise, so E[x y rho] = E[rho^2]
    # (about 0.03), where noise that ignored rho would give 0
    x, y, r = n[0][both] / wl.sigma[0][both], n[1][both] / wl.sigma[1][both], wl.rho[0][both]
    assert np.mean(x * y * r) == pytest.approx(np.mean(r * r), abs=5 * np.std(x * y * r) / np.sqrt(both.sum()))
    assert W.make_flat_workload([6], N=N).rho is None
