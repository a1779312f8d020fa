"""Pins for the oracle's ring DFTs and spherical harmonic transforms.

Synthesis Y maps (T, E, B) harmonic coefficients to (I, Q, U) maps; analysis
A = Omega Y^dagger is the sphere counterpart of sigma^{-1} F^dagger
(Section 2.1, Eqs. 12-16, Algorithm 1).
"""
import numpy as np
import pytest

import workloads as W
from tests.harmonics_ref import dense_synthesis, params_to_alm, real_param_index


@pytest.mark.parametrize("nside", [1, 3, 8])
def test_ring_dft_forward_matches_numpy_fft(orc, nside):
    rng = np.random.default_rng(5)
    npix = 12 * nside * nside
    f = rng.standard_normal(npix)
    mmax = 3 * nside + 2
    rc = orc.ring_dft_forward(nside, mmax, f)
    for i in range(1, 4 * nside):
        nr, st, z, omz, opz, p0 = orc.ring_info(nside, i)
        F = np.fft.fft(f[st:st + nr])
        for m in range(mmax + 1):
            ref = np.exp(-1j * m * p0) * F[m % nr]
            assert abs(rc[i - 1, m] - ref) < 1e-12 * max(1, abs(ref))


@pytest.mark.parametrize("nside", [1, 3, 8])
def test_ring_dft_inverse_is_real_fold(orc, nside):
    rng = np.random.default_rng(6)
    mmax = 2 * nside + 3
    rc = rng.standard_normal((4 * nside - 1, mmax + 1)) + 1j * rng.standard_normal((4 * nside - 1, mmax + 1))
    rc[:, 0] = rc[:, 0].real
    f = orc.ring_dft_inverse(nside, mmax, rc)
    z, phi = W.pixel_centers(nside)
    for i in range(1, 4 * nside):
        nr, st, _, _, _, _ = orc.ring_info(nside, i)
        ms = np.arange(-mmax, mmax + 1)
        coef = np.concatenate([np.conj(rc[i - 1, 1:][::-1]), rc[i - 1]])
        ref = (coef[None, :] * np.exp(1j * ms[None, :] * phi[st:st + nr, None])).sum(1)
        assert np.max(np.abs(ref.imag)) < 1e-10
        assert np.max(np.abs(f[st:st + nr] - ref.real)) < 1e-10


@pytest.mark.parametrize("nside,lmax", [(2, 4), (4, 7)])
def test_synthesis_matches_dense_brute_force(orc, nside, lmax):
    """Full -l..l brute-force sum with scipy Y_lm and Goldberg 2Y_lm, with the
    real-field symmetry a_{l,-m} = (-1)^m a*_lm and (Q + iU) from 2Y only."""
    z, phi = W.pixel_centers(nside)
    params = real_param_index(lmax)
    Y = dense_synthesis(nside, lmax, z, phi, params)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(len(params))
    alm = params_to_alm(x, params, lmax)
    m_or = orc.alm2map(nside, lmax, alm)
    ref = (Y @ x).reshape(3, -1)
    assert np.max(np.abs(m_or - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("nside,lmax", [(4, 8), (8, 23)])
def test_analysis_is_scaled_adjoint_of_synthesis(orc, nside, lmax):
    """<Y a, f>_pix = <a, A f>_alm / Omega with the real-field alm inner product
    (m = 0 once, m > 0 twice)."""
    npix = 12 * nside * nside
    omega = 4 * np.pi / npix
    a = W.random_alm(lmax, 1, 11)[0]
    f = W.random_maps(nside, 1, 12)[0]
    lhs = np.sum(orc.alm2map(nside, lmax, a) * f)
    Af = orc.map2alm(nside, lmax, f)
    ms = np.concatenate([np.full(lmax + 1 - m, m) for m in range(lmax + 1)])
    wgt = np.where(ms == 0, 1.0, 2.0)
    rhs = np.sum(wgt[None, :] * (np.conj(a) * Af).real) / omega
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_roundtrip_low_l(orc):
    """A Y ~ 1 for l << nside (the HEALPix quadrature error is small there)."""
    nside, lmax = 32, 16
    a = W.random_alm(lmax, 1, 3)[0]
    b = orc.map2alm(nside, lmax, orc.alm2map(nside, lmax, a))
    assert np.linalg.norm(b - a) / np.linalg.norm(a) < 2e-3


def test_legendre_split_consistent(orc):
    """Synthesis = ring inverse DFT of the Legendre stage, analysis = Legendre
    analysis of the ring forward DFT (the two halves compose)."""
    nside, lmax = 8, 16
    a = W.random_alm(lmax, 1, 4)[0]
    rc = orc.legendre_synthesis(nside, lmax, a)
    maps = np.stack([orc.ring_dft_inverse(nside, lmax, rc[f]) for f in range(3)])
    assert np.allclose(maps, orc.alm2map(nside, lmax, a), atol=1e-13)
    f = W.random_maps(nside, 1, 5)[0]
    rc2 = np.stack([orc.ring_dft_forward(nside, lmax, f[k]) for k in range(3)])
    assert np.allclose(orc.legendre_analysis(nside, lmax, rc2), orc.map2alm(nside, lmax, f), atol=1e-13)


@pytest.mark.parametrize("nside,lmax", [(2, 5), (8, 16), (12, 30)])
def test_sampled_transforms_match_full(orc, nside, lmax):
    """The one-ring synthesis and the one-order analysis reproduce the
    corresponding slices of the full transforms (same sums, restricted)."""
    a = W.random_alm(lmax, 1, 31)[0]
    f = W.random_maps(nside, 1, 32)[0]
    full_map = orc.alm2map(nside, lmax, a)
    full_alm = orc.map2alm(nside, lmax, f)
    for i in sorted({1, 2, nside, 2 * nside, 3 * nside, 4 * nside - 1}):
        nr, st = orc.ring_info(nside, i)[:2]
        got = orc.ring_alm2map(nside, lmax, a, i)
        ref = full_map[:, st:st + nr]
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    for m in sorted({0, 1, 2, lmax // 2, lmax}):
        got = orc.map2alm_m(nside, lmax, f, m)
        idx = [orc.almidx(lmax, l, m) for l in range(m, lmax + 1)]
        ref = full_alm[:, idx]
        assert np.all(got[:, :m] == 0)
        assert np.max(np.abs(got[:, m:] - ref)) <= 1e-13 * np.max(np.abs(full_alm))
