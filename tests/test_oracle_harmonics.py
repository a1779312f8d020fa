"""Pins for the oracle's spin-0 and spin-+-2 harmonics.

The paper's transforms are flat-sky Fourier transforms with an E/B rotation
(Section 2.1, Eqs. 12-16); on the sphere their counterparts are the spin-0 and
spin-+-2 spherical harmonics.  The oracle generates them with a Wigner-d
recurrence; these tests check it against scipy's Y_lm, against the Goldberg
et al. (1967) closed form, and against orthonormality by Gauss-Legendre
quadrature at high l.
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from tests.harmonics_ref import goldberg, ylm


@pytest.mark.parametrize("theta", [0.013, 0.4, 1.1, np.pi / 2, 2.3, 3.1])
def test_spin0_matches_scipy(orc, theta):
    lmax = 120
    for m in [0, 1, 2, 7, 40, 119]:
        l0, _, _ = orc.lam_theta(lmax, m, theta)
        ref = np.array([ylm(l, m, theta, 0.0).real if l >= m else 0.0 for l in range(lmax + 1)])
        # a 1-ulp change of cos(theta) moves P_l by ~ l ulp / sin(theta)
        tol = 1e-14 * lmax * max(1.0, 1.0 / np.sin(theta))
        assert np.max(np.abs(l0 - ref)) < tol


def test_goldberg_reduces_to_scipy_at_spin0():
    for theta in [0.3, 1.0, 2.5]:
        for l in range(0, 9):
            for m in range(-l, l + 1):
                assert abs(goldberg(0, l, m, theta, 0.7) - ylm(l, m, theta, 0.7)) < 1e-13


@pytest.mark.parametrize("theta", [0.05, 0.7, 1.4, 2.0, 3.0])
def test_spin2_matches_goldberg(orc, theta):
    lmax = 12
    for m in range(0, lmax + 1):
        _, lp, lm = orc.lam_theta(lmax, m, theta)
        rp = np.array([goldberg(2, l, m, theta).real for l in range(lmax + 1)])
        rm = np.array([goldberg(-2, l, m, theta).real for l in range(lmax + 1)])
        scale = max(1.0, np.max(np.abs(rp)), np.max(np.abs(rm)))
        assert np.max(np.abs(lp - rp)) < 1e-12 * scale
        assert np.max(np.abs(lm - rm)) < 1e-12 * scale


def test_explicit_low_l_spin2():
    """Textbook l = 2 forms: 2Y_20 = (1/4) sqrt(15/2pi) sin^2 theta and
    2Y_22 = (1/8) sqrt(5/pi) (1 - cos theta)^2 e^{2 i phi} (Goldberg phases)."""
    for th in [0.2, 1.0, 2.2]:
        assert goldberg(2, 2, 0, th).real == pytest.approx(0.25 * np.sqrt(15 / (2 * np.pi)) * np.sin(th) ** 2,
                                                           rel=1e-13)
        assert goldberg(2, 2, 2, th).real == pytest.approx(np.sqrt(5 / np.pi) / 8 * (1 - np.cos(th)) ** 2,
                                                           rel=1e-13)


@pytest.mark.parametrize("lmax,ms", [(300, [0, 1, 2, 3, 150, 299]), (1500, [0, 2, 700, 1400])])
def test_orthonormality_high_l(orc, lmax, ms):
    """int_0^pi sY_lm sY_l'm 2pi sin(theta) dtheta = delta_ll' for each spin."""
    x, wq = leggauss(lmax + 3)
    for m in ms:
        cols = [np.zeros((x.size, lmax + 1)) for _ in range(3)]
        for q, xx in enumerate(x):
            th = np.arccos(xx)
            vals = orc.lam_theta(lmax, m, th)
            for k in range(3):
                cols[k][q] = vals[k]
        for k, lmin in zip(range(3), [m, max(m, 2), max(m, 2)]):
            G = 2 * np.pi * (cols[k] * wq[:, None]).T @ cols[k]
            sub = G[lmin:, lmin:]
            # at l ~ 1500 the Gauss-Legendre sum itself floors near 8e-11 (scipy's
            # own eval_legendre values give the same Gram error)
            tol = 1e-11 if lmax <= 300 else 1.5e-10
            assert np.max(np.abs(sub - np.eye(sub.shape[0]))) < tol, (m, k)


def test_parity_under_reflection(orc):
    """lambda_lm(pi - theta) = (-1)^{l+m} lambda_lm(theta);
    sY_lm(pi - theta) = (-1)^{l+m} (-s)Y_lm(theta)."""
    lmax = 60
    for th in [0.3, 1.2]:
        for m in [0, 1, 5, 33]:
            a0, ap, am = orc.lam_theta(lmax, m, th)
            b0, bp, bm = orc.lam_theta(lmax, m, np.pi - th)
            sgn = np.array([(-1) ** (l + m) for l in range(lmax + 1)])
            assert np.max(np.abs(b0 - sgn * a0)) < 1e-12
            assert np.max(np.abs(bp - sgn * am)) < 1e-12
            assert np.max(np.abs(bm - sgn * ap)) < 1e-12


def test_no_underflow_garbage_near_poles(orc):
    """Near the pole the large-m functions are negligible; the rescaled
    recurrence returns finite values and stays normalised further from it."""
    lmax = 4096
    th = 1e-3
    for m in [0, 1, 2, 100, 2000, 4096]:
        vals = orc.lam_theta(lmax, m, th)
        for v in vals:
            assert np.all(np.isfinite(v))
        if m >= 100:
            assert np.max(np.abs(vals[0])) < 1e-100
    # at a latitude where m = 3000 is just oscillatory below lmax = 4096
    th = np.arcsin(3000 / 3600.0)
    v0, vp, vm = orc.lam_theta(lmax, 3000, th)
    assert np.all(np.isfinite(v0)) and np.max(np.abs(v0)) > 1e-3


def test_spin2_near_pole_high_l_accuracy(orc):
    """Accuracy of the oracle's spin-2 recurrences at the first polar ring of
    nside 2048 (theta = 4e-4) up to l = 4096, against the Wigner-d closed sum
    evaluated with 60 digits: the FP64 recurrences stay within 2e-9 relative
    (this bounds how closely any FP64 implementation can be compared there)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    nside, lmax = 2048, 4096
    _, _, _, omz, opz, _ = orc.ring_info(nside, 1)
    th = mp.acos(1 - mp.mpf(1) / (3 * nside * nside))

    def dlm(l, m, k):  # Wigner d^l_{m,k}(th) by its finite sum
        c, s = mp.cos(th / 2), mp.sin(th / 2)
        pre = mp.sqrt(mp.factorial(l + m) * mp.factorial(l - m) * mp.factorial(l + k) * mp.factorial(l - k))
        tot = mp.mpf(0)
        for j in range(max(0, k - m), min(l + k, l - m) + 1):
            tot += (-1) ** (j - k + m) * c ** (2 * l - 2 * j + k - m) * s ** (2 * j - k + m) / (
                mp.factorial(l + k - j) * mp.factorial(j) * mp.factorial(m - k + j) * mp.factorial(l - m - j))
        return pre * tot

    for m, l in [(2, 4096), (3, 2000)]:
        _, lp2, lm2 = orc.lam_ring(lmax, m, omz, opz)
        nrm = mp.sqrt((2 * l + 1) / (4 * mp.pi))
        for val, k in [(lp2[l], -2), (lm2[l], 2)]:
            ref = float(nrm * dlm(l, m, k))
            assert abs(val - ref) <= 2e-9 * abs(ref)
