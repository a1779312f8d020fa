"""Independent closed forms used to pin the oracle's harmonics.

Goldberg et al. (1967), J. Math. Phys. 8, 2155: the explicit sum for the
spin-weighted spherical harmonics.  At s = 0 it reduces to the ordinary Y_lm,
which the tests compare with scipy's library routine.
"""
from math import comb, factorial, pi, sqrt

import numpy as np
from scipy.special import sph_harm_y


def goldberg(s, l, m, theta, phi=0.0):
    if l < abs(s) or l < abs(m):
        return 0.0 + 0.0j
    pref = (-1) ** m * sqrt(factorial(l + m) * factorial(l - m) * (2 * l + 1)
                            / (4 * pi * factorial(l + s) * factorial(l - s)))
    tot = 0.0
    cot = 1.0 / np.tan(theta / 2)
    for r in range(0, l - s + 1):
        k = r + s - m
        if k < 0 or k > l + s:
            continue
        tot += comb(l - s, r) * comb(l + s, k) * (-1) ** (l - r - s) * cot ** (2 * r + s - m)
    return pref * np.sin(theta / 2) ** (2 * l) * tot * np.exp(1j * m * phi)


def ylm(l, m, theta, phi):
    return sph_harm_y(l, m, theta, phi)


def real_param_index(lmax):
    """Real parameters of a real-field T/E/B alm vector with C_l > 0 modes:
    list of (field, l, m, part) with part 0 = re, 1 = im (m > 0 only)."""
    out = []
    for f in range(3):
        lmin = 0 if f == 0 else 2
        for m in range(lmax + 1):
            for l in range(max(m, lmin), lmax + 1):
                out.append((f, l, m, 0))
                if m > 0:
                    out.append((f, l, m, 1))
    return out


def dense_synthesis(nside, lmax, z, phi, params):
    """Dense real matrix Yr [3 npix, nparams] mapping real alm parameters to
    (I, Q, U) with (Q + iU) = -sum (aE + i aB) 2Y and T = sum aT Y, summed over
    -l..l with a_{l,-m} = (-1)^m a*_{lm}.  Built from scipy Y_lm and Goldberg."""
    npix = z.size
    th = np.arccos(z)
    Y = np.zeros((3 * npix, len(params)))
    cache = {}
    for j, (f, l, m, part) in enumerate(params):
        coef = 1.0 if part == 0 else 1j
        key = (f, l, m)
        if key not in cache:
            if f == 0:
                cache[key] = (ylm(l, m, th, phi), ylm(l, -m, th, phi))
            else:
                g = np.array([goldberg(2, l, m, t, p) for t, p in zip(th, phi)])
                gm = np.array([goldberg(2, l, -m, t, p) for t, p in zip(th, phi)])
                cache[key] = (g, gm)
        yp, ym = cache[key]
        # contribution of a_{lm} = coef and of a_{l,-m} = (-1)^m conj(coef)
        if f == 0:
            tmap = coef * yp + ((-1) ** m * np.conj(coef) * ym if m > 0 else 0)
            Y[:npix, j] = tmap.real
        else:
            # P = Q + iU = -sum (aE + i aB) 2Y over +-m
            if f == 1:
                a_p, a_m = coef, (-1) ** m * np.conj(coef)
                P = -(a_p * yp + (a_m * ym if m > 0 else 0))
            else:
                a_p, a_m = coef, (-1) ** m * np.conj(coef)
                P = -(1j * a_p * yp + (1j * a_m * ym if m > 0 else 0))
            Y[npix:2 * npix, j] = P.real
            Y[2 * npix:, j] = P.imag
    return Y


def params_to_alm(x, params, lmax):
    nalm = (lmax + 1) * (lmax + 2) // 2
    a = np.zeros((3, nalm), dtype=np.complex128)
    for v, (f, l, m, part) in zip(x, params):
        ix = m * (2 * lmax + 1 - m) // 2 + l
        if part == 0:
            a[f, ix] += v
        else:
            a[f, ix] += 1j * v
    return a


def alm_to_params(a, params, lmax):
    x = np.zeros(len(params))
    for j, (f, l, m, part) in enumerate(params):
        ix = m * (2 * lmax + 1 - m) // 2 + l
        x[j] = a[f, ix].real if part == 0 else a[f, ix].imag
    return x
