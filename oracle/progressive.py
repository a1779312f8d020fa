"""Progressive working resolution of the dual messenger solve (the speed-up
the paper proposes in Section 4): each cooling level runs at the smallest
HEALPix resolution whose band limit stays a margin above the current
l_iter, so that early levels cost a fraction of the full transforms.

TEST INFRASTRUCTURE ONLY: tests/ call it; the CUDA product path never
imports it.  Plain numpy (float64) around the C oracle's transforms.

Reading (the paper gives the idea in one sentence):

* l_iter(mu) (Section 2): the largest l at which the truncated signal
  covariance S-bar = Theta(S - U) still has power, i.e. the largest l whose
  (TT, TE, EE) block or BB has an eigenvalue above mu; 0 when none has.
* Level k, mu_k = (lambda_k - 1) T_h with T_h = alpha Omega of the FULL
  resolution (the schedule is a property of the problem):
  band limit L_k = min(lmax, max(l_min, ceil((1 + margin) l_iter(mu_k))));
  nside_k = the smallest power of two n <= nside with 2 n >= L_k.  The last
  level (mu = 0) always runs at the full (nside, lmax).
* The data of a coarse level: per Stokes component the inverse-noise
  weighted mean of the observed children of each coarse pixel (HEALPix
  nested hierarchy), with noise variance 1 / sum N_c^-1; a coarse pixel with
  no observed child is masked.  alpha_k, w_k and T_h,k follow from that noise
  at that resolution, and the level's filter uses mu_k with T_h,k:
  f = max(S_e, mu_k) / (max(S_e, mu_k) + T_h,k), i.e. lambda'_k = 1 +
  mu_k / T_h,k in the coarse plan's own parametrisation.
* Between levels the harmonic iterate carries over: modes l <= L_k are kept
  (zero above), and the next level continues the iteration from it,
  a <- F_k [a + A(w (d - Y a))] (the step of the usual iteration).  The first
  level starts as Algorithm 1 does (s_0 = 0, t_0 = d).
With margin large enough that every level runs at full resolution this is
the usual solve, iteration for iteration.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O

# HEALPix base faces (Gorski et al. 2005): ring index of the southernmost
# corner row (in units of nside) and the longitude index of the face centre
JRLL = np.array([2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4])
JPLL = np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7])


def _spread(v: np.ndarray) -> np.ndarray:
    """bits of v at the even positions of the result (bit interleaving)"""
    out = np.zeros_like(v)
    for b in range(16):
        out |= ((v >> b) & 1) << (2 * b)
    return out


def nest2ring(nside: int, pn: np.ndarray) -> np.ndarray:
    """RING index of the NESTED pixels pn: face f = pn // nside^2, in-face
    x and y from the even and odd bits of pn mod nside^2, then the ring
    number jr = JRLL[f] nside - x - y - 1 and the position along the ring."""
    pn = np.asarray(pn, dtype=np.int64)
    npface = nside * nside
    f = pn // npface
    ipf = pn % npface
    x = np.zeros_like(ipf)
    y = np.zeros_like(ipf)
    for b in range(16):
        x |= ((ipf >> (2 * b)) & 1) << b
        y |= ((ipf >> (2 * b + 1)) & 1) << b
    jr = JRLL[f] * nside - x - y - 1
    npix = 12 * npface
    ncap = 2 * nside * (nside - 1)
    nr = np.where(jr < nside, jr, np.where(jr > 3 * nside, 4 * nside - jr, nside))
    before = np.where(jr < nside, 2 * nr * (nr - 1),
                      np.where(jr > 3 * nside, npix - 2 * nr * (nr + 1), ncap + (jr - nside) * 4 * nside))
    kshift = np.where((jr >= nside) & (jr <= 3 * nside), (jr - nside) & 1, 0)
    jp = (JPLL[f] * nr + x - y + 1 + kshift) // 2
    jp = np.where(jp > 4 * nr, jp - 4 * nr, jp)
    jp = np.where(jp < 1, jp + 4 * nr, jp)
    return before + jp - 1


def ring2nest_table(nside: int) -> np.ndarray:
    """nest[ring pixel] for every pixel (the inverse permutation of nest2ring)."""
    npix = 12 * nside * nside
    r = nest2ring(nside, np.arange(npix))
    nest = np.empty(npix, dtype=np.int64)
    nest[r] = np.arange(npix)
    return nest


def parent_map(nside: int, nside_k: int) -> np.ndarray:
    """RING index at nside_k of the coarse pixel containing each RING pixel
    at nside (nside / nside_k a power of two): the nested index shifted by
    two bits per halving."""
    j = int(round(math.log2(nside // nside_k)))
    nest = ring2nest_table(nside)
    return nest2ring(nside_k, nest >> (2 * j))


def degrade(d, sigma, mask, nside: int, nside_k: int):
    """(d_k, sigma_k, mask_k) at nside_k: per component the inverse-noise
    weighted mean over the observed children, variance 1 / sum N_c^-1."""
    if nside_k == nside:
        return np.asarray(d, float), np.asarray(sigma, float), np.asarray(mask, np.uint8)
    par = parent_map(nside, nside_k)
    npk = 12 * nside_k * nside_k
    obs = np.asarray(mask, bool)
    winv = np.where(obs[None, :], 1.0 / np.where(obs[None, :], sigma, 1.0) ** 2, 0.0)
    W = np.zeros((3, npk))
    num = np.zeros((3, npk))
    for f in range(3):
        W[f] = np.bincount(par, weights=winv[f], minlength=npk)
        num[f] = np.bincount(par, weights=winv[f] * np.where(obs, d[f], 0.0), minlength=npk)
    mk = (W[0] > 0).astype(np.uint8)
    safe = np.where(W > 0, W, 1.0)
    dk = np.where(W > 0, num / safe, 0.0)
    sk = np.where(W > 0, 1.0 / np.sqrt(safe), 1.0)
    return dk, sk, mk


def ell_iter(cl: np.ndarray, mu: float) -> int:
    """Largest l whose TE block or BB has an eigenvalue above mu (0 if none)."""
    tt, ee, bb, te = cl
    tr, det = tt + ee, tt * ee - te * te
    emax = 0.5 * tr + np.sqrt(np.maximum(0.25 * tr * tr - det, 0.0))
    above = np.nonzero((np.maximum(emax, bb) > mu))[0]
    return int(above[-1]) if above.size else 0


def level_resolution(nside: int, lmax: int, cl: np.ndarray, mu: float, margin: float, lmin: int):
    """(nside_k, L_k) of a level with threshold mu (mu = 0: full resolution)."""
    if mu <= 0.0:
        return nside, lmax
    Lk = min(lmax, max(lmin, int(math.ceil((1.0 + margin) * ell_iter(cl, mu)))))
    nk = 1
    while 2 * nk < Lk and nk < nside:
        nk *= 2
    return min(nk, nside), Lk


def _almidx(lmax):
    return np.array([O.almidx(lmax, l, m) for m in range(lmax + 1) for l in range(m, lmax + 1)])


def change_band(a: np.ndarray, l_from: int, l_to: int) -> np.ndarray:
    """Harmonic coefficients [3, nalm] at band limit l_from to l_to: the modes
    l <= min(l_from, l_to) kept, zero above."""
    out = np.zeros((3, O.nalm(l_to)), dtype=np.complex128)
    lc = min(l_from, l_to)
    for m in range(lc + 1):
        for l in range(m, lc + 1):
            out[:, O.almidx(l_to, l, m)] = a[:, O.almidx(l_from, l, m)]
    return out


def dm_solve_progressive(nside, lmax, cl, sigma, mask, d, lambdas, eps=None, forced_iters=None, margin=0.25,
                         lmin=8, max_iter=100000):
    """The dual messenger solve with a working resolution per level (see the
    module docstring).  Returns s and alm at full resolution, the per-level
    counts and each level's (nside_k, L_k)."""
    nl = len(lambdas)
    mask = np.ones(12 * nside * nside, np.uint8) if mask is None else np.asarray(mask, np.uint8)
    alpha = O.alpha(sigma, mask)
    th = alpha * 4.0 * math.pi / (12 * nside * nside)
    a, Lprev = None, None
    counts, res, total = [], [], 0
    for k in range(nl):
        mu = (lambdas[k] - 1.0) * th
        nk, Lk = level_resolution(nside, lmax, cl, mu, margin, lmin)
        if k == nl - 1:
            nk, Lk = nside, lmax
        res.append((nk, Lk))
        dk, sk, mk = degrade(d, sigma, mask, nside, nk)
        alk = O.alpha(sk, mk)
        thk = alk * 4.0 * math.pi / (12 * nk * nk)
        lamk = 1.0 + mu / thk
        clk = np.ascontiguousarray(cl[:, :Lk + 1])
        want = None if forced_iters is None else int(forced_iters[k])
        ek = None if eps is None else float(eps[k])
        if a is None:  # Algorithm 1's start: s_0 = 0, t_0 = d
            r = O.dm_solve(nk, Lk, clk, sk, mk, dk, [lamk], eps=None if ek is None else [ek],
                           forced_iters=None if want is None else [want], max_iter=max_iter - total)
            a, n = r["alm"], r["iters"]
        else:
            a, n = _continue(nk, Lk, clk, sk, mk, dk, lamk, thk, change_band(a, Lprev, Lk), ek, want,
                             max_iter - total)
        counts.append(n)
        total += n
        Lprev = Lk
    return {"alm": a, "s": O.alm2map(nside, lmax, a), "iters_per_level": np.array(counts), "iters": total,
            "levels": res}


def _continue(nside, lmax, cl, sigma, mask, d, lam, th, a, eps, want, max_iter):
    """One level of the usual iteration from the iterate a:
    a <- F [a + A(w (d - Y a))], s = Y a, until the Cauchy ratio drops below
    eps or `want` iterations ran."""
    alpha = O.alpha(sigma, mask)
    w = O.weights(sigma, mask, alpha)
    coef = O.filter_coefs(lmax, cl, (lam - 1.0) * th, th)
    s = O.alm2map(nside, lmax, a)
    n = 0
    while True:
        if want is not None and n >= want:
            break
        if want is None and n >= max_iter:
            break
        r = w * (d - s)
        a = O.apply_filter(lmax, coef, a + O.map2alm(nside, lmax, r))
        sn = O.alm2map(nside, lmax, a)
        c = np.sqrt(np.sum((sn - s) ** 2) / np.sum(sn * sn))
        s = sn
        n += 1
        if want is None and c < eps:
            break
    return a, n
