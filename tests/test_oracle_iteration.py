"""Pins of the level iteration's operator and rate, and of the quadrature it
works around (Algorithm 1 in the sphere reading a <- F [a + A (t - Y a)],
with t = (1 - w) Y a + w d).

At a fixed level that update is affine in a after the first step:
a_{k+1} = M a_k + F A W d with M = F (I - A W Y), W = diag(w), w = alpha/N on
observed pixel-components.  M is built here densely with no oracle code:
harmonics from scipy and Goldberg et al. (1967), A = Omega D^{-1} Y^T in the
real-parameter basis (D = 1 for m = 0, 2 for m > 0) and the per-l filter from
numpy's eigh (Eq. 10).  Then, at nside 4 / lmax 8, lambda = 1 and 40:

- the oracle's first iterate is F A d (t_0 = d on observed pixels), its
  second M a_1 + F A W d, and its differences obey Delta_{k+1} = M Delta_k;
- the spectral radius of M is below 1, so the level converges, and the
  oracle's differences shrink by that radius per iteration asymptotically
  (power iteration on M), which sets the iteration count of a level;
- at lmax 11 = 3 nside - 1, where A Y spans 0.53 to 1.48, the radius is still
  below 1 (0.996).

Quadrature: on HEALPix A Y is not the identity.  At fixed lmax its error
falls as nside^-2 (the ring rule is second order in the ring spacing), and
the E -> B leakage of a pure-E input falls at the same rate."""
import numpy as np
import pytest

import workloads as W
from tests.harmonics_ref import alm_to_params, dense_synthesis, params_to_alm, real_param_index
from tests.test_oracle_dm import _dense_problem, _sblock


def _filter_matrix(cl, params, mu, th):
    """F = S'(S' + T_h)^{-1} per (l, m, part) on the T/E/B parameters present,
    S' = V max(S_e, mu) V^T from numpy's eigh of the 3x3 block."""
    idx = {p: j for j, p in enumerate(params)}
    F = np.zeros((len(params), len(params)))
    for (f, l, m, part) in params:
        if f != 0:
            continue
        e, v = np.linalg.eigh(_sblock(cl, l))
        sp = np.maximum(np.maximum(e, 0.0), mu)
        Fl = (v * (sp / (sp + th))) @ v.T
        ids = [(k, idx[(k, l, m, part)]) for k in range(3) if (k, l, m, part) in idx]
        for a, ja in ids:
            for b, jb in ids:
                F[ja, jb] = Fl[a, b]
    return F


@pytest.fixture(scope="module")
def dense_level():
    nside, lmax = 4, 8
    cl, params, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    npix = z.size
    omega = 4 * np.pi / npix
    Y = dense_synthesis(nside, lmax, z, phi, params)
    D = np.array([1.0 if p[2] == 0 else 2.0 for p in params])
    A = omega * (Y.T / D[:, None])
    obs = np.tile(mask, 3).astype(bool)
    N = (sigma ** 2).reshape(-1)
    alpha = N[obs].min()
    w = np.where(obs, alpha / N, 0.0)
    d = W.random_maps(nside, 1, 8)[0] * 0.05 * mask
    return dict(nside=nside, lmax=lmax, cl=cl, params=params, sigma=sigma, mask=mask, Y=Y, A=A, w=w,
                obs=obs, th=alpha * omega, d=d)


def _iterates(orc, g, lam, ks):
    out = []
    for k in ks:
        r = orc.dm_solve(g["nside"], g["lmax"], g["cl"], g["sigma"], g["mask"], g["d"], [lam], forced_iters=[k])
        out.append(alm_to_params(r["alm"], g["params"], g["lmax"]))
    return out


@pytest.mark.parametrize("lam", [1.0, 40.0])
def test_iteration_is_the_dense_affine_map(orc, dense_level, lam):
    g = dense_level
    n = len(g["params"])
    F = _filter_matrix(g["cl"], g["params"], (lam - 1.0) * g["th"], g["th"])
    M = F @ (np.eye(n) - g["A"] @ (g["w"][:, None] * g["Y"]))
    c = F @ g["A"] @ (g["w"] * g["d"].reshape(-1))
    a1, a2, a3 = _iterates(orc, g, lam, [1, 2, 3])
    rel = lambda x, y: np.linalg.norm(x - y) / np.linalg.norm(y)
    assert rel(a1, F @ g["A"] @ (g["obs"] * g["d"].reshape(-1))) < 1e-13
    assert rel(a2, M @ a1 + c) < 1e-13
    assert rel(a3 - a2, M @ (a2 - a1)) < 1e-12


@pytest.mark.parametrize("lam", [1.0, 40.0])
def test_contraction_rate_is_the_spectral_radius(orc, dense_level, lam):
    g = dense_level
    n = len(g["params"])
    F = _filter_matrix(g["cl"], g["params"], (lam - 1.0) * g["th"], g["th"])
    M = F @ (np.eye(n) - g["A"] @ (g["w"][:, None] * g["Y"]))
    rho = np.abs(np.linalg.eigvals(M)).max()
    assert 0.5 < rho < 1.0
    K = 800
    a0, a1, a2 = _iterates(orc, g, lam, [K, K + 1, K + 2])
    ratio = np.linalg.norm(a2 - a1) / np.linalg.norm(a1 - a0)
    assert abs(ratio / rho - 1.0) < 2e-3


def _ay(orc, nside, lmax, params):
    n = len(params)
    G = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        m = orc.alm2map(nside, lmax, params_to_alm(e, params, lmax))
        G[:, j] = alm_to_params(orc.map2alm(nside, lmax, m), params, lmax)
    return G


def test_quadrature_error_is_second_order_in_ring_spacing(orc):
    """max |eig(AY) - 1| and the largest E -> B coefficient of AY, at lmax 8
    for nside 8, 16, 32: each doubling of nside divides both by 4 (to 10 %),
    and both are small at nside 32."""
    lmax = 8
    params = real_param_index(lmax)
    field = np.array([p[0] for p in params])
    err, leak = [], []
    for nside in [8, 16, 32]:
        G = _ay(orc, nside, lmax, params)
        err.append(np.abs(np.linalg.eigvals(G) - 1.0).max())
        leak.append(np.abs(G[np.ix_(field == 2, field == 1)]).max())
    for e in (err, leak):
        for a, b in zip(e[:-1], e[1:]):
            assert 3.6 < a / b < 4.4
    assert err[-1] < 3e-3 and leak[-1] < 6e-4


@pytest.mark.parametrize("lam", [1.0, 40.0])
def test_spectral_radius_below_one_at_lmax_11(lam):
    """At nside 4 / lmax 11 (= 3 nside - 1) A Y spans 0.53 to 1.48, yet the
    level still contracts: rho(M) = 0.996 (against 0.978 at lmax 8)."""
    nside, lmax = 4, 11
    cl, params, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    npix = z.size
    Y = dense_synthesis(nside, lmax, z, phi, params)
    D = np.array([1.0 if p[2] == 0 else 2.0 for p in params])
    A = 4 * np.pi / npix * (Y.T / D[:, None])
    ay = np.linalg.eigvals(A @ Y).real
    assert ay.max() > 1.4 and ay.min() < 0.6
    obs = np.tile(mask, 3).astype(bool)
    N = (sigma ** 2).reshape(-1)
    alpha = N[obs].min()
    w = np.where(obs, alpha / N, 0.0)
    th = alpha * 4 * np.pi / npix
    F = _filter_matrix(cl, params, (lam - 1.0) * th, th)
    rho = np.abs(np.linalg.eigvals(F @ (np.eye(len(params)) - A @ (w[:, None] * Y)))).max()
    assert 0.99 < rho < 1.0
