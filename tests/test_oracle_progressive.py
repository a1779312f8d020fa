"""Pins of the progressive-resolution oracle (oracle/progressive.py; the
paper's Section 4 proposal of a working resolution that follows l_iter):

- the HEALPix nested hierarchy it degrades by: nest2ring is a permutation,
  the identity at nside 1, and every coarse pixel holds exactly 4^j fine
  pixels whose centres lie within one coarse pixel size of its centre (a
  wrong face, bit order or ring shift fails this for many pixels);
- the inverse-noise weighted degrade: a map constant on coarse pixels comes
  back unchanged, the noise variance is 1 / sum N_c^-1 over observed children,
  masked children carry no weight and a coarse pixel with none is masked;
- l_iter against a brute-force eigenvalue search per l, and the band and
  resolution rule;
- with every level at full resolution the solve is the usual one
  (orc_dm_solve) iteration for iteration;
- after coarse levels, the last level's fixed point is still the dense Wiener
  filter of the full-resolution problem."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import progressive as P
from tests.harmonics_ref import alm_to_params, dense_synthesis, real_param_index
from tests.test_oracle_dm import _dense_problem, _prior_precision


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
def test_nest2ring_is_a_permutation(nside):
    npix = 12 * nside * nside
    r = P.nest2ring(nside, np.arange(npix))
    assert sorted(r.tolist()) == list(range(npix))
    if nside == 1:
        assert r.tolist() == list(range(12))


def _centres(nside):
    z, phi = W.pixel_centers(nside)
    st = np.sqrt(1.0 - z * z)
    return np.stack([st * np.cos(phi), st * np.sin(phi), z])


@pytest.mark.parametrize("nside,nk", [(8, 4), (8, 2), (16, 4)])
def test_children_lie_in_their_parent(nside, nk):
    par = P.parent_map(nside, nk)
    counts = np.bincount(par, minlength=12 * nk * nk)
    assert np.all(counts == (nside // nk) ** 2)
    cf, cc = _centres(nside), _centres(nk)
    ang = np.arccos(np.clip(np.sum(cf * cc[:, par], axis=0), -1.0, 1.0))
    size = math.sqrt(4 * math.pi / (12 * nk * nk))
    assert ang.max() < size


def test_degrade_weights():
    nside, nk = 8, 2
    rng = np.random.default_rng(1)
    npix = 12 * nside * nside
    par = P.parent_map(nside, nk)
    coarse = rng.standard_normal((3, 12 * nk * nk))
    sigma = 0.5 + rng.random((3, npix))
    mask = (rng.random(npix) > 0.3).astype(np.uint8)
    mask[par == 5] = 0  # one coarse pixel with no observed child
    d = coarse[:, par]
    dk, sk, mk = P.degrade(d, sigma, mask, nside, nk)
    assert mk[5] == 0 and mk.sum() == 12 * nk * nk - 1
    assert np.allclose(dk[:, mk > 0], coarse[:, mk > 0], rtol=1e-13, atol=1e-13)
    for q in np.nonzero(mk)[0][:10]:
        ch = (par == q) & (mask > 0)
        assert np.allclose(sk[:, q], 1.0 / np.sqrt(np.sum(1.0 / sigma[:, ch] ** 2, axis=1)), rtol=1e-13)


def test_ell_iter_and_resolution_rule():
    lmax = 60
    cl = W.cl_analytic(lmax)
    for mu in [1e-2, 1e-4, 1e-6, 1e-9, 0.0]:
        brute = 0
        for l in range(lmax + 1):
            blk = np.array([[cl[0, l], cl[3, l]], [cl[3, l], cl[1, l]]])
            if max(np.linalg.eigvalsh(blk).max(), cl[2, l]) > mu:
                brute = l
        assert P.ell_iter(cl, mu) == brute
        nk, Lk = P.level_resolution(64, lmax, cl, mu, 0.25, 4)
        if mu == 0.0:
            assert (nk, Lk) == (64, lmax)
        else:
            assert Lk == min(lmax, max(4, math.ceil(1.25 * brute)))
            assert 2 * nk >= Lk and (nk == 1 or 2 * (nk // 2) < Lk)


def test_full_resolution_levels_are_the_usual_solve(orc):
    wl = W.make_workload("nside16", [2], nside=8, lmax=16)
    d = wl.data([orc.alm2map(8, 16, wl.alm_true[0])])[0]
    lam = W.lambda_schedule(1000.0, 3)
    ref = orc.dm_solve(8, 16, wl.cl, wl.sigma, wl.mask, d, lam, forced_iters=[4, 4, 4])
    got = P.dm_solve_progressive(8, 16, wl.cl, wl.sigma, wl.mask, d, lam, forced_iters=[4, 4, 4], margin=1e9)
    assert got["levels"] == [(8, 16)] * 3
    assert np.linalg.norm(got["s"] - ref["s"]) / np.linalg.norm(ref["s"]) < 1e-13
    assert np.linalg.norm(got["alm"] - ref["alm"]) / np.linalg.norm(ref["alm"]) < 1e-13


def test_coarse_levels_keep_the_dense_wiener_filter(orc):
    """A first level at nside 2 (l_iter 3 at lambda 4000), then the full
    resolution run to convergence: the dense Wiener filter of nside 4."""
    nside, lmax = 4, 8
    cl, params_all, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Ninv = (mask[None, :] / sigma ** 2).reshape(-1)
    d = W.random_maps(nside, 1, 8)[0] * 0.05 * mask[None, :]
    Pm = _prior_precision(cl, params, 0.0)
    x = np.linalg.solve(Pm + Y.T @ (Ninv[:, None] * Y), Y.T @ (Ninv * d.reshape(-1)))
    r = P.dm_solve_progressive(nside, lmax, cl, sigma, mask, d, [4000.0, 1.0], eps=[1e-6, 1e-15], margin=0.25,
                               lmin=2, max_iter=60000)
    assert r["levels"][0][0] == 2 and r["levels"][1] == (4, 8)
    xo = alm_to_params(r["alm"], params, lmax)
    assert np.linalg.norm(xo - x) / np.linalg.norm(x) < 1e-9
