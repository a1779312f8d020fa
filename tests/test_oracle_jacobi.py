"""Pins of the oracle's modified Jacobi refinement on the sphere (Appendix A,
harmonic form): a <- a + W~(P g(a)), g(a) = A(w (d - Y a)) - alpha Omega C^+ a,
W~ the dual messenger operator at fixed per-level counts driven by g.

- C^+ and the range projector P against numpy's pinv of each l's block;
- at the dense Wiener filter of the nside-4 problem (scipy and Goldberg
  harmonics) g vanishes, and it does not away from it;
- W~ with the source A(w d) and the counts of a forced solve is that
  solve's iteration from another start (t_0 = d there, w d here): their
  difference shrinks by more than 1e3 from 20 to 200 iterations a level;
- refinement from a deliberately short solve converges to the dense Wiener
  filter;
- the true residual ||A x - y|| / ||y|| of the Wiener-filter equation (the
  paper's diagnostic) against the dense normal equations."""
import numpy as np
import pytest

import workloads as W
from tests.harmonics_ref import alm_to_params, dense_synthesis, params_to_alm
from tests.test_oracle_dm import _dense_problem, _prior_precision, _sblock


def test_pinv_and_projector_match_numpy(orc):
    lmax = 40
    cl = W.cl_analytic(lmax)
    pinv, proj = orc.cl_pinv(lmax, cl)
    for l in range(lmax + 1):
        blk = _sblock(cl, l)
        got = np.array([[pinv[l, 0], pinv[l, 1], 0], [pinv[l, 1], pinv[l, 2], 0], [0, 0, pinv[l, 3]]])
        ref = np.linalg.pinv(blk, rcond=1e-300, hermitian=True)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
        gp = np.array([[proj[l, 0], proj[l, 1], 0], [proj[l, 1], proj[l, 2], 0], [0, 0, proj[l, 3]]])
        assert np.max(np.abs(gp - ref @ blk)) < 1e-12


def _dense_wf(orc, seed):
    nside, lmax = 4, 8
    cl, params_all, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Ninv = (mask[None, :] / sigma ** 2).reshape(-1)
    d = W.random_maps(nside, 1, seed)[0] * 0.05 * mask[None, :]
    A = _prior_precision(cl, params, 0.0) + Y.T @ (Ninv[:, None] * Y)
    x = np.linalg.solve(A, Y.T @ (Ninv * d.reshape(-1)))
    return nside, lmax, cl, sigma, mask, d, params_to_alm(x, params, lmax)


def test_source_vanishes_at_the_wiener_filter(orc):
    nside, lmax, cl, sigma, mask, d, a_wf = _dense_wf(orc, 31)
    g = orc.jacobi_source(nside, lmax, cl, sigma, mask, d, a_wf)
    alpha = np.min((sigma ** 2)[:, mask > 0])
    w = np.where(mask[None, :] > 0, alpha / sigma ** 2, 0.0)
    ref = np.max(np.abs(orc.map2alm(nside, lmax, w * d)))
    assert np.max(np.abs(g)) < 1e-9 * ref
    a_off = a_wf + 1e-3 * np.max(np.abs(a_wf)) * orc.map2alm(nside, lmax, W.random_maps(nside, 1, 32)[0])
    assert np.max(np.abs(orc.jacobi_source(nside, lmax, cl, sigma, mask, d, a_off))) > 1e-4 * ref


def test_frozen_operator_is_the_usual_iteration(orc):
    nside, lmax, cl, sigma, mask, d, _ = _dense_wf(orc, 33)
    alpha = np.min((sigma ** 2)[:, mask > 0])
    w = np.where(mask[None, :] > 0, alpha / sigma ** 2, 0.0)
    g = orc.map2alm(nside, lmax, w * d)
    lam = [30.0, 1.0]
    diffs = []
    for n in [20, 200]:
        a_f = orc.dm_frozen(nside, lmax, cl, sigma, mask, g, lam, [n, n])
        a_u = orc.dm_solve(nside, lmax, cl, sigma, mask, d, lam, forced_iters=[n, n])["alm"]
        diffs.append(np.linalg.norm(a_f - a_u) / np.linalg.norm(a_u))
    assert diffs[1] < 1e-3 * diffs[0]  # the start's difference decays at the iteration's rate


def test_refinement_converges_to_the_wiener_filter(orc):
    nside, lmax, cl, sigma, mask, d, a_wf = _dense_wf(orc, 34)
    r = orc.jacobi_refine(nside, lmax, cl, sigma, mask, d, [20.0, 4.0, 1.0], forced_iters=[15, 15, 15],
                          n_refine=25)
    err = [np.linalg.norm(a - a_wf) / np.linalg.norm(a_wf) for a in r["steps"]]
    assert err[0] > 1e-3
    assert all(b < a for a, b in zip(err[:8], err[1:9]))
    assert err[-1] < 1e-10


def test_true_residual_against_the_dense_normal_equations(orc):
    """||A x - y|| / ||y|| with A = 1 + P^-1/2 Y^T N^-1 Y P^-1/2 on the real
    parameters of the nside-4 problem (P the prior precision, Y from scipy
    and Goldberg): the oracle's residual equals it at random iterates and
    vanishes at the dense Wiener filter."""
    nside, lmax = 4, 8
    cl, params_all, sigma, mask, z, phi = _dense_problem(nside, lmax, 3)
    params = [p for p in params_all if not (p[0] == 0 and p[1] == 0)]
    Y = dense_synthesis(nside, lmax, z, phi, params)
    Ninv = (mask[None, :] / sigma ** 2).reshape(-1)
    d = W.random_maps(nside, 1, 35)[0] * 0.05 * mask[None, :]
    P = _prior_precision(cl, params, 0.0)
    e, v = np.linalg.eigh(P)
    Pmh = (v / np.sqrt(e)) @ v.T
    H = P + Y.T @ (Ninv[:, None] * Y)
    rhs = Y.T @ (Ninv * d.reshape(-1))
    dense = lambda x: np.linalg.norm(Pmh @ (H @ x - rhs)) / np.linalg.norm(Pmh @ rhs)
    x_wf = np.linalg.solve(H, rhs)
    assert orc.wf_residual(nside, lmax, cl, sigma, mask, d, params_to_alm(x_wf, params, lmax)) < 1e-10
    rng = np.random.default_rng(36)
    for scale in [1e-3, 1e-1, 1.0]:
        x = x_wf + scale * np.linalg.norm(x_wf) / np.sqrt(len(x_wf)) * rng.standard_normal(len(x_wf))
        got = orc.wf_residual(nside, lmax, cl, sigma, mask, d, params_to_alm(x, params, lmax))
        assert got == pytest.approx(dense(x), rel=1e-9)
