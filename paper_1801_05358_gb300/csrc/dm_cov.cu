// dm_cov.cu -- correlated 3x3 per-pixel noise with distinct temperature and
// polarisation masks (the noise covariance of Section 2.1 and Appendix B).
//
// Per pixel N = Sigma C Sigma, Sigma = diag(sigma_I, sigma_Q, sigma_U), C the
// unit-diagonal correlation matrix of (rho_IQ, rho_IU, rho_QU).  Masked
// components carry Sigma^{-1} = 0 (Appendix B): the temperature mask for I,
// the polarisation mask for Q and U, so N^{-1} = Sigma^{-1} C^{-1} Sigma^{-1}
// has zero rows and columns there.  T = alpha 1 with alpha the smallest
// eigenvalue of N over the observed components of every pixel.  The messenger
// equation of Appendix B, t = (Nbar^{-1} + T^{-1})^{-1} (T^{-1} s + Nbar^{-1} d),
// Nbar = N - T, is t = s + W (d - s) with W = alpha N^{-1}: with C = P^T Delta P
// and G = Sigma^{-1} P^T the Appendix B form of Nbar^{-1} is
// G (Delta - alpha G^T G)^{-1} G^T, and (G M^{-1} G^T + 1/alpha)^{-1} G M^{-1} G^T =
// alpha G (M + alpha G^T G)^{-1} G^T = alpha G Delta^{-1} G^T.  The last form has
// no inverse of M, so it also covers the corner case Nbar = 0 of Section 2.1.
//
// The iteration keeps the harmonic steps and runs the pixel part in three
// launches: the inverse ring transform of the synthesis to s, the per-pixel
// update r = W (d - s) with the Cauchy partials (which couples the three
// Stokes components of a pixel), and the forward ring transform of r.  FP64
// modes only (DM_FP64, DM_FLOAT_FLOAT).
#include <math.h>

#include <vector>

#include "dm_internal.h"

namespace dmwf {

// wd = W d per pixel (W symmetric, [npix][6] = xx, yy, zz, xy, xz, yz), every RHS
__global__ void k_wd_cov(const double *__restrict__ d, const double *__restrict__ wc, double *__restrict__ wd,
                         int64_t npix, int batch) {
  const int64_t total = npix * batch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / npix, p = i - b * npix;
    const double *w = wc + 6 * p;
    const double *db = d + b * 3 * npix;
    const double d0 = db[p], d1 = db[npix + p], d2 = db[2 * npix + p];
    double *o = wd + b * 3 * npix;
    o[p] = w[0] * d0 + w[3] * d1 + w[4] * d2;
    o[npix + p] = w[3] * d0 + w[1] * d1 + w[5] * d2;
    o[2 * npix + p] = w[4] * d0 + w[5] * d1 + w[2] * d2;
  }
}

// One block per (ring, RHS): s_new (from the inverse ring transform, in sn)
// against the state s: Cauchy partials per Stokes component into norms, s <- s_new,
// and the messenger correction t - s = W d - W s_new written over sn.  Finished
// RHS are left untouched.
__global__ void __launch_bounds__(256) k_cov_update(const RingDev *__restrict__ rings, double *__restrict__ s,
                                                    double *__restrict__ sn, const double *__restrict__ wd,
                                                    const double *__restrict__ wc, double *__restrict__ norms,
                                                    const SolveState *__restrict__ state, int64_t npix, int nrings) {
  const int r = blockIdx.x, b = blockIdx.y;
  if (state[b].done) return;  // uniform over the block
  const RingDev R = rings[r];
  double acc[6] = {0, 0, 0, 0, 0, 0};  // dd_f, ss_f for f = 0, 1, 2
  const int64_t base = (int64_t)b * 3 * npix;
  for (int j = threadIdx.x; j < R.n; j += blockDim.x) {
    const int64_t p = R.start + j;
    double x[3];
    for (int f = 0; f < 3; ++f) {
      const int64_t i = base + f * npix + p;
      const double v = sn[i], dv = v - s[i];
      acc[2 * f] += dv * dv;
      acc[2 * f + 1] += v * v;
      s[i] = v;
      x[f] = v;
    }
    const double *w = wc + 6 * p;
    const double y0 = w[0] * x[0] + w[3] * x[1] + w[4] * x[2];
    const double y1 = w[3] * x[0] + w[1] * x[1] + w[5] * x[2];
    const double y2 = w[4] * x[0] + w[5] * x[1] + w[2] * x[2];
    sn[base + p] = wd[base + p] - y0;
    sn[base + npix + p] = wd[base + npix + p] - y1;
    sn[base + 2 * npix + p] = wd[base + 2 * npix + p] - y2;
  }
  __shared__ double red[8][6];
  for (int k = 0; k < 6; ++k)
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 6; ++k) red[threadIdx.x >> 5][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) t += red[wv][threadIdx.x];
    const int f = threadIdx.x >> 1, k = threadIdx.x & 1;
    norms[(((int64_t)b * 3 + f) * nrings + r) * 2 + k] = t;
  }
}

// Mixed mode, between anchors: the state is the FP32 map Y e (s32), the full
// map s = s_anchor + Y e (s_anchor in FP32 in shi32), and the data part
// W (d - s_anchor) is carried in FP64 by the anchor, so the correction is
// r = -W (Y e).  One block per (ring, RHS): Cauchy partials of s (the change
// of Y e is the change of s), s32 <- the new Y e (from the inverse ring
// transform, in sn), and r written over sn.  Finished RHS are left untouched.
__global__ void __launch_bounds__(256) k_cov_update32(const RingDev *__restrict__ rings, float *__restrict__ s32,
                                                      double *__restrict__ sn, const float *__restrict__ shi32,
                                                      const double *__restrict__ wc, double *__restrict__ norms,
                                                      const SolveState *__restrict__ state, int64_t npix,
                                                      int nrings) {
  const int r = blockIdx.x, b = blockIdx.y;
  if (state[b].done) return;  // uniform over the block
  const RingDev R = rings[r];
  float acc[6] = {0, 0, 0, 0, 0, 0};  // per thread in FP32, the sums over threads in FP64
  const int64_t base = (int64_t)b * 3 * npix;
  for (int j = threadIdx.x; j < R.n; j += blockDim.x) {
    const int64_t p = R.start + j;
    float x[3];
    for (int f = 0; f < 3; ++f) {
      const int64_t i = base + f * npix + p;
      const float v = (float)sn[i], dv = v - s32[i], full = shi32[i] + v;
      acc[2 * f] += dv * dv;
      acc[2 * f + 1] += full * full;
      s32[i] = v;
      x[f] = v;
    }
    const double *w = wc + 6 * p;
    sn[base + p] = -(w[0] * x[0] + w[3] * x[1] + w[4] * x[2]);
    sn[base + npix + p] = -(w[3] * x[0] + w[1] * x[1] + w[5] * x[2]);
    sn[base + 2 * npix + p] = -(w[4] * x[0] + w[5] * x[1] + w[2] * x[2]);
  }
  __shared__ double red[8][6];
  double a[6];
  for (int k = 0; k < 6; ++k) {
    a[k] = acc[k];
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
  }
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 6; ++k) red[threadIdx.x >> 5][k] = a[k];
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) t += red[wv][threadIdx.x];
    const int f = threadIdx.x >> 1, k = threadIdx.x & 1;
    norms[(((int64_t)b * 3 + f) * nrings + r) * 2 + k] = t;
  }
}

// An anchor's residual under correlated noise: r = W d - W s_hi (W d stored in
// FP64 by cov_prepare_wd), shi32 = s_hi in FP32
__global__ void k_anchor_resid_wd_cov(const double *__restrict__ wd, const double *__restrict__ s_hi,
                                      const double *__restrict__ wc, double *__restrict__ r,
                                      float *__restrict__ shi32, int64_t npix, int batch) {
  const int64_t total = npix * batch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / npix, p = i - b * npix, base = b * 3 * npix;
    const double *w = wc + 6 * p;
    const double x0 = s_hi[base + p], x1 = s_hi[base + npix + p], x2 = s_hi[base + 2 * npix + p];
    r[base + p] = wd[base + p] - (w[0] * x0 + w[3] * x1 + w[4] * x2);
    r[base + npix + p] = wd[base + npix + p] - (w[3] * x0 + w[1] * x1 + w[5] * x2);
    r[base + 2 * npix + p] = wd[base + 2 * npix + p] - (w[4] * x0 + w[5] * x1 + w[2] * x2);
    shi32[base + p] = (float)x0;
    shi32[base + npix + p] = (float)x1;
    shi32[base + 2 * npix + p] = (float)x2;
  }
}

cudaError_t cov_prepare_wd(dm_plan *p, const double *d, cudaStream_t st) {
  k_wd_cov<<<2048, 256, 0, st>>>(d, p->wcov, p->wd, p->npix, p->batch);
  return cudaGetLastError();
}

// the pixel part of an iteration with correlated noise (FP64 state p->s64);
// its scratch map is rhi, which only the mixed mode's anchors use otherwise
// (tmpmap keeps shat of a constrained realisation across the solve)
cudaError_t cov_ring_stage(dm_plan *p, cudaStream_t st) {
  cudaError_t e = ring_stage(p, RING_INV_MAP, nullptr, p->rhi, st);
  if (e) return e;
  k_cov_update<<<dim3(p->nrings, p->batch), 256, 0, st>>>(p->rings, p->s64, p->rhi, p->wd, p->wcov, p->norms,
                                                          p->state, p->npix, p->nrings);
  if ((e = cudaGetLastError())) return e;
  return ring_stage(p, RING_FWD_MAP, p->rhi, nullptr, st);
}

// The same in the mixed mode (FP32 ring transforms of the FP32 state; rhi,
// which holds an anchor's residual only until that anchor's analysis, is the
// scratch map between anchors)
cudaError_t cov_ring_stage32(dm_plan *p, cudaStream_t st) {
  cudaError_t e = ring_stage(p, RING_INV_MAP, nullptr, p->rhi, st);
  if (e) return e;
  k_cov_update32<<<dim3(p->nrings, p->batch), 256, 0, st>>>(p->rings, p->s32, p->rhi, p->shi32, p->wcov, p->norms,
                                                            p->state, p->npix, p->nrings);
  if ((e = cudaGetLastError())) return e;
  return ring_stage(p, RING_FWD_MAP, p->rhi, nullptr, st);
}

cudaError_t anchor_residual_wd_cov(dm_plan *p, const double *s_hi, cudaStream_t st) {
  k_anchor_resid_wd_cov<<<2048, 256, 0, st>>>(p->wd, s_hi, p->wcov, p->rhi, p->shi32, p->npix, p->batch);
  return cudaGetLastError();
}

// Largest eigenvalue of a symmetric 3x3 matrix from the roots of its
// characteristic polynomial (trigonometric form for three real roots).
static double sym3_max_eig(double a00, double a11, double a22, double a01, double a02, double a12) {
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  if (p1 == 0.0) return fmax(a00, fmax(a11, a22));
  const double q = (a00 + a11 + a22) / 3.0;
  const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
  const double pp = sqrt(p2 / 6.0);
  // r = det((A - q) / pp) / 2
  const double c00 = b00 / pp, c11 = b11 / pp, c22 = b22 / pp, c01 = a01 / pp, c02 = a02 / pp, c12 = a12 / pp;
  const double det = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02);
  double r = 0.5 * det;
  r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
  const double phi = acos(r) / 3.0;
  return q + 2.0 * pp * cos(phi);
}

// The noise draw of a constrained realisation under this noise model,
// n = D z for unit normals z (Eq. 18 needs the covariance that the solve's
// precision inverts): C = L L^T row by row, x = L z; on a pixel with masked
// components the observed block of N^{-1} inverts to
// Sigma_o (C_oo - C_om C_mm^{-1} C_mo) Sigma_o, drawn by subtracting
// C_om C_mm^{-1} x_m from x_o (the draw conditioned on zero noise on the
// masked components); masked components get n = 0.  D[9] row-major,
// D = diag(sigma on observed components) K L with K that conditioning.
static void noise_draw_matrix(double s0, double s1, double s2, double r01, double r02, double r12, bool ot,
                              bool op, double *D) {
  const double l10 = r01, l20 = r02, l11 = sqrt(1.0 - l10 * l10);
  const double l21 = (r12 - l20 * l10) / l11, l22 = sqrt(1.0 - l20 * l20 - l21 * l21);
  const double L[3][3] = {{1.0, 0.0, 0.0}, {l10, l11, 0.0}, {l20, l21, l22}};
  double K[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  if (!ot && op) {  // I masked: x_Q -= r01 x_I, x_U -= r02 x_I
    K[1][0] = -r01;
    K[2][0] = -r02;
  } else if (ot && !op) {  // Q, U masked: x_I -= (r01, r02) C_mm^{-1} (x_Q, x_U)
    const double q = 1.0 - r12 * r12;
    K[0][1] = -(r01 - r02 * r12) / q;
    K[0][2] = -(r02 - r01 * r12) / q;
  }
  const double sg[3] = {ot ? s0 : 0.0, op ? s1 : 0.0, op ? s2 : 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += K[i][k] * L[k][j];
      D[3 * i + j] = sg[i] * acc;
    }
}

}  // namespace dmwf

using namespace dmwf;

extern "C" dm_status dm_set_noise_cov(dm_plan *p, const double *sigma, const double *rho, const uint8_t *mask_t,
                                      const uint8_t *mask_p) {
  if (p && p->flat) {
    p->err = "sphere plans only";
    return DM_EINVAL;
  }
  if (!p || !sigma || !rho) return DM_EINVAL;
  if (p->session) {
    p->err = "a solve is in progress on this plan";
    return DM_EBUSY;
  }
  const int64_t np = p->npix;
  std::vector<double> ninv(6 * (size_t)np), wdiag(3 * (size_t)np), dmat(9 * (size_t)np);
  double alpha = INFINITY;
  int64_t nobs = 0;
  for (int64_t i = 0; i < np; ++i) {
    const bool ot = !mask_t || mask_t[i], op = !mask_p || mask_p[i];
    const double r01 = rho[i], r02 = rho[np + i], r12 = rho[2 * np + i];
    const double det = 1.0 + 2.0 * r01 * r02 * r12 - r01 * r01 - r02 * r02 - r12 * r12;
    if (!(fabs(r01) < 1.0 && fabs(r02) < 1.0 && fabs(r12) < 1.0 && det > 0.0) || !std::isfinite(det)) {
      p->err = "correlations must give a positive definite correlation matrix at pixel " + std::to_string(i);
      return DM_EINVAL;
    }
    double si[3];
    for (int f = 0; f < 3; ++f) {
      const bool obs = f == 0 ? ot : op;
      const double sg = sigma[f * np + i];
      if (obs && (!(sg > 0.0) || !std::isfinite(sg))) {
        p->err = "sigma must be finite and > 0 on observed components";
        return DM_EINVAL;
      }
      si[f] = obs ? 1.0 / sg : 0.0;
    }
    if (ot || op) ++nobs;
    noise_draw_matrix(sigma[i], sigma[np + i], sigma[2 * np + i], r01, r02, r12, ot, op, dmat.data() + 9 * i);
    // C^{-1} (adjugate over the determinant), then Sigma^{-1} C^{-1} Sigma^{-1}
    const double i00 = (1.0 - r12 * r12) / det, i11 = (1.0 - r02 * r02) / det, i22 = (1.0 - r01 * r01) / det;
    const double i01 = (r02 * r12 - r01) / det, i02 = (r01 * r12 - r02) / det, i12 = (r01 * r02 - r12) / det;
    double *n = ninv.data() + 6 * i;
    n[0] = si[0] * si[0] * i00;
    n[1] = si[1] * si[1] * i11;
    n[2] = si[2] * si[2] * i22;
    n[3] = si[0] * si[1] * i01;
    n[4] = si[0] * si[2] * i02;
    n[5] = si[1] * si[2] * i12;
    if (ot || op) {
      const double emax = sym3_max_eig(n[0], n[1], n[2], n[3], n[4], n[5]);
      if (emax > 0.0) alpha = fmin(alpha, 1.0 / emax);
    }
  }
  if (nobs == 0 || !std::isfinite(alpha)) {
    p->err = "the masks leave no observed component";
    return DM_EINVAL;
  }
  for (size_t k = 0; k < ninv.size(); ++k) ninv[k] *= alpha;  // W = alpha N^{-1}
  for (int64_t i = 0; i < np; ++i)
    for (int f = 0; f < 3; ++f) wdiag[f * np + i] = ninv[6 * i + f];
  if (!p->wcov) {
    cudaError_t e = cudaMalloc(&p->wcov, sizeof(double) * 6 * (size_t)np);
    if (e) {
      p->err = "alloc correlated-noise weights";
      return DM_ENOMEM;
    }
    p->bytes += (int64_t)(sizeof(double) * 6 * (size_t)np);
  }
  if (!p->covdraw) {
    cudaError_t e = cudaMalloc(&p->covdraw, sizeof(double) * 9 * (size_t)np);
    if (e) {
      p->err = "alloc correlated-noise draw matrices";
      return DM_ENOMEM;
    }
    p->bytes += (int64_t)(sizeof(double) * 9 * (size_t)np);
  }
  cudaError_t e = cudaMemcpy(p->wcov, ninv.data(), sizeof(double) * 6 * (size_t)np, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(p->covdraw, dmat.data(), sizeof(double) * 9 * (size_t)np, cudaMemcpyHostToDevice);
  std::vector<uint8_t> any(np);
  for (int64_t i = 0; i < np; ++i) any[i] = ((!mask_t || mask_t[i]) || (!mask_p || mask_p[i])) ? 1 : 0;
  for (int b = 0; b < p->batch && !e; ++b) {
    // diag(W) > 0 exactly on observed components: the per-component weights
    // that the initial step (t_0 = d on observed components) reads
    e = cudaMemcpy(p->w + (size_t)b * 3 * np, wdiag.data(), sizeof(double) * 3 * np, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(p->mask + (size_t)b * np, any.data(), np, cudaMemcpyHostToDevice);
    p->alpha[b] = alpha;
    p->t_h[b] = alpha * 4.0 * M_PI / (double)np;
  }
  if (e) {  // the weights are partly overwritten: the plan needs its noise set again
    p->have_noise = false;
    p->cov = false;
    p->err = "upload correlated-noise weights";
    return DM_ECUDA;
  }
  p->cov = true;
  p->have_noise = true;
  if (p->have_cl)
    for (int b = 0; b < p->batch; ++b) {
      if ((e = build_filters(p, b, 0))) break;
    }
  if (!e) e = cudaDeviceSynchronize();
  if (e) {
    p->err = "filters";
    return DM_ECUDA;
  }
  return DM_OK;
}
