// dm_diag.cu -- the paper's two quality measures of a Wiener-filter solution,
// evaluated on the device in FP64 at the end of a solve (Section 3.2 and
// Appendix C; Table 1 reports both beside every run):
//
//  true residual  ||A x - y|| / ||y|| of the Wiener-filter equation with
//                 A = 1 + S^1/2 Y^T N^-1 Y S^1/2, x = S^-1/2 a, y = S^1/2 Y^T N^-1 d.
//                 With the analysis A = Omega Y^T and w = alpha / N this is
//                 ||C^1/2 (A(w (d - Y a)) - alpha Omega C^+ a)|| / ||C^1/2 A(w d)||,
//                 each (l, m > 0) counted twice (its -m partner), C^1/2 and C^+
//                 per l from the (TT, TE, EE; BB) block;
//  chi^2          (d - s)^T N^-1 (d - s) + a^T S^-1 a (Eq. 3), the data term over
//                 observed pixel-components, the prior with C^+ (m > 0 twice).
//
// Both reuse the FP64 (or float-float) stages of the plan: one ring analysis
// of w d and one of the residual map w (d - Y a), where s = Y a is the final
// map the solve already holds.  Under correlated noise (Appendix B) w is the
// 3 x 3 block W = alpha N^-1 of each pixel, and the data term of chi^2 is
// formed from r = W (d - s) by the inverse of W's observed block.  Sums run per block in FP64 and are added on
// the host in a fixed order.
#include <math.h>

#include <vector>

#include "dm_internal.h"

namespace dmwf {

namespace {

constexpr int DG_THREADS = 256;
constexpr int DG_MAP_BLOCKS = 512;  // blocks per RHS of the map reduction

__device__ __forceinline__ int64_t dg_alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// r = w d - w s (written to r), and per block sum over w > 0 of r^2 / w
// (= w (d - s)^2 = alpha (d - s)^2 / N).  grid (DG_MAP_BLOCKS, batch).
__global__ void __launch_bounds__(DG_THREADS) k_diag_resid_map(const double *__restrict__ wd,
                                                               const double *__restrict__ w,
                                                               const double *__restrict__ s, double *__restrict__ r,
                                                               int64_t n3, double *__restrict__ part) {
  __shared__ double red[DG_THREADS / 32];
  const int b = blockIdx.y;
  const int64_t off = (int64_t)b * n3;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)DG_THREADS + threadIdx.x; i < n3; i += (int64_t)gridDim.x * DG_THREADS) {
    const double ww = w[off + i];
    const double ri = wd[off + i] - ww * s[off + i];
    r[off + i] = ri;
    if (ww > 0.0) acc += ri * ri / ww;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < DG_THREADS / 32; ++k) t += red[k];
    part[(int64_t)b * gridDim.x + blockIdx.x] = t;
  }
}

// r_o^T M^-1 r_o for the block M of the symmetric 3 x 3 w (xx, yy, zz, xy,
// xz, yz) over the components o whose diagonal entry is positive (the
// observed ones: masked components have zero rows and columns), by the
// Cholesky factor of that block; 0 when none is observed.
__device__ __forceinline__ double quad_inv_observed(const double *w, const double r[3]) {
  int idx[3], k = 0;
  for (int i = 0; i < 3; ++i)
    if (w[i] > 0.0) idx[k++] = i;
  auto W = [&](int a, int b) -> double {
    if (a == b) return w[a];
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? (hi == 1 ? w[3] : w[4]) : w[5];
  };
  double L[3][3], y[3], out = 0.0;
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j <= i; ++j) {
      double v = W(idx[i], idx[j]);
      for (int q = 0; q < j; ++q) v -= L[i][q] * L[j][q];
      L[i][j] = (i == j) ? sqrt(v) : v / L[j][j];
    }
    double v = r[idx[i]];
    for (int q = 0; q < i; ++q) v -= L[i][q] * y[q];
    y[i] = v / L[i][i];
    out += y[i] * y[i];
  }
  return out;
}

// The same under correlated noise (Appendix B): W = alpha N^-1 is a symmetric
// 3 x 3 block per pixel (wc[p][6] = xx, yy, zz, xy, xz, yz, shared by every
// RHS), r = W d - W s, and per block the sum over pixels of r_o^T W_oo^-1 r_o
// over the observed components o; since r_o = W_oo (d - s)_o this is
// alpha (d - s)^T N^-1 (d - s).  grid (DG_MAP_BLOCKS, batch).
__global__ void __launch_bounds__(DG_THREADS) k_diag_resid_map_cov(const double *__restrict__ wd,
                                                                   const double *__restrict__ wc,
                                                                   const double *__restrict__ s,
                                                                   double *__restrict__ r, int64_t npix,
                                                                   double *__restrict__ part) {
  __shared__ double red[DG_THREADS / 32];
  const int b = blockIdx.y;
  const int64_t off = (int64_t)b * 3 * npix;
  double acc = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)DG_THREADS + threadIdx.x; p < npix; p += (int64_t)gridDim.x * DG_THREADS) {
    const double *w = wc + 6 * p;
    const double x0 = s[off + p], x1 = s[off + npix + p], x2 = s[off + 2 * npix + p];
    double rr[3];
    rr[0] = wd[off + p] - (w[0] * x0 + w[3] * x1 + w[4] * x2);
    rr[1] = wd[off + npix + p] - (w[3] * x0 + w[1] * x1 + w[5] * x2);
    rr[2] = wd[off + 2 * npix + p] - (w[4] * x0 + w[5] * x1 + w[2] * x2);
    r[off + p] = rr[0];
    r[off + npix + p] = rr[1];
    r[off + 2 * npix + p] = rr[2];
    acc += quad_inv_observed(w, rr);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < DG_THREADS / 32; ++k) t += red[k];
    part[(int64_t)b * gridDim.x + blockIdx.x] = t;
  }
}

// Per (m, RHS) block, over l: mode 0 sums fac |C^1/2 g|^2 (den); mode 1 sums
// fac |C^1/2 (g - alpha Omega C^+ a)|^2 (num) and fac a^T C^+ a (prior).
// tab[l][DIAG_TAB_W] = C^1/2, C^+ and the range projector P, each (tt, te, ee,
// bb).  grid (mmax+1, batch).  Flat-sky plans (flatN = N > 0): the block is
// the column kx = m of modes (kx, ky), ky = 0 .. N-1 stored at kx N + ky, the
// table is per mode, and fac = 2 for kx > 0 stands for the Hermitian partner
// (-kx, -ky) that is not stored.
__global__ void __launch_bounds__(DG_THREADS) k_diag_alm(const double2 *__restrict__ g,
                                                         const double2 *__restrict__ a,
                                                         const double *__restrict__ tab,
                                                         const double *__restrict__ aomega, int lmax, int64_t nalm,
                                                         int mode, int flatN, double *__restrict__ part) {
  __shared__ double red[2][DG_THREADS / 32];
  const int m = blockIdx.x, b = blockIdx.y;
  const int64_t base = flatN ? (int64_t)m * flatN : dg_alm_base(lmax, m);
  const int lo = flatN ? 0 : m, hi = flatN ? flatN - 1 : lmax;
  const double fac = (m == 0) ? 1.0 : 2.0;
  const double ao = mode ? aomega[b] : 0.0;
  const double2 *gb = g + (int64_t)b * 3 * nalm + base;
  const double2 *ab = a + (int64_t)b * 3 * nalm + base;
  double acc = 0.0, pri = 0.0;
  for (int l = lo + threadIdx.x; l <= hi; l += DG_THREADS) {
    const double *h = tab + DIAG_TAB_W * (flatN ? base + l : (int64_t)l), *q = h + 4;
    double2 gt = gb[l], ge = gb[nalm + l], gbb = gb[2 * nalm + l];
    if (mode) {
      const double2 at = ab[l], ae = ab[nalm + l], abb = ab[2 * nalm + l];
      // C^+ a, and the prior a^T C^+ a (real and imaginary parts)
      const double ct_x = q[0] * at.x + q[1] * ae.x, ct_y = q[0] * at.y + q[1] * ae.y;
      const double ce_x = q[1] * at.x + q[2] * ae.x, ce_y = q[1] * at.y + q[2] * ae.y;
      const double cb_x = q[3] * abb.x, cb_y = q[3] * abb.y;
      pri += fac * (at.x * ct_x + at.y * ct_y + ae.x * ce_x + ae.y * ce_y + abb.x * cb_x + abb.y * cb_y);
      gt.x -= ao * ct_x;
      gt.y -= ao * ct_y;
      ge.x -= ao * ce_x;
      ge.y -= ao * ce_y;
      gbb.x -= ao * cb_x;
      gbb.y -= ao * cb_y;
    }
    const double ht_x = h[0] * gt.x + h[1] * ge.x, ht_y = h[0] * gt.y + h[1] * ge.y;
    const double he_x = h[1] * gt.x + h[2] * ge.x, he_y = h[1] * gt.y + h[2] * ge.y;
    const double hb_x = h[3] * gbb.x, hb_y = h[3] * gbb.y;
    acc += fac * (ht_x * ht_x + ht_y * ht_y + he_x * he_x + he_y * he_y + hb_x * hb_x + hb_y * hb_y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_down_sync(0xffffffffu, acc, o);
    pri += __shfl_down_sync(0xffffffffu, pri, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = acc;
    red[1][threadIdx.x >> 5] = pri;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int k = 0; k < DG_THREADS / 32; ++k) {
      t0 += red[0][k];
      t1 += red[1][k];
    }
    const int64_t o = ((int64_t)b * gridDim.x + m) * 2;
    part[o] = t0;
    part[o + 1] = t1;
  }
}

// eigen-decomposition of the symmetric block [[tt, te], [te, ee]]: e1, e2 with
// unit eigenvectors v1 = (c, s), v2 = (-s, c); a zero off-diagonal keeps the
// diagonal exactly (so a zero spectrum gives exact zero eigenvalues)
void eig_sym2(double tt, double te, double ee, double &e1, double &e2, double &c, double &s) {
  if (te == 0.0) {
    e1 = tt;
    e2 = ee;
    c = 1.0;
    s = 0.0;
    return;
  }
  const double th = 0.5 * atan2(2.0 * te, tt - ee);
  c = cos(th);
  s = sin(th);
  e1 = tt * c * c + 2.0 * te * c * s + ee * s * s;
  e2 = tt * s * s - 2.0 * te * c * s + ee * c * c;
}

}  // namespace

// One table row: C^1/2, C^+ and the range projector of the block
// [[tt, te], [te, ee]] and of bb, each as (tt, te, ee, bb).
static void diag_row(double tt, double te, double ee, double bb, double *h) {
  double e1, e2, c, s;
  eig_sym2(tt, te, ee, e1, e2, c, s);
  const double r1 = e1 > 0.0 ? sqrt(e1) : 0.0, r2 = e2 > 0.0 ? sqrt(e2) : 0.0;
  const double i1 = e1 > 0.0 ? 1.0 / e1 : 0.0, i2 = e2 > 0.0 ? 1.0 / e2 : 0.0;
  // f(C) = f(e1) v1 v1^T + f(e2) v2 v2^T, v1 = (c, s), v2 = (-s, c)
  double *q = h + 4, *pr = h + 8;
  h[0] = r1 * c * c + r2 * s * s;
  h[1] = (r1 - r2) * c * s;
  h[2] = r1 * s * s + r2 * c * c;
  h[3] = bb > 0.0 ? sqrt(bb) : 0.0;
  q[0] = i1 * c * c + i2 * s * s;
  q[1] = (i1 - i2) * c * s;
  q[2] = i1 * s * s + i2 * c * c;
  q[3] = bb > 0.0 ? 1.0 / bb : 0.0;
  const double p1 = e1 > 0.0 ? 1.0 : 0.0, p2 = e2 > 0.0 ? 1.0 : 0.0;
  pr[0] = p1 * c * c + p2 * s * s;
  pr[1] = (p1 - p2) * c * s;
  pr[2] = p1 * s * s + p2 * c * c;
  pr[3] = bb > 0.0 ? 1.0 : 0.0;
}

static cudaError_t upload_diag_tab(dm_plan *p, const std::vector<double> &t, size_t rows) {
  cudaError_t e = cudaSuccess;
  if (!p->diag_tab) {
    e = cudaMalloc((void **)&p->diag_tab, sizeof(double) * DIAG_TAB_W * rows);
    if (e) return e;
    p->bytes += (int64_t)(sizeof(double) * DIAG_TAB_W * rows);
  }
  return cudaMemcpy(p->diag_tab, t.data(), sizeof(double) * DIAG_TAB_W * rows, cudaMemcpyHostToDevice);
}

// C^1/2, C^+ and the range projector per l on the host (FP64), uploaded
// beside the spectra.
cudaError_t diag_tables(dm_plan *p) {
  const int L = p->lmax + 1;
  std::vector<double> t(DIAG_TAB_W * (size_t)L, 0.0);
  for (int l = 0; l < L; ++l)
    diag_row(p->cl_h[l], p->cl_h[3 * L + l], p->cl_h[L + l], p->cl_h[2 * L + l], &t[DIAG_TAB_W * (size_t)l]);
  return upload_diag_tab(p, t, (size_t)L);
}

// The same per mode of a flat-sky plan, from its spectra in the stored mode
// order (cl[4][nmodes]: TT, EE, BB, TE).
cudaError_t diag_tables_flat(dm_plan *p, const std::vector<double> &cl) {
  const int64_t nm = p->nmodes;
  std::vector<double> t(DIAG_TAB_W * (size_t)nm, 0.0);
  for (int64_t k = 0; k < nm; ++k)
    diag_row(cl[k], cl[3 * nm + k], cl[nm + k], cl[2 * nm + k], &t[DIAG_TAB_W * (size_t)k]);
  return upload_diag_tab(p, t, (size_t)nm);
}

// The diagnostics of every RHS of the plan's final iterate (p->a, with
// s64 = Y a).  Runs the FP64-class stages (FP64 or float-float, as the
// plan's anchors do in the mixed mode); synchronises the stream.
cudaError_t diagnostics(dm_plan *p, cudaStream_t st, std::vector<double> &resid, std::vector<double> &chi2) {
  const int B = p->batch;
  resid.assign(B, NAN);
  chi2.assign(B, NAN);
  if (!p->diag_tab) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  const size_t an = sizeof(double2) * 3 * (size_t)p->nalm * B;
  const int nm = p->mmax + 1;
  const size_t npart = (size_t)B * std::max(DG_MAP_BLOCKS, 2 * nm);
  if (!p->diag_alm) {
    if ((e = cudaMalloc((void **)&p->diag_alm, an))) return e;
    p->bytes += (int64_t)an;
  }
  if (!p->diag_part) {
    if ((e = cudaMalloc((void **)&p->diag_part, sizeof(double) * 3 * npart))) return e;
    p->bytes += (int64_t)(sizeof(double) * 3 * npart);
  }
  if (!p->diag_ao) {
    if ((e = cudaMalloc((void **)&p->diag_ao, sizeof(double) * B))) return e;
    p->bytes += (int64_t)(sizeof(double) * B);
  }
  const double hpix = p->flat ? p->flatL / p->flatN : 0.0;
  const double omega = p->flat ? hpix * hpix : 4.0 * M_PI / (double)p->npix;  // Omega_p on a flat patch
  std::vector<double> ao(B);
  for (int b = 0; b < B; ++b) ao[b] = p->alpha[b] * omega;
  if ((e = cudaMemcpyAsync(p->diag_ao, ao.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st))) return e;
  double *part_map = p->diag_part, *part_den = p->diag_part + npart, *part_num = p->diag_part + 2 * npart;
  // the FP64-class stages, on every RHS
  const bool sa = p->state_active;
  const dm_precision prec = p->prec;
  const bool ffn = p->ff_now;
  p->state_active = false;
  if (prec != DM_FP64) {
    p->prec = DM_FP64;
    p->ff_now = p->anchor_ff;
  }
  const int64_t n3 = 3 * p->npix;
  // r = w (d - Y a) (W (d - Y a) under correlated noise) into tmpmap2, and
  // the data term of chi^2
  if (p->cov)
    k_diag_resid_map_cov<<<dim3(DG_MAP_BLOCKS, B), DG_THREADS, 0, st>>>(p->wd, p->wcov, p->s64, p->tmpmap2,
                                                                        p->npix, part_map);
  else
    k_diag_resid_map<<<dim3(DG_MAP_BLOCKS, B), DG_THREADS, 0, st>>>(p->wd, p->w, p->s64, p->tmpmap2, n3, part_map);
  e = cudaGetLastError();
  // den: A(w d)
  if (!e) e = ring_stage(p, RING_FWD_MAP, p->wd, nullptr, st);
  if (!e) e = legendre_analysis(p, ANA_PLAIN, p->diag_alm, st);
  if (!e) {
    k_diag_alm<<<dim3(nm, B), DG_THREADS, 0, st>>>(p->diag_alm, p->a, p->diag_tab, p->diag_ao, p->lmax, p->nalm, 0,
                                                    p->flat ? p->flatN : 0, part_den);
    e = cudaGetLastError();
  }
  // num and prior: A(r) - alpha Omega C^+ a
  if (!e) e = ring_stage(p, RING_FWD_MAP, p->tmpmap2, nullptr, st);
  if (!e) e = legendre_analysis(p, ANA_PLAIN, p->diag_alm, st);
  if (!e) {
    k_diag_alm<<<dim3(nm, B), DG_THREADS, 0, st>>>(p->diag_alm, p->a, p->diag_tab, p->diag_ao, p->lmax, p->nalm, 1,
                                                    p->flat ? p->flatN : 0, part_num);
    e = cudaGetLastError();
  }
  p->prec = prec;
  p->ff_now = ffn;
  p->state_active = sa;
  p->launches += 7;
  if (e) return e;
  std::vector<double> h(3 * npart);
  if ((e = cudaMemcpyAsync(h.data(), p->diag_part, sizeof(double) * 3 * npart, cudaMemcpyDeviceToHost, st)))
    return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  for (int b = 0; b < B; ++b) {
    double dat = 0.0, den = 0.0, num = 0.0, pri = 0.0;
    for (int k = 0; k < DG_MAP_BLOCKS; ++k) dat += h[(size_t)b * DG_MAP_BLOCKS + k];
    for (int m = 0; m < nm; ++m) {
      den += h[npart + ((size_t)b * nm + m) * 2];
      num += h[2 * npart + ((size_t)b * nm + m) * 2];
      pri += h[2 * npart + ((size_t)b * nm + m) * 2 + 1];
    }
    resid[b] = den > 0.0 ? sqrt(num / den) : 0.0;
    // flat sky: the prior is a^H (L^2 S)^+ a, <|a_l|^2> = L^2 S per mode
    chi2[b] = dat / p->alpha[b] + pri * (p->flat ? 1.0 / (p->flatL * p->flatL) : 1.0);
  }
  return cudaSuccess;
}

}  // namespace dmwf
