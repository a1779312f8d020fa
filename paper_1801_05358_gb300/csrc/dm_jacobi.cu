// dm_jacobi.cu -- the modified Jacobi refinement of Appendix A on the device,
// in the harmonic form the sphere allows (and the flat patch, whose transform
// pair is exact, with per-mode spectra and the pixel area for Omega):
//
//   a <- a + W~(P g(a)),   g(a) = A(w (d - Y a)) - alpha Omega C^+ a,
//
// where W~ is the dual messenger operator run at the per-level iteration
// counts of the usual solve, driven by the harmonic source g instead of data:
// from a = 0, a <- F_k [a + g - A(w Y a)] (the usual iteration with w d = 0 and
// g added before the filter).  g is the harmonic image of the correction's
// data term w d - T Z with T Z = alpha (S^+ + N^-1) s (Appendix A's rewriting
// of the data term of W^+ s = N (S^-1 + N^-1) s; on the sphere A S^+ Y a =
// Omega C^+ a, so no pixel-space inverse is needed).  P projects each l's
// (TT, TE, EE; BB) block onto the range of C: along its null directions no
// equation holds, yet W~ at mu > 0 would pass them.  At the fixed point of the
// usual iteration at lambda = 1, g = 0 on the range of C, so the refinement
// converges to that fixed point (the Wiener filter) for any counts.
#include <math.h>

#include "dm_internal.h"

namespace dmwf {

namespace {

__device__ __forceinline__ int64_t jb_alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// r = w d - w s on every pixel-component of every RHS
__global__ void k_jacobi_resid(const double *__restrict__ wd, const double *__restrict__ w,
                               const double *__restrict__ s, double *__restrict__ r, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = wd[i] - w[i] * s[i];
}

// g <- P (g - alpha Omega C^+ a) per (l, m), in place.  tab[l] holds C^1/2,
// C^+ and P (each tt, te, ee, bb).  grid (mmax + 1, batch).  Flat-sky plans
// (flatN = N > 0): block m is the column kx of modes kx N + ky, ky < N, with
// the tables per mode and Omega the pixel area.
__global__ void k_jacobi_source(double2 *__restrict__ g, const double2 *__restrict__ a,
                                const double *__restrict__ tab, const double *__restrict__ aomega, int lmax,
                                int64_t nalm, int flatN) {
  const int m = blockIdx.x, b = blockIdx.y;
  const double ao = aomega[b];
  const int64_t col = flatN ? (int64_t)m * flatN : jb_alm_base(lmax, m);
  const int64_t base = (int64_t)b * 3 * nalm + col;
  const int lo = flatN ? 0 : m, hi = flatN ? flatN - 1 : lmax;
  for (int l = lo + threadIdx.x; l <= hi; l += blockDim.x) {
    const double *q = tab + DIAG_TAB_W * (flatN ? col + l : (int64_t)l) + 4, *pr = q + 4;
    const int64_t i = base + l;
    const double2 at = a[i], ae = a[i + nalm], ab = a[i + 2 * nalm];
    double2 gt = g[i], ge = g[i + nalm], gb = g[i + 2 * nalm];
    gt.x -= ao * (q[0] * at.x + q[1] * ae.x);
    gt.y -= ao * (q[0] * at.y + q[1] * ae.y);
    ge.x -= ao * (q[1] * at.x + q[2] * ae.x);
    ge.y -= ao * (q[1] * at.y + q[2] * ae.y);
    gb.x -= ao * q[3] * ab.x;
    gb.y -= ao * q[3] * ab.y;
    g[i] = make_double2(pr[0] * gt.x + pr[1] * ge.x, pr[0] * gt.y + pr[1] * ge.y);
    g[i + nalm] = make_double2(pr[1] * gt.x + pr[2] * ge.x, pr[1] * gt.y + pr[2] * ge.y);
    g[i + 2 * nalm] = make_double2(pr[3] * gb.x, pr[3] * gb.y);
  }
}

// run f with the plan's FP64-class stages (FP64, or float-float where the
// plan's anchors are), on every RHS
template <typename F>
cudaError_t fp64_class(dm_plan *p, F f) {
  const bool sa = p->state_active;
  const dm_precision prec = p->prec;
  const bool ffn = p->ff_now;
  p->state_active = false;
  if (prec != DM_FP64) {
    p->prec = DM_FP64;
    p->ff_now = p->anchor_ff;
  }
  cudaError_t e = f();
  p->prec = prec;
  p->ff_now = ffn;
  p->state_active = sa;
  return e;
}

}  // namespace

// Buffers of the refinement, made on first use.
cudaError_t jacobi_alloc(dm_plan *p) {
  const size_t an = sizeof(double2) * 3 * (size_t)p->nalm * p->batch;
  cudaError_t e = cudaSuccess;
  if (!p->jsrc) {
    if ((e = cudaMalloc((void **)&p->jsrc, an))) return e;
    p->bytes += (int64_t)an;
  }
  if (!p->jacc) {
    if ((e = cudaMalloc((void **)&p->jacc, an))) return e;
    p->bytes += (int64_t)an;
  }
  if (!p->diag_ao) {
    if ((e = cudaMalloc((void **)&p->diag_ao, sizeof(double) * p->batch))) return e;
    p->bytes += (int64_t)(sizeof(double) * p->batch);
  }
  return e;
}

// jsrc = P g(jacc) for every RHS, from the data d (device, [B][3][npix]).
cudaError_t jacobi_source(dm_plan *p, const double *d, cudaStream_t st) {
  const double hpix = p->flat ? p->flatL / p->flatN : 0.0;
  const double omega = p->flat ? hpix * hpix : 4.0 * M_PI / (double)p->npix;
  std::vector<double> ao(p->batch);
  for (int b = 0; b < p->batch; ++b) ao[b] = p->alpha[b] * omega;
  cudaError_t e = cudaMemcpyAsync(p->diag_ao, ao.data(), sizeof(double) * p->batch, cudaMemcpyHostToDevice, st);
  if (e) return e;
  e = fp64_class(p, [&]() {
    cudaError_t r = legendre_synthesis(p, p->jacc, st);  // s = Y a
    if (!r) r = ring_stage(p, RING_INV_MAP, nullptr, p->tmpmap, st);
    if (!r) r = prepare_wd(p, d, st);  // w d
    if (!r) {
      k_jacobi_resid<<<2048, 256, 0, st>>>(p->wd, p->w, p->tmpmap, p->tmpmap2, 3 * p->npix * p->batch);
      r = cudaGetLastError();
    }
    if (!r) r = ring_stage(p, RING_FWD_MAP, p->tmpmap2, nullptr, st);  // A(w (d - Y a))
    if (!r) r = legendre_analysis(p, ANA_PLAIN, p->jsrc, st);
    return r;
  });
  if (e) return e;
  k_jacobi_source<<<dim3(p->mmax + 1, p->batch), 128, 0, st>>>(p->jsrc, p->jacc, p->diag_tab, p->diag_ao, p->lmax,
                                                               p->nalm, p->flat ? p->flatN : 0);
  // a synchronous copy keeps ao alive until the upload has run
  e = cudaGetLastError();
  if (!e) e = cudaStreamSynchronize(st);
  return e;
}

// The final map s64 = Y a and w d of the data, in FP64-class arithmetic (what
// the stats' diagnostics read).
cudaError_t jacobi_final(dm_plan *p, const double *d, cudaStream_t st) {
  return fp64_class(p, [&]() {
    cudaError_t r = legendre_synthesis(p, p->a, st);
    if (!r) r = ring_stage(p, RING_INV_MAP, nullptr, p->s64, st);
    if (!r) r = prepare_wd(p, d, st);
    return r;
  });
}

}  // namespace dmwf
