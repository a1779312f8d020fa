// dm_flat.cu -- the paper's own setting (Section 2.1 and 3.1): the dual
// messenger Wiener filter of T/Q/U maps on a flat square patch of side L with
// N x N pixels, whose transform pair is the 2-D FFT with the E/B rotation of
// Eqs. 12-16.
//
// The plan reuses the sphere machinery: the N rows of the grid are the
// "rings" of the ring kernels (n = N pixels at phi_j = 2 pi j / N), so the
// row transforms, the messenger update, the Cauchy partials and the level
// control are those of the sphere; the Legendre stages are replaced by the
// column transforms below.  Conventions, with pixel (y, x) at (y L/N, x L/N)
// and l = 2 pi k / L:
//   analysis   a_l = Omega_p sum_x m(x) e^{-i l.x},  Omega_p = (L/N)^2,
//              T = a^I, E = a^Q cos 2phi + a^U sin 2phi, B = -a^Q sin 2phi + a^U cos 2phi
//              (phi the angle of l from the l_x axis);
//   synthesis  m(x) = L^-2 sum_l a_l e^{i l.x}, with the inverse rotation
//              Q = E cos 2phi - B sin 2phi, U = E sin 2phi + B cos 2phi.
// These are exact inverses on the harmonic space, so the warm-started step
// a <- F [a + A (t - s)] of the driver is Algorithm 1 as printed.  Real maps
// keep the modes kx in [0, N/2) and every ky (the rest follow from Hermitian
// symmetry); the Nyquist row and column of the even grid are left out of the
// harmonic space, since a rotation by phi cannot keep real fields real there.
// Stored modes: a[b][f][kx N + ky], ky in FFT order.  The per-mode filter
// (S-bar + U)(S-bar + xi)^-1 takes the spectra of each mode, <|a_l|^2> =
// L^2 C_|l|, with T_h = alpha Omega_p (the pixel noise's Fourier power per
// unit area), as on the sphere.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "dm_fft.cuh"
#include "dm_internal.h"

namespace dmwf {

namespace {

// rc index of row y in column kx: the ring pairs (y, N - 1 - y) of the flat plan
__device__ __forceinline__ int64_t flat_rc(int b, int f, int kx, int mmax, int y, int N) {
  const int pair = y < N / 2 ? y : N - 1 - y, side = y < N / 2 ? 0 : 1;
  return ((((int64_t)b * 3 + f) * (mmax + 1) + kx) * (N / 2) + pair) * 2 + side;
}

// cos 2phi, sin 2phi of the mode (kx, ky signed), exactly from the integers
__device__ __forceinline__ void rot2(int kx, int ky, double &c, double &s) {
  const double x = (double)kx, y = (double)ky, r = x * x + y * y;
  if (r == 0.0) {
    c = 1.0;
    s = 0.0;
  } else {
    c = (x * x - y * y) / r;
    s = 2.0 * x * y / r;
  }
}

// One column kx of one RHS per block, the three fields as lanes y = 0, 1, 2
// (blockDim.x threads each).  Analysis: the column FFT of the row
// coefficients of each field, then per mode the E/B rotation, Omega_p and
// the epilogue (plain: out = a_l; DM step: out = F_level (out + a_l)).
__global__ void __launch_bounds__(768) k_flat_ana(const double2 *__restrict__ rc, double2 *out,
                                                  const double2 *__restrict__ twid, int N, int mmax, double omega,
                                                  int epilogue, const double *__restrict__ filt, int64_t nmodes,
                                                  const SolveState *__restrict__ state,
                                                  const double2 *__restrict__ src) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int kx = blockIdx.x, b = blockIdx.y, f = threadIdx.y, tx = threadIdx.x, T = blockDim.x;
  if (state != nullptr && state[b].done) return;  // uniform over the block
  const int slots = N + N / 32 + 1;
  double2 *tw = reinterpret_cast<double2 *>(sm_raw);
  double2 *buf = tw + (N - 1) + (size_t)f * slots;
  const int tflat = f * T + tx, nflat = 3 * T;
  for (int i = tflat; i < N - 1; i += nflat) tw[i] = twid[i];
  for (int y = tx; y < N; y += T) buf[spad(y)] = rc[flat_rc(b, f, kx, mmax, y, N)];
  __syncthreads();
  fft_dif(buf, N, tw);  // natural -> bit-reversed, block barrier at the end
  const int logN = 31 - __clz(N);
  const double2 *b0 = tw + (N - 1), *b1 = b0 + slots, *b2 = b1 + slots;
  for (int ky = tflat; ky < N; ky += nflat) {
    const int sl = spad(bitrev(ky, logN));
    const double2 g0 = b0[sl], g1 = b1[sl], g2 = b2[sl];
    const int kys = ky < N / 2 ? ky : ky - N;
    const bool keep = ky != N / 2;
    double c, s;
    rot2(kx, kys, c, s);
    const double w = keep ? omega : 0.0;
    double2 aT = make_double2(w * g0.x, w * g0.y);
    double2 aE = make_double2(w * (g1.x * c + g2.x * s), w * (g1.y * c + g2.y * s));
    double2 aB = make_double2(w * (-g1.x * s + g2.x * c), w * (-g1.y * s + g2.y * c));
    const int64_t mode = (int64_t)kx * N + ky;
    double2 *o = out + (int64_t)b * 3 * nmodes + mode;
    if (epilogue == ANA_FLAT_DRAW) {
      // the signal draw of a constrained realisation: the 2-D FFT of white
      // noise maps, unrotated and scaled by L/N (passed as omega), times the
      // per-mode Cholesky factor of the TE block and sqrt(BB) (filt holds the
      // spectra, [4][nmodes]: TT, EE, BB, TE), so that <a a^H> = L^2 S
      const double tt = filt[mode], ee = filt[nmodes + mode], bb = filt[2 * nmodes + mode],
                   te = filt[3 * nmodes + mode];
      const double l11 = sqrt(fmax(tt, 0.0));
      const double l21 = (l11 > 0.0) ? te / l11 : 0.0;
      const double l22 = sqrt(fmax(ee - l21 * l21, 0.0));
      const double lbb = sqrt(fmax(bb, 0.0));
      const double2 h0 = make_double2(w * g0.x, w * g0.y), h1 = make_double2(w * g1.x, w * g1.y),
                    h2 = make_double2(w * g2.x, w * g2.y);
      o[0] = make_double2(l11 * h0.x, l11 * h0.y);
      o[nmodes] = make_double2(l21 * h0.x + l22 * h1.x, l21 * h0.y + l22 * h1.y);
      o[2 * nmodes] = make_double2(lbb * h2.x, lbb * h2.y);
      continue;
    }
    if (epilogue == ANA_DM_STEP) {
      const double *cf = filt + ((int64_t)state[b].level * nmodes + mode) * 4;
      double2 t = cadd(o[0], aT), e = cadd(o[nmodes], aE), bb = cadd(o[2 * nmodes], aB);
      if (src != nullptr) {  // the harmonic source of a Jacobi refinement's W~ run, before the filter
        const double2 *g = src + (int64_t)b * 3 * nmodes + mode;
        t = cadd(t, g[0]);
        e = cadd(e, g[nmodes]);
        bb = cadd(bb, g[2 * nmodes]);
      }
      aT = make_double2(cf[0] * t.x + cf[1] * e.x, cf[0] * t.y + cf[1] * e.y);
      aE = make_double2(cf[1] * t.x + cf[2] * e.x, cf[1] * t.y + cf[2] * e.y);
      aB = make_double2(cf[3] * bb.x, cf[3] * bb.y);
    }
    o[0] = aT;
    o[nmodes] = aE;
    o[2 * nmodes] = aB;
  }
}

// Synthesis of one column kx of one RHS: the inverse rotation and L^-2 per
// mode, then the inverse column FFT (conj(FFT(conj(.)))) into the row
// coefficients of each field.
__global__ void __launch_bounds__(768) k_flat_syn(const double2 *__restrict__ alm, double2 *__restrict__ rc,
                                                  const double2 *__restrict__ twid, int N, int mmax,
                                                  double inv_area, int64_t nmodes,
                                                  const SolveState *__restrict__ state) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int kx = blockIdx.x, b = blockIdx.y, f = threadIdx.y, tx = threadIdx.x, T = blockDim.x;
  if (state != nullptr && state[b].done) return;
  const int slots = N + N / 32 + 1;
  double2 *tw = reinterpret_cast<double2 *>(sm_raw);
  double2 *b0 = tw + (N - 1), *b1 = b0 + slots, *b2 = b1 + slots;
  const int tflat = f * T + tx, nflat = 3 * T;
  for (int i = tflat; i < N - 1; i += nflat) tw[i] = twid[i];
  const double2 *ab = alm + (int64_t)b * 3 * nmodes + (int64_t)kx * N;
  for (int ky = tflat; ky < N; ky += nflat) {
    const double2 aT = ab[ky], aE = ab[nmodes + ky], aB = ab[2 * nmodes + ky];
    const int kys = ky < N / 2 ? ky : ky - N;
    const double w = (ky != N / 2) ? inv_area : 0.0;
    double c, s;
    rot2(kx, kys, c, s);
    const double2 hq = make_double2(aE.x * c - aB.x * s, aE.y * c - aB.y * s);
    const double2 hu = make_double2(aE.x * s + aB.x * c, aE.y * s + aB.y * c);
    b0[spad(ky)] = make_double2(w * aT.x, -w * aT.y);  // conjugated input
    b1[spad(ky)] = make_double2(w * hq.x, -w * hq.y);
    b2[spad(ky)] = make_double2(w * hu.x, -w * hu.y);
  }
  __syncthreads();
  double2 *buf = b0 + (size_t)f * slots;
  fft_dif(buf, N, tw);
  const int logN = 31 - __clz(N);
  for (int y = tx; y < N; y += T) {
    const double2 v = buf[spad(bitrev(y, logN))];
    rc[flat_rc(b, f, kx, mmax, y, N)] = make_double2(v.x, -v.y);
  }
}

size_t flat_smem(int N) { return sizeof(double2) * ((size_t)(N - 1) + 3 * (size_t)(N + N / 32 + 1)); }

}  // namespace

cudaError_t flat_synthesis(dm_plan *p, const double2 *alm, cudaStream_t st) {
  const int N = p->flatN;
  const size_t sm = flat_smem(N);
  cudaError_t e = dyn_smem_allow(k_flat_syn, sm);
  if (e) return e;
  const int T = std::min(256, std::max(32, N / 4));
  k_flat_syn<<<dim3(N / 2, p->batch), dim3(T, 3), sm, st>>>(alm, p->rc, p->twid, N, p->mmax,
                                                            1.0 / (p->flatL * p->flatL), p->nmodes,
                                                            p->state_active ? p->state : nullptr);
  return cudaGetLastError();
}

cudaError_t flat_analysis(dm_plan *p, int epilogue, double2 *out, cudaStream_t st, cudaEvent_t mid) {
  const int N = p->flatN;
  const size_t sm = flat_smem(N);
  cudaError_t e = dyn_smem_allow(k_flat_ana, sm);
  if (e) return e;
  const int T = std::min(256, std::max(32, N / 4));
  const double h = p->flatL / N;
  const bool draw = epilogue == ANA_FLAT_DRAW;
  const SolveState *stp = (epilogue == ANA_DM_STEP || (p->state_active && !draw)) ? p->state : nullptr;
  const double2 *src = (epilogue == ANA_DM_STEP && p->src_active) ? p->jsrc : nullptr;
  k_flat_ana<<<dim3(N / 2, p->batch), dim3(T, 3), sm, st>>>(p->rc, out, p->twid, N, p->mmax, draw ? h : h * h,
                                                            epilogue, draw ? p->cl : p->filt, p->nmodes, stp, src);
  if (mid) cudaEventRecord(mid, st);
  return cudaGetLastError();
}

// a_hat of a constrained realisation on a flat plan: white noise maps z,
// their row transforms (the ring kernels) and the draw epilogue of the column
// transforms, into ahat [batch][3][nmodes].  The maps pass through tmpmap.
cudaError_t flat_draw_signal(dm_plan *p, const uint64_t *seeds_dev, double2 *ahat, cudaStream_t st) {
  cudaError_t e = draw_white_maps(p, seeds_dev, p->tmpmap, st);
  const bool sa = p->state_active;
  p->state_active = false;
  if (!e) e = ring_stage(p, RING_FWD_MAP, p->tmpmap, nullptr, st);
  if (!e) e = flat_analysis(p, ANA_FLAT_DRAW, ahat, st, nullptr);
  p->state_active = sa;
  return e;
}

}  // namespace dmwf

using namespace dmwf;

extern "C" {

dm_status dm_plan_create_flat(int N, double L, int batch, dm_plan **out) {
  if (!out) return DM_EINVAL;
  *out = nullptr;
  if (N < 16 || N > 2048 || (N & (N - 1)) != 0 || !(L > 0.0) || !std::isfinite(L) || batch < 1 || batch > 4096)
    return DM_EINVAL;
  if ((int64_t)batch * 3 * N * N > INT32_MAX) return DM_EINVAL;
  dm_plan *p = new dm_plan();
  cudaGetDevice(&p->device);
  p->flat = true;
  p->flatN = N;
  p->flatL = L;
  p->batch = batch;
  p->npix = (int64_t)N * N;
  p->nrings = N;
  p->npairs = N / 2;
  p->mmax = p->lmax = N / 2 - 1;
  p->nmodes = p->nalm = (int64_t)(N / 2) * N;
  p->nchunk = 1;
  p->nslot = 1;
  cudaError_t e = build_tables_flat(p);
  if (e) {
    p->err = std::string("build flat tables: ") + cudaGetErrorString(e);
    fprintf(stderr, "dm_plan_create_flat: %s\n", p->err.c_str());
    dm_plan_destroy(p);
    return e == cudaErrorMemoryAllocation ? DM_ENOMEM : DM_ECUDA;
  }
  return plan_workspace(p, out);
}

dm_status dm_set_spectra_flat(dm_plan *p, const double *S) {
  if (!p || !S) return DM_EINVAL;
  if (!p->flat) {
    p->err = "dm_set_spectra_flat needs a flat-sky plan (dm_plan_create_flat)";
    return DM_EINVAL;
  }
  if (p->session) {
    p->err = "a solve is in progress on this plan";
    return DM_EBUSY;
  }
  const int N = p->flatN;
  const int64_t nn = (int64_t)N * N, nm = p->nmodes;
  std::vector<double> cl(4 * (size_t)nm);
  for (int kx = 0; kx < N / 2; ++kx)
    for (int ky = 0; ky < N; ++ky) {
      const int64_t src = (int64_t)ky * N + kx, dst = (int64_t)kx * N + ky;
      const double tt = S[src], ee = S[nn + src], bb = S[2 * nn + src], te = S[3 * nn + src];
      if (!std::isfinite(tt) || !std::isfinite(ee) || !std::isfinite(bb) || !std::isfinite(te) || tt < 0 ||
          ee < 0 || bb < 0 || te * te > tt * ee * (1.0 + 1e-12)) {
        p->err = "spectrum block not finite or not positive semi-definite at mode (ky " + std::to_string(ky) +
                 ", kx " + std::to_string(kx) + ")";
        return DM_EINVAL;
      }
      cl[dst] = tt;
      cl[nm + dst] = ee;
      cl[2 * nm + dst] = bb;
      cl[3 * nm + dst] = te;
    }
  cudaError_t e = cudaMemcpy(p->cl, cl.data(), sizeof(double) * 4 * nm, cudaMemcpyHostToDevice);
  if (!e) e = diag_tables_flat(p, cl);  // the end-of-solve diagnostics' per-mode tables
  if (e) {
    p->err = "upload spectra";
    return DM_ECUDA;
  }
  p->have_cl = true;
  if (p->have_noise) {
    if ((e = build_filters(p, 0, 0)) || (e = cudaDeviceSynchronize())) {
      p->err = "filters";
      return DM_ECUDA;
    }
  }
  return DM_OK;
}

dm_status dm_set_noise_flat(dm_plan *p, const double *sigma, const uint8_t *mask_t, const uint8_t *mask_p) {
  if (!p || !sigma) return DM_EINVAL;
  if (!p->flat) {
    p->err = "dm_set_noise_flat needs a flat-sky plan (dm_plan_create_flat)";
    return DM_EINVAL;
  }
  if (p->session) {
    p->err = "a solve is in progress on this plan";
    return DM_EBUSY;
  }
  const int64_t np = p->npix;
  double alpha = INFINITY;
  for (int64_t i = 0; i < np; ++i)
    for (int f = 0; f < 3; ++f) {
      const bool obs = f == 0 ? (!mask_t || mask_t[i]) : (!mask_p || mask_p[i]);
      if (!obs) continue;
      const double sg = sigma[f * np + i];
      if (!(sg > 0.0) || !std::isfinite(sg)) {
        p->err = "sigma must be finite and > 0 on observed components";
        return DM_EINVAL;
      }
      alpha = fmin(alpha, sg * sg);
    }
  if (!std::isfinite(alpha)) {
    p->err = "the masks leave no observed component";
    return DM_EINVAL;
  }
  std::vector<double> w(3 * (size_t)np);
  std::vector<uint8_t> any(np);
  for (int64_t i = 0; i < np; ++i) {
    const bool ot = !mask_t || mask_t[i], op = !mask_p || mask_p[i];
    any[i] = (ot || op) ? 1 : 0;
    for (int f = 0; f < 3; ++f) {
      const bool obs = f == 0 ? ot : op;
      const double sg = sigma[f * np + i];
      w[f * np + i] = obs ? alpha / (sg * sg) : 0.0;
    }
  }
  p->have_noise = false;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < p->batch && !e; ++b) {
    e = cudaMemcpy(p->w + (size_t)b * 3 * np, w.data(), sizeof(double) * 3 * np, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(p->sigma + (size_t)b * 3 * np, sigma, sizeof(double) * 3 * np, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(p->mask + (size_t)b * np, any.data(), np, cudaMemcpyHostToDevice);
    const double h = p->flatL / p->flatN;
    p->alpha[b] = alpha;
    p->t_h[b] = alpha * h * h;
  }
  if (e) {
    p->err = "upload noise";
    return DM_ECUDA;
  }
  p->have_noise = true;
  if (p->have_cl) {
    if ((e = build_filters(p, 0, 0)) || (e = cudaDeviceSynchronize())) {
      p->have_noise = false;
      p->err = "filters";
      return DM_ECUDA;
    }
  }
  return DM_OK;
}

}  // extern "C"
