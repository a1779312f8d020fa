// dm_control.cu -- device-side control of Algorithm 1 (Cauchy test, cooling
// levels, stopping), the data weighting w d of Eq. 9, and the random inputs of
// the constrained realisations of Section 2.2 (Eq. 19).
#include "dm_internal.h"

namespace dmwf {

// ----------------------------------------------------------------- control
__global__ void k_control_init(SolveState *st, const LevelDev *levs, int batch) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const LevelDev *lev = levs + b;
  SolveState s;
  s.level = 0;
  s.iter_in_level = 0;
  s.iters_total = 0;
  s.done = 0;
  s.first = 1;
  s.notconv = 0;
  s.cauchy = 1.0;
  for (int k = 0; k < DM_MAX_LEVELS; ++k) s.iters_per_level[k] = 0;
  if (lev->forced) {  // skip leading levels with no iterations
    while (s.level < lev->n_levels && lev->fixed_iters[s.level] == 0) ++s.level;
    if (s.level >= lev->n_levels) {
      s.level = lev->n_levels - 1;
      s.done = 1;
    }
  }
  st[b] = s;
}

// One block per RHS: ||s_i - s_{i-1}||^2 and ||s_i||^2 from the per-ring
// partials in a fixed order, then the stopping rule of Algorithm 1:
// a level ends when the Cauchy ratio falls below eps_k (or after its fixed
// count); the next level lowers xi (lambda) and the last level ends the run.
__global__ void k_control_step(SolveState *st, const LevelDev *__restrict__ levs, const double *__restrict__ norms,
                               int nrings, int *clev) {
  const int b = blockIdx.x;
  if (st[b].done) return;
  // the filtered step of this iteration ran at st[b].level (mixed mode: its c is formed)
  if (clev != nullptr && threadIdx.x == 0) clev[b] = st[b].level;
  const LevelDev *lev = levs + b;
  __shared__ double r0[256], r1[256];
  double dd = 0.0, ss = 0.0;
  const int n = 3 * nrings;
  const double *nb = norms + (int64_t)b * n * 2;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    dd += nb[2 * i];
    ss += nb[2 * i + 1];
  }
  r0[threadIdx.x] = dd;
  r1[threadIdx.x] = ss;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      r0[threadIdx.x] += r0[threadIdx.x + s];
      r1[threadIdx.x] += r1[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  SolveState s = st[b];
  double cauchy = (r1[0] > 0.0) ? sqrt(r0[0] / r1[0]) : 0.0;
  s.cauchy = cauchy;
  s.first = 0;
  s.iters_total += 1;
  s.iter_in_level += 1;
  s.iters_per_level[s.level] += 1;
  bool stop;
  if (lev->forced)
    stop = s.iter_in_level >= lev->fixed_iters[s.level];
  else
    stop = cauchy < lev->eps[s.level];
  if (stop) {
    int k = s.level + 1;
    if (lev->forced)
      while (k < lev->n_levels && lev->fixed_iters[k] == 0) ++k;
    if (k >= lev->n_levels) {
      s.done = 1;
    } else {
      s.level = k;
      s.iter_in_level = 0;
    }
  }
  if (!s.done && !lev->forced && s.iters_total >= lev->max_iter) {
    s.done = 1;
    s.notconv = 1;
  }
  st[b] = s;
}

cudaError_t control_init(dm_plan *p, cudaStream_t st) {
  k_control_init<<<(p->batch + 127) / 128, 128, 0, st>>>(p->state, p->lev, p->batch);
  return cudaGetLastError();
}

cudaError_t control_step(dm_plan *p, cudaStream_t st) {
  k_control_step<<<p->batch, 256, 0, st>>>(p->state, p->lev, p->norms, p->nrings,
                                           p->anchor_active ? p->clev : nullptr);
  return cudaGetLastError();
}

// w d on observed pixels (masked pixels of d are ignored, even if not finite)
__global__ void k_wd(const double *__restrict__ d, const double *__restrict__ w, double *__restrict__ wd,
                     int64_t n3, int batch) {
  int64_t total = n3 * batch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    double ww = w[i];
    wd[i] = (ww > 0.0) ? ww * d[i] : 0.0;
  }
}

// FP32 iteration maps: w32 = w and wd32 = w d, both rounded once from FP64
__global__ void k_wd32(const double *__restrict__ d, const double *__restrict__ w, float *__restrict__ w32,
                       float *__restrict__ wd32, int64_t n3, int batch) {
  int64_t total = n3 * batch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    double ww = w[i];
    wd32[i] = (ww > 0.0) ? (float)(ww * d[i]) : 0.0f;
    w32[i] = (float)ww;
  }
}

cudaError_t prepare_wd(dm_plan *p, const double *d, cudaStream_t st) {
  k_wd<<<2048, 256, 0, st>>>(d, p->w, p->wd, 3 * p->npix, p->batch);
  if (p->prec != DM_FP64) k_wd32<<<2048, 256, 0, st>>>(d, p->w, p->w32, p->wd32, 3 * p->npix, p->batch);
  return cudaGetLastError();
}

__global__ void k_anchor_resid(const double *__restrict__ d, const double *__restrict__ s_hi,
                               const double *__restrict__ w, double *__restrict__ r, float *__restrict__ shi32,
                               int64_t n3, int batch) {
  int64_t total = n3 * batch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const double ww = w[i];
    if (s_hi == nullptr) {  // t_0 - s_0 = d on observed pixels (Algorithm 1 initial guess)
      r[i] = (ww > 0.0) ? d[i] : 0.0;
      shi32[i] = 0.0f;
    } else {
      const double sh = s_hi[i];
      r[i] = (ww > 0.0) ? ww * (d[i] - sh) : 0.0;
      shi32[i] = (float)sh;
    }
  }
}

cudaError_t anchor_residual(dm_plan *p, const double *d, const double *s_hi, cudaStream_t st) {
  k_anchor_resid<<<2048, 256, 0, st>>>(d, s_hi, p->w, p->rhi, p->shi32, 3 * p->npix, p->batch);
  return cudaGetLastError();
}

// r = w d - w s_hi from the stored w d (FP64), shi32 = s_hi in FP32
__global__ void k_anchor_resid_wd(const double *__restrict__ wd, const double *__restrict__ s_hi,
                                  const double *__restrict__ w, double *__restrict__ r, float *__restrict__ shi32,
                                  int64_t n3, int batch) {
  int64_t total = n3 * batch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const double sh = s_hi[i];
    r[i] = wd[i] - w[i] * sh;
    shi32[i] = (float)sh;
  }
}

cudaError_t anchor_residual_wd(dm_plan *p, const double *s_hi, cudaStream_t st) {
  k_anchor_resid_wd<<<2048, 256, 0, st>>>(p->wd, s_hi, p->w, p->rhi, p->shi32, 3 * p->npix, p->batch);
  return cudaGetLastError();
}

__global__ void k_f2d(const float *__restrict__ in, double *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

cudaError_t copy_s32_to_user(dm_plan *p, double *s_out, cudaStream_t st) {
  k_f2d<<<2048, 256, 0, st>>>(p->s32, s_out, 3 * p->npix * p->batch);
  return cudaGetLastError();
}

__global__ void k_axpy(int64_t n, const double *__restrict__ x, double a, double *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

cudaError_t axpy_maps(int64_t n, const double *x, double a, double *y, cudaStream_t st) {
  k_axpy<<<2048, 256, 0, st>>>(n, x, a, y);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the key bumped by the Weyl
// constants (0x9E3779B9, 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Two unit normals: uniforms u = ((w_hi >> 5) 2^26 + (w_lo >> 6) + 1/2) 2^-53 from
// word pairs (0,1) and (2,3), then Box-Muller.
__device__ __forceinline__ double2 gauss2(uint64_t seed, unsigned c0, unsigned c1, unsigned c2) {
  uint4 o = philox10(make_uint4(c0, c1, c2, 0u), make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const double u1 = ((double)((((uint64_t)(o.x >> 5)) << 26) | (o.y >> 6)) + 0.5) * 0x1.0p-53;
  const double u2 = ((double)((((uint64_t)(o.z >> 5)) << 26) | (o.w >> 6)) + 0.5) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return make_double2(r * cs, r * sn);
}

// ahat = L z per (l, m): L = chol([[TT, TE], [TE, EE]]), sqrt(BB) for B;
// m = 0 real at full variance, m > 0 re and im at half variance.
__global__ void k_draw_signal(const uint64_t *__restrict__ seeds, const double *__restrict__ cl, double2 *ahat,
                              int lmax, int64_t nalm) {
  const int b = blockIdx.y, m = blockIdx.z;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const int64_t i = (int64_t)m * (2 * lmax + 1 - m) / 2 + l;
  const uint64_t seed = seeds[b];
  double2 zt = gauss2(seed, (unsigned)i, 0u, 0u);
  double2 ze = gauss2(seed, (unsigned)i, 1u, 0u);
  double2 zb = gauss2(seed, (unsigned)i, 2u, 0u);
  const double tt = cl[l], ee = cl[(lmax + 1) + l], bb = cl[2 * (lmax + 1) + l], te = cl[3 * (lmax + 1) + l];
  const double l11 = sqrt(fmax(tt, 0.0));
  const double l21 = (l11 > 0.0) ? te / l11 : 0.0;
  const double l22 = sqrt(fmax(ee - l21 * l21, 0.0));
  const double lbb = sqrt(fmax(bb, 0.0));
  const double sc = (m == 0) ? 1.0 : sqrt(0.5);
  const double si = (m == 0) ? 0.0 : sc;
  double2 *o = ahat + (int64_t)b * 3 * nalm + i;
  o[0] = make_double2(sc * l11 * zt.x, si * l11 * zt.y);
  o[nalm] = make_double2(sc * (l21 * zt.x + l22 * ze.x), si * (l21 * zt.y + l22 * ze.y));
  o[2 * nalm] = make_double2(sc * lbb * zb.x, si * lbb * zb.y);
}

cudaError_t draw_signal(dm_plan *p, const uint64_t *seeds_dev, double2 *ahat, cudaStream_t st) {
  dim3 g((p->lmax + 1 + 127) / 128, p->batch, p->mmax + 1);
  k_draw_signal<<<g, 128, 0, st>>>(seeds_dev, p->cl, ahat, p->lmax, p->nalm);
  return cudaGetLastError();
}

// dhat = shat + sigma z on observed pixels, 0 on masked ones; with w given
// (flat plans, whose temperature and polarisation masks differ) a component
// is observed where its weight is positive.
__global__ void k_draw_noise(const uint64_t *__restrict__ seeds, const double *__restrict__ sigma,
                             const uint8_t *__restrict__ mask, const double *__restrict__ w,
                             const double *__restrict__ shat, double *dhat, int64_t npix) {
  const int b = blockIdx.y;
  const uint64_t seed = seeds[b];
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
    double2 z01 = gauss2(seed, (unsigned)p, 0u, 1u);
    double2 z2 = gauss2(seed, (unsigned)p, 1u, 1u);
    const bool obs = (mask == nullptr) || mask[(int64_t)b * npix + p];
    const int64_t o = (int64_t)b * 3 * npix + p;
    const double zz[3] = {z01.x, z01.y, z2.x};
    for (int f = 0; f < 3; ++f) {
      const int64_t i = o + f * npix;
      const bool ob = (w != nullptr) ? (w[i] > 0.0) : obs;
      dhat[i] = ob ? shat[i] + sigma[i] * zz[f] : 0.0;
    }
  }
}

// Correlated noise (dm_set_noise_cov): n = D z per pixel with the same unit
// normals as the diagonal draw and the per-pixel draw matrix D; a component
// is observed where its weight diag(W) is positive.
__global__ void k_draw_noise_cov(const uint64_t *__restrict__ seeds, const double *__restrict__ D,
                                 const double *__restrict__ w, const double *__restrict__ shat, double *dhat,
                                 int64_t npix) {
  const int b = blockIdx.y;
  const uint64_t seed = seeds[b];
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
    const double2 z01 = gauss2(seed, (unsigned)p, 0u, 1u);
    const double2 z2 = gauss2(seed, (unsigned)p, 1u, 1u);
    const double *Dp = D + 9 * p;
    const int64_t o = (int64_t)b * 3 * npix + p;
    for (int f = 0; f < 3; ++f) {
      const double n = Dp[3 * f] * z01.x + Dp[3 * f + 1] * z01.y + Dp[3 * f + 2] * z2.x;
      const int64_t i = o + f * npix;
      dhat[i] = (w[i] > 0.0) ? shat[i] + n : 0.0;
    }
  }
}

// Unit white-noise maps z [batch][3][npix] for the flat constrained-realisation
// signal draw: per RHS seed and pixel p, the pair (p, 0, 2) gives the I and Q
// values and the first normal of (p, 1, 2) the U value (the third counter word
// is 0 for the sphere's signal draw and 1 for the noise draws).
__global__ void k_white_maps(const uint64_t *__restrict__ seeds, double *__restrict__ z, int64_t npix) {
  const int b = blockIdx.y;
  const uint64_t seed = seeds[b];
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
    const double2 z01 = gauss2(seed, (unsigned)p, 0u, 2u);
    const double2 z2 = gauss2(seed, (unsigned)p, 1u, 2u);
    const int64_t o = (int64_t)b * 3 * npix + p;
    z[o] = z01.x;
    z[o + npix] = z01.y;
    z[o + 2 * npix] = z2.x;
  }
}

cudaError_t draw_white_maps(dm_plan *p, const uint64_t *seeds_dev, double *z, cudaStream_t st) {
  k_white_maps<<<dim3(256, p->batch), 256, 0, st>>>(seeds_dev, z, p->npix);
  return cudaGetLastError();
}

cudaError_t draw_noise_add(dm_plan *p, const uint64_t *seeds_dev, const double *shat, double *dhat,
                           cudaStream_t st) {
  dim3 g(1024, p->batch);
  if (p->cov)
    k_draw_noise_cov<<<g, 256, 0, st>>>(seeds_dev, p->covdraw, p->w, shat, dhat, p->npix);
  else
    k_draw_noise<<<g, 256, 0, st>>>(seeds_dev, p->sigma, p->mask, p->flat ? p->w : nullptr, shat, dhat, p->npix);
  return cudaGetLastError();
}

// ----------------------------------------------------------- peak probe
template <typename T>
__global__ void k_fma_chain(T *out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
static double time_fma(int blocks, int iters) {
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * 256)) return -1.0;
  k_fma_chain<T><<<blocks, 256>>>(out, 4, (T)0.999, (T)0.001);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0);
    k_fma_chain<T><<<blocks, 256>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  double flops = 2.0 * 64.0 * (double)blocks * 256.0 * (double)iters;
  return flops / (best * 1e-3) / 1e12;
}

}  // namespace dmwf

extern "C" dm_status dm_measure_alu_peaks(double *fp64_tflops, double *fp32_tflops) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (fp64_tflops) *fp64_tflops = dmwf::time_fma<double>(sms * 4, 1024);
  if (fp32_tflops) *fp32_tflops = dmwf::time_fma<float>(sms * 8, 8192);
  return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ECUDA;
}
