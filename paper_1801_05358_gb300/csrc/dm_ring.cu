// dm_ring.cu -- the pixel-space half of a dual messenger iteration, one CTA per
// (ring, Stokes component, RHS):
//   inverse ring DFT  F_m -> s           (synthesis F, Algorithm 1)
//   Cauchy partials   ||s - s_prev||^2, ||s||^2   (stopping rule, Section 3.2)
//   messenger update  t - s = w (d - s)           (Eq. 9, diagonal N)
//   forward ring DFT  (t - s) -> G_m     (analysis F^dagger, Algorithm 1)
// A real ring of n pixels is packed as a complex sequence of h = n/2 points.
//
// Ring coefficients live in rc[b][f][m][pair][side] (double2): the Legendre
// kernels read a ring pair (north, south) as one 32-byte item.
#include "dm_fft.cuh"
#include "dm_internal.h"

namespace dmwf {

__device__ __forceinline__ int64_t rc_index(int b, int f, int m, int mmax, int pair, int npairs, int side) {
  return ((((int64_t)b * 3 + f) * (mmax + 1) + m) * npairs + pair) * 2 + side;
}

template <int MODE>
__global__ void __launch_bounds__(256) k_ring(const RingDev *__restrict__ rings, const double2 *__restrict__ phase,
                                              const double2 *__restrict__ bhat, const double2 *__restrict__ twid,
                                              int Mtab, double2 *__restrict__ rc, int mmax, int npairs, int64_t npix,
                                              int nrings, const double *__restrict__ in_map, double *out_map,
                                              const double *__restrict__ w, const double *__restrict__ wd,
                                              double *__restrict__ norms, const SolveState *__restrict__ state) {
  extern __shared__ double2 sm[];
  const int r = blockIdx.x, f = blockIdx.y, b = blockIdx.z;
  if ((MODE == RING_ITER || MODE == RING_INIT) && state != nullptr && state[b].done) return;
  const RingDev R = rings[r];
  const int n = R.n, h = R.h;
  const int64_t n2 = 2LL * n;
  const double2 *ph = phase + R.ph_off;  // e^{-i pi q / n}, q < 2n
  double2 *buf = sm;                     // FFT work area, M entries
  double2 *cb = sm + Mtab;               // h + 1 <= Mtab + 1 spectrum entries
  const int64_t moff = ((int64_t)b * 3 + f) * npix + R.start;

  if (MODE == RING_INV_MAP || MODE == RING_ITER) {
    // Fold F_m (m = -mmax..mmax, F_{-m} = conj F_m) into C_k = sum_{m = k mod n} F_m e^{i m phi0}, k <= h.
    for (int k = threadIdx.x; k <= h; k += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      for (int m = k; m <= mmax; m += n) {
        double2 F = rc[rc_index(b, f, m, mmax, R.pair, npairs, R.side)];
        double2 e = cconj(ph[((int64_t)m * R.shift) % n2]);
        acc = cadd(acc, cmul(F, e));
      }
      for (int m = n - k; m <= mmax; m += n) {
        if (m < 1) continue;
        double2 F = rc[rc_index(b, f, m, mmax, R.pair, npairs, R.side)];
        double2 e = cconj(ph[((int64_t)m * R.shift) % n2]);
        acc = cadd(acc, cconj(cmul(F, e)));
      }
      cb[k] = acc;
    }
    __syncthreads();
    // Pack for the half-length inverse: Z_k = E_k + i O_k with
    // E_k = C_k + conj(C_{h-k}),  O_k = (C_k - conj(C_{h-k})) e^{2 pi i k/n}; stored conjugated
    // so that a forward FFT followed by conjugation gives the inverse.
    for (int k = threadIdx.x; k < h; k += blockDim.x) {
      double2 ck = cb[k], cc = cconj(cb[h - k]);
      double2 E = cadd(ck, cc);
      double2 O = cmul(csub(ck, cc), cconj(ph[2 * k]));
      double2 Z = make_double2(E.x - O.y, E.y + O.x);
      buf[k] = cconj(Z);
    }
    __syncthreads();
    dft_forward(buf, h, R.M, R.bluestein, ph, bhat + (R.bh_off < 0 ? 0 : R.bh_off), twid, Mtab);
    // z_j = conj(buf_j) = s_{2j} + i s_{2j+1}
    if (MODE == RING_INV_MAP) {
      for (int j = threadIdx.x; j < h; j += blockDim.x) {
        double2 z = buf[j];
        out_map[moff + 2 * j] = z.x;
        out_map[moff + 2 * j + 1] = -z.y;
      }
      return;
    }
    // RING_ITER: Cauchy partials, store s, form t - s = w d - w s and pack it.
    double dd = 0.0, ss = 0.0;
    const int64_t wo = (int64_t)f * npix + R.start;
    for (int j = threadIdx.x; j < h; j += blockDim.x) {
      double2 z = buf[j];
      double s0 = z.x, s1 = -z.y;
      double o0 = out_map[moff + 2 * j], o1 = out_map[moff + 2 * j + 1];
      dd += (s0 - o0) * (s0 - o0) + (s1 - o1) * (s1 - o1);
      ss += s0 * s0 + s1 * s1;
      out_map[moff + 2 * j] = s0;
      out_map[moff + 2 * j + 1] = s1;
      double r0 = wd[moff + 2 * j] - w[wo + 2 * j] * s0;
      double r1 = wd[moff + 2 * j + 1] - w[wo + 2 * j + 1] * s1;
      buf[j] = make_double2(r0, r1);
    }
    // block reduction of (dd, ss)
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
      dd += __shfl_down_sync(0xffffffffu, dd, o);
      ss += __shfl_down_sync(0xffffffffu, ss, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = dd;
      red[1][threadIdx.x >> 5] = ss;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, c = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
        a += red[0][i];
        c += red[1][i];
      }
      int64_t no = (((int64_t)b * 3 + f) * nrings + r) * 2;
      norms[no] = a;
      norms[no + 1] = c;
    }
  } else {
    // forward only: load the real ring (RING_INIT: t_0 - s_0 = d on observed pixels)
    const int64_t wo = (int64_t)f * npix + R.start;
    for (int j = threadIdx.x; j < h; j += blockDim.x) {
      double x0 = in_map[moff + 2 * j], x1 = in_map[moff + 2 * j + 1];
      if (MODE == RING_INIT) {
        x0 = (w[wo + 2 * j] > 0.0) ? x0 : 0.0;
        x1 = (w[wo + 2 * j + 1] > 0.0) ? x1 : 0.0;
      }
      buf[j] = make_double2(x0, x1);
    }
  }
  __syncthreads();
  // forward: Z = FFT_h(z), X_k = E_k + e^{-2 pi i k/n} O_k, k = 0..h
  dft_forward(buf, h, R.M, R.bluestein, ph, bhat + (R.bh_off < 0 ? 0 : R.bh_off), twid, Mtab);
  for (int k = threadIdx.x; k <= h; k += blockDim.x) {
    double2 zk = buf[k == h ? 0 : k], zc = cconj(buf[k == 0 ? 0 : h - k]);
    if (k == h) zc = cconj(buf[0]);
    double2 E = make_double2(0.5 * (zk.x + zc.x), 0.5 * (zk.y + zc.y));
    double2 D = csub(zk, zc);                          // = 2i O_k
    double2 O = make_double2(0.5 * D.y, -0.5 * D.x);   // D / (2i)
    cb[k] = cadd(E, cmul(O, ph[2 * k]));
  }
  __syncthreads();
  for (int m = threadIdx.x; m <= mmax; m += blockDim.x) {
    int q = m % n;
    double2 X = (q <= h) ? cb[q] : cconj(cb[n - q]);
    rc[rc_index(b, f, m, mmax, R.pair, npairs, R.side)] = cmul(X, ph[((int64_t)m * R.shift) % n2]);
  }
}

cudaError_t ring_stage(dm_plan *p, int mode, const double *in_map, double *out_map, cudaStream_t st) {
  dim3 grid(p->nrings, 3, p->batch);
  size_t smem = sizeof(double2) * (2 * (size_t)p->fft_M_max + 1);
  const SolveState *stp = p->state;
  switch (mode) {
    case RING_FWD_MAP:
      cudaFuncSetAttribute(k_ring<RING_FWD_MAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_ring<RING_FWD_MAP><<<grid, 256, smem, st>>>(p->rings, p->phase, p->bhat, p->twid, p->fft_M_max, p->rc,
                                                    p->mmax, p->npairs, p->npix, p->nrings, in_map, out_map, p->w,
                                                    p->wd, p->norms, nullptr);
      break;
    case RING_INV_MAP:
      cudaFuncSetAttribute(k_ring<RING_INV_MAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_ring<RING_INV_MAP><<<grid, 256, smem, st>>>(p->rings, p->phase, p->bhat, p->twid, p->fft_M_max, p->rc,
                                                    p->mmax, p->npairs, p->npix, p->nrings, in_map, out_map, p->w,
                                                    p->wd, p->norms, nullptr);
      break;
    case RING_ITER:
      cudaFuncSetAttribute(k_ring<RING_ITER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_ring<RING_ITER><<<grid, 256, smem, st>>>(p->rings, p->phase, p->bhat, p->twid, p->fft_M_max, p->rc,
                                                 p->mmax, p->npairs, p->npix, p->nrings, in_map, out_map, p->w,
                                                 p->wd, p->norms, stp);
      break;
    case RING_INIT:
      cudaFuncSetAttribute(k_ring<RING_INIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_ring<RING_INIT><<<grid, 256, smem, st>>>(p->rings, p->phase, p->bhat, p->twid, p->fft_M_max, p->rc,
                                                 p->mmax, p->npairs, p->npix, p->nrings, in_map, out_map, p->w,
                                                 p->wd, p->norms, stp);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// public layout rc_pub[b][f][ring][m] <-> internal rc[b][f][m][pair][side]
__global__ void k_rc_pub(const RingDev *rings, double2 *rc, double2 *pub, int mmax, int npairs, int nrings,
                         int to_public) {
  int r = blockIdx.x, f = blockIdx.y, b = blockIdx.z;
  RingDev R = rings[r];
  for (int m = threadIdx.x; m <= mmax; m += blockDim.x) {
    int64_t pi = (((int64_t)b * 3 + f) * nrings + r) * (mmax + 1) + m;
    int64_t ii = rc_index(b, f, m, mmax, R.pair, npairs, R.side);
    if (to_public)
      pub[pi] = rc[ii];
    else
      rc[ii] = pub[pi];
  }
}

cudaError_t rc_to_public(dm_plan *p, double2 *pub, cudaStream_t st) {
  k_rc_pub<<<dim3(p->nrings, 3, p->batch), 128, 0, st>>>(p->rings, p->rc, pub, p->mmax, p->npairs, p->nrings, 1);
  return cudaGetLastError();
}
cudaError_t rc_from_public(dm_plan *p, const double2 *pub, cudaStream_t st) {
  k_rc_pub<<<dim3(p->nrings, 3, p->batch), 128, 0, st>>>(p->rings, p->rc, const_cast<double2 *>(pub), p->mmax,
                                                          p->npairs, p->nrings, 0);
  return cudaGetLastError();
}

}  // namespace dmwf
