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
#include <algorithm>

#include "dm_fft.cuh"
#include "dm_internal.h"

namespace dmwf {

__device__ __forceinline__ int64_t rc_index(int b, int f, int m, int mmax, int pair, int npairs, int side) {
  return ((((int64_t)b * 3 + f) * (mmax + 1) + m) * npairs + pair) * 2 + side;
}

// R: real type of the FFT and of the iteration maps (double or float); C its
// complex type.  User maps (in_map, out_user) are always FP64.
// Block = (blockDim.x threads per lane) x (blockDim.y lanes); the lanes are
// consecutive (RHS, Stokes) pairs of the same ring, so every lane runs the
// same FFT plan in lockstep and the block-wide barriers of the FFT stages are
// shared by blockDim.y transforms.  Lanes of finished RHS compute in shared
// memory but write nothing.
template <typename R, typename C, int MODE>
__global__ void __launch_bounds__(512) k_ring(const RingDev *__restrict__ rings, const C *__restrict__ phase,
                                              const C *__restrict__ bhat, const C *__restrict__ twid, int Mtab,
                                              int lane_words, int nlanes, C *__restrict__ rc, int mmax, int npairs,
                                              int64_t npix, int nrings, const double *__restrict__ in_map,
                                              double *__restrict__ out_user, R *s_state, const R *__restrict__ w,
                                              const R *__restrict__ wd, double *__restrict__ norms,
                                              const SolveState *__restrict__ state,
                                              const R *__restrict__ s_anchor) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ double red[8][16][2];
  const int r = blockIdx.x;
  const int g = threadIdx.y;
  const int L = blockIdx.y * blockDim.y + g;
  const bool valid = L < nlanes;
  const int b = valid ? L / 3 : 0, f = valid ? L % 3 : 0;
  bool live = valid;
  if ((MODE == RING_ITER || MODE == RING_INIT) && state != nullptr && valid && state[b].done) live = false;
  if (!__syncthreads_or(live)) return;
  C *sm = reinterpret_cast<C *>(sm_raw) + (size_t)g * lane_words;
  const RingDev Rg = rings[r];
  const int n = Rg.n, h = Rg.h;
  const int64_t n2 = 2LL * n;
  const C *ph = phase + Rg.ph_off;  // e^{-i pi q / n}, q < 2n
  C *buf = sm;                      // FFT work area, M entries
  C *cb = sm + Rg.M;                // h + 1 spectrum entries
  const int64_t moff = ((int64_t)b * 3 + f) * npix + Rg.start;
  const C *bh = bhat + (Rg.bh_off < 0 ? 0 : Rg.bh_off);
  const int tx = threadIdx.x, nt = blockDim.x;

  if (MODE == RING_INV_MAP || MODE == RING_ITER) {
    // Fold F_m (m = -mmax..mmax, F_{-m} = conj F_m) into C_k = sum_{m = k mod n} F_m e^{i m phi0}, k <= h.
    for (int k = tx; k <= h; k += nt) {
      C acc;
      acc.x = 0;
      acc.y = 0;
      for (int m = k; m <= mmax; m += n) {
        C F = rc[rc_index(b, f, m, mmax, Rg.pair, npairs, Rg.side)];
        C e = cconj(ph[((int64_t)m * Rg.shift) % n2]);
        acc = cadd(acc, cmul(F, e));
      }
      for (int m = n - k; m <= mmax; m += n) {
        if (m < 1) continue;
        C F = rc[rc_index(b, f, m, mmax, Rg.pair, npairs, Rg.side)];
        C e = cconj(ph[((int64_t)m * Rg.shift) % n2]);
        acc = cadd(acc, cconj(cmul(F, e)));
      }
      cb[k] = acc;
    }
    __syncthreads();
    // Pack for the half-length inverse: Z_k = E_k + i O_k with
    // E_k = C_k + conj(C_{h-k}),  O_k = (C_k - conj(C_{h-k})) e^{2 pi i k/n}; stored conjugated
    // so that a forward FFT followed by conjugation gives the inverse.
    for (int k = tx; k < h; k += nt) {
      C ck = cb[k], cc = cconj(cb[h - k]);
      C E = cadd(ck, cc);
      C O = cmul(csub(ck, cc), cconj(ph[2 * k]));
      C Z;
      Z.x = E.x - O.y;
      Z.y = E.y + O.x;
      buf[k] = cconj(Z);
    }
    __syncthreads();
    dft_forward(buf, h, Rg.M, Rg.bluestein, ph, bh, twid, Mtab);
    // z_j = conj(buf_j) = s_{2j} + i s_{2j+1}
    if (MODE == RING_INV_MAP) {
      if (live)
        for (int j = tx; j < h; j += nt) {
          C z = buf[j];
          out_user[moff + 2 * j] = (double)z.x;
          out_user[moff + 2 * j + 1] = -(double)z.y;
        }
      return;
    }
    // RING_ITER: Cauchy partials (FP64), store s, form t - s = w d - w s and pack it.
    // With an anchor (mixed precision) the state is Y e, s = s_anchor + Y e, and
    // the data part w (d - s_anchor) is carried in FP64 by the anchor: r = -w Y e.
    double dd = 0.0, ss = 0.0;
    const int64_t wo = moff;  // per-RHS weights share the map layout
    for (int j = tx; j < h; j += nt) {
      C z = buf[j];
      R s0 = z.x, s1 = -z.y;
      C rr;
      if (live) {
        R o0 = s_state[moff + 2 * j], o1 = s_state[moff + 2 * j + 1];
        double d0 = (double)s0 - (double)o0, d1 = (double)s1 - (double)o1;
        dd += d0 * d0 + d1 * d1;
        s_state[moff + 2 * j] = s0;
        s_state[moff + 2 * j + 1] = s1;
        if (s_anchor != nullptr) {
          const double f0 = (double)s_anchor[moff + 2 * j] + (double)s0;
          const double f1 = (double)s_anchor[moff + 2 * j + 1] + (double)s1;
          ss += f0 * f0 + f1 * f1;
          rr.x = -w[wo + 2 * j] * s0;
          rr.y = -w[wo + 2 * j + 1] * s1;
        } else {
          ss += (double)s0 * (double)s0 + (double)s1 * (double)s1;
          rr.x = wd[moff + 2 * j] - w[wo + 2 * j] * s0;
          rr.y = wd[moff + 2 * j + 1] - w[wo + 2 * j + 1] * s1;
        }
      } else {
        rr.x = 0;
        rr.y = 0;
      }
      buf[j] = rr;
    }
    // per-lane reduction of (dd, ss): warps never straddle lanes (blockDim.x % 32 == 0)
    for (int o = 16; o > 0; o >>= 1) {
      dd += __shfl_down_sync(0xffffffffu, dd, o);
      ss += __shfl_down_sync(0xffffffffu, ss, o);
    }
    if ((tx & 31) == 0) {
      red[g][tx >> 5][0] = dd;
      red[g][tx >> 5][1] = ss;
    }
    __syncthreads();
    if (tx == 0 && live) {
      double a = 0.0, c = 0.0;
      for (int i = 0; i < (nt >> 5); ++i) {
        a += red[g][i][0];
        c += red[g][i][1];
      }
      int64_t no = (((int64_t)b * 3 + f) * nrings + r) * 2;
      norms[no] = a;
      norms[no + 1] = c;
    }
  } else {
    // forward only: load the real ring (RING_INIT: t_0 - s_0 = d on observed pixels)
    const int64_t wo = moff;
    for (int j = tx; j < h; j += nt) {
      double x0 = 0.0, x1 = 0.0;
      if (valid) {
        x0 = in_map[moff + 2 * j];
        x1 = in_map[moff + 2 * j + 1];
        if (MODE == RING_INIT) {
          x0 = (w[wo + 2 * j] > (R)0) ? x0 : 0.0;
          x1 = (w[wo + 2 * j + 1] > (R)0) ? x1 : 0.0;
        }
      }
      C v;
      v.x = (R)x0;
      v.y = (R)x1;
      buf[j] = v;
    }
  }
  __syncthreads();
  // forward: Z = FFT_h(z), X_k = E_k + e^{-2 pi i k/n} O_k, k = 0..h
  dft_forward(buf, h, Rg.M, Rg.bluestein, ph, bh, twid, Mtab);
  const R half = (R)0.5;
  for (int k = tx; k <= h; k += nt) {
    C zk = buf[k == h ? 0 : k], zc = cconj(buf[k == 0 ? 0 : h - k]);
    if (k == h) zc = cconj(buf[0]);
    C E, O;
    E.x = half * (zk.x + zc.x);
    E.y = half * (zk.y + zc.y);
    C D = csub(zk, zc);  // = 2i O_k
    O.x = half * D.y;
    O.y = -half * D.x;   // D / (2i)
    cb[k] = cadd(E, cmul(O, ph[2 * k]));
  }
  __syncthreads();
  if (!live) return;
  for (int m = tx; m <= mmax; m += nt) {
    int q = m % n;
    C X = (q <= h) ? cb[q] : cconj(cb[n - q]);
    rc[rc_index(b, f, m, mmax, Rg.pair, npairs, Rg.side)] = cmul(X, ph[((int64_t)m * Rg.shift) % n2]);
  }
}

template <typename R, typename C, int MODE>
static cudaError_t launch_ring(dm_plan *p, const C *phase, const C *bhat, const C *twid, C *rc,
                               const double *in_map, double *out_user, R *s_state, const R *w, const R *wd,
                               cudaStream_t st, const R *s_anchor = nullptr) {
  int hmax = 0;
  for (const RingDev &Rg : p->rings_h) hmax = Rg.h > hmax ? Rg.h : hmax;
  int lane_words = 0;
  for (const RingDev &Rg : p->rings_h) lane_words = std::max(lane_words, Rg.M + Rg.h + 1);
  const int nlanes = 3 * p->batch;
  const size_t lane_bytes = sizeof(C) * (size_t)lane_words;
  int G = (int)std::max<size_t>(1, std::min<size_t>(4, (100u << 10) / lane_bytes));
  G = std::min(G, nlanes);
  const int T = 128;
  dim3 grid(p->nrings, (nlanes + G - 1) / G);
  dim3 block(T, G);
  size_t smem = lane_bytes * G;
  const SolveState *stp = (MODE == RING_ITER || MODE == RING_INIT) ? p->state : nullptr;
  cudaFuncSetAttribute(k_ring<R, C, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_ring<R, C, MODE><<<grid, block, smem, st>>>(p->rings, phase, bhat, twid, p->fft_M_max, lane_words, nlanes, rc,
                                                p->mmax, p->npairs, p->npix, p->nrings, in_map, out_user, s_state, w,
                                                wd, p->norms, stp, s_anchor);
  return cudaGetLastError();
}

// FP64 maps for the user-facing modes; the iteration state is s_iter (FP64:
// the caller's s buffer; FP32: the plan's s32).
cudaError_t ring_stage(dm_plan *p, int mode, const double *in_map, double *out_map, cudaStream_t st) {
  if (p->prec == DM_FP64) {
    switch (mode) {
      case RING_FWD_MAP:
        return launch_ring<double, double2, RING_FWD_MAP>(p, p->phase, p->bhat, p->twid, p->rc, in_map, nullptr,
                                                          nullptr, p->w, p->wd, st);
      case RING_INV_MAP:
        return launch_ring<double, double2, RING_INV_MAP>(p, p->phase, p->bhat, p->twid, p->rc, nullptr, out_map,
                                                          nullptr, p->w, p->wd, st);
      case RING_ITER:
        return launch_ring<double, double2, RING_ITER>(p, p->phase, p->bhat, p->twid, p->rc, nullptr, nullptr,
                                                       out_map, p->w, p->wd, st);
      case RING_INIT:
        return launch_ring<double, double2, RING_INIT>(p, p->phase, p->bhat, p->twid, p->rc, in_map, nullptr,
                                                       nullptr, p->w, p->wd, st);
    }
  } else {
    switch (mode) {
      case RING_FWD_MAP:
        return launch_ring<float, float2, RING_FWD_MAP>(p, p->phase32, p->bhat32, p->twid32, p->rc32, in_map,
                                                        nullptr, nullptr, p->w32, p->wd32, st);
      case RING_INV_MAP:
        return launch_ring<float, float2, RING_INV_MAP>(p, p->phase32, p->bhat32, p->twid32, p->rc32, nullptr,
                                                        out_map, nullptr, p->w32, p->wd32, st);
      case RING_ITER:
        return launch_ring<float, float2, RING_ITER>(p, p->phase32, p->bhat32, p->twid32, p->rc32, nullptr,
                                                     nullptr, p->s32, p->w32, p->wd32, st,
                                                     p->anchor_active ? p->shi32 : nullptr);
      case RING_INIT:
        return launch_ring<float, float2, RING_INIT>(p, p->phase32, p->bhat32, p->twid32, p->rc32, in_map,
                                                     nullptr, nullptr, p->w32, p->wd32, st);
    }
  }
  return cudaErrorInvalidValue;
}

// public layout rc_pub[b][f][ring][m] (complex128) <-> internal rc[b][f][m][pair][side]
template <typename C>
__global__ void k_rc_pub(const RingDev *rings, C *rc, double2 *pub, int mmax, int npairs, int nrings,
                         int to_public) {
  int r = blockIdx.x, f = blockIdx.y, b = blockIdx.z;
  RingDev R = rings[r];
  for (int m = threadIdx.x; m <= mmax; m += blockDim.x) {
    int64_t pi = (((int64_t)b * 3 + f) * nrings + r) * (mmax + 1) + m;
    int64_t ii = rc_index(b, f, m, mmax, R.pair, npairs, R.side);
    if (to_public) {
      pub[pi] = make_double2(rc[ii].x, rc[ii].y);
    } else {
      C v;
      v.x = pub[pi].x;
      v.y = pub[pi].y;
      rc[ii] = v;
    }
  }
}

cudaError_t rc_to_public(dm_plan *p, double2 *pub, cudaStream_t st) {
  dim3 g(p->nrings, 3, p->batch);
  if (p->prec == DM_FP64)
    k_rc_pub<<<g, 128, 0, st>>>(p->rings, p->rc, pub, p->mmax, p->npairs, p->nrings, 1);
  else
    k_rc_pub<<<g, 128, 0, st>>>(p->rings, p->rc32, pub, p->mmax, p->npairs, p->nrings, 1);
  return cudaGetLastError();
}
cudaError_t rc_from_public(dm_plan *p, const double2 *pub, cudaStream_t st) {
  dim3 g(p->nrings, 3, p->batch);
  if (p->prec == DM_FP64)
    k_rc_pub<<<g, 128, 0, st>>>(p->rings, p->rc, const_cast<double2 *>(pub), p->mmax, p->npairs, p->nrings, 0);
  else
    k_rc_pub<<<g, 128, 0, st>>>(p->rings, p->rc32, const_cast<double2 *>(pub), p->mmax, p->npairs, p->nrings, 0);
  return cudaGetLastError();
}

}  // namespace dmwf
