// dm_ring.cu -- the pixel-space half of a dual messenger iteration, one CTA per
// ring (or, in the paired fixed-size kernels, per northern/southern ring pair)
// and up to sixteen (Stokes component, RHS) lanes:
//   inverse ring DFT  F_m -> s           (synthesis F, Algorithm 1)
//   Cauchy partials   ||s - s_prev||^2, ||s||^2   (stopping rule, Section 3.2)
//   messenger update  t - s = w (d - s)           (Eq. 9, diagonal N)
//   forward ring DFT  (t - s) -> G_m     (analysis F^dagger, Algorithm 1)
// A real ring of n pixels is packed as a complex sequence of h = n/2 points.
//
// Ring coefficients live in rc[b][f][m][pair][side] (double2 in the FP64
// modes, float2 in the mixed mode): the Legendre kernels read a ring pair
// (north, south) as one item, and so does the paired ring kernel.
#include <algorithm>

#include "dm_fft.cuh"
#include "dm_internal.h"

namespace dmwf {

__device__ __forceinline__ int64_t rc_index(int b, int f, int m, int mmax, int pair, int npairs, int side) {
  return ((((int64_t)b * 3 + f) * (mmax + 1) + m) * npairs + pair) * 2 + side;
}

// e^{-i pi q / n} for 0 <= q < 2n from the quarter table Tq[r] = e^{-i pi r / n},
// r <= n/2 (n = 4i is a multiple of 4): e^{-i pi q/n} = (-i)^quad Tq[q - quad n/2].
template <typename C>
__device__ __forceinline__ C phase_q(const C *Tq, int q, int n) {
  const int hq = n >> 1;
  int quad = 0;
  if (q >= n) {
    q -= n;
    quad = 2;
  }
  if (q >= hq) {
    q -= hq;
    quad += 1;
  }
  const C v = Tq[q];
  C r;
  if (quad == 0) {
    r = v;
  } else if (quad == 1) {
    r.x = v.y;
    r.y = -v.x;
  } else if (quad == 2) {
    r.x = -v.x;
    r.y = -v.y;
  } else {
    r.x = -v.y;
    r.y = v.x;
  }
  return r;
}

// L2 prefetch of a contiguous byte range by the TMA engine (16-byte aligned
// start and size): the map segments of a ring are fetched while the inverse
// transform runs.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Fold the staged S_m = F_m e^{i m phi0} (m = 0..mmax; F_{-m} = conj F_m) into
// C_k = sum_{m = k mod n, |m| <= mmax} F_m e^{i m phi0}.
template <typename C>
__device__ __forceinline__ C fold_one(const C *S, int k, int n, int mmax) {
  C acc;
  acc.x = 0;
  acc.y = 0;
  for (int m = k; m <= mmax; m += n) acc = cadd(acc, S[m]);
  for (int m = n - k; m <= mmax; m += n)
    if (m >= 1) acc = cadd(acc, cconj(S[m]));
  return acc;
}


// x mod n for 0 <= x, skipping the division in the common case x < n
__device__ __forceinline__ int mod_small(int x, int n) { return x < n ? x : x % n; }

// The same fold reading F_m from global memory (compact mode).
template <typename C>
__device__ __forceinline__ C fold_one_g(const C *__restrict__ rc, const C *Tq, int k, int n, int shift, int mmax,
                                        int64_t base, int64_t mstride) {
  C acc;
  acc.x = 0;
  acc.y = 0;
  const int n2 = 2 * n;
  for (int m = k; m <= mmax; m += n)
    acc = cadd(acc, cmulc(rc[base + (int64_t)m * mstride], phase_q(Tq, mod_small(m * shift, n2), n)));
  for (int m = n - k; m <= mmax; m += n)
    if (m >= 1) acc = cadd(acc, cconj(cmulc(rc[base + (int64_t)m * mstride], phase_q(Tq, mod_small(m * shift, n2), n))));
  return acc;
}

// The coefficients of the northern and southern rings of a pair for one
// (RHS, field, m) are adjacent (side 0, side 1): one 16-byte access for FP32,
// two adjacent ones (one sector) for FP64.
template <typename C>
__device__ __forceinline__ void ld2(const C *__restrict__ p, C &a, C &b) {
  if constexpr (sizeof(C) == 8) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a.x = v.x;
    a.y = v.y;
    b.x = v.z;
    b.y = v.w;
  } else {
    a = p[0];
    b = p[1];
  }
}
template <typename C>
__device__ __forceinline__ void st2(C *p, C a, C b) {
  if constexpr (sizeof(C) == 8) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    p[0] = a;
    p[1] = b;
  }
}

// fold_one_g for both rings of a pair at once (base: side-0 index of m = 0);
// the two rings share n, the phase offset and hence every phase.
template <typename C>
__device__ __forceinline__ void fold_pair_g(const C *__restrict__ rc, const C *Tq, int k, int n, int shift, int mmax,
                                            int64_t base, int64_t mstride, C &an, C &as) {
  an.x = an.y = 0;
  as.x = as.y = 0;
  const int n2 = 2 * n;
  for (int m = k; m <= mmax; m += n) {
    C vn, vs;
    ld2(rc + base + (int64_t)m * mstride, vn, vs);
    const C ph = phase_q(Tq, mod_small(m * shift, n2), n);
    an = cadd(an, cmulc(vn, ph));
    as = cadd(as, cmulc(vs, ph));
  }
  for (int m = n - k; m <= mmax; m += n)
    if (m >= 1) {
      C vn, vs;
      ld2(rc + base + (int64_t)m * mstride, vn, vs);
      const C ph = phase_q(Tq, mod_small(m * shift, n2), n);
      an = cadd(an, cconj(cmulc(vn, ph)));
      as = cadd(as, cconj(cmulc(vs, ph)));
    }
}

// Length-h forward DFT of the CTA's lanes in place.  Direct rings (h = M a
// power of two): bit-reversed input -> natural output.  Bluestein rings:
// natural input already multiplied by the chirp and zero-padded (to M/2, or to
// M when M < 8), bluestein_conv (DIF -> product with the kernel spectrum in
// bit-reversed order -> DIT); the caller applies conj(.) / M and the output
// chirp when it reads.
template <typename C>
__device__ __forceinline__ void ring_dft(C *buf, int M, int bluestein, const C *__restrict__ bhat, const C *tws) {
  if (!bluestein) {
    fft_dit(buf, M, tws);
    return;
  }
  bluestein_conv(buf, M, tws, bhat);
}

// end of the zero padding a Bluestein input needs (see bluestein_conv)
__device__ __forceinline__ int bl_zero_end(int M) { return M >= 8 ? (M >> 1) : M; }

// Output k of ring_dft (k < h)
// slot of element i of a lane buffer: padded (generic kernels) or swizzled
// (fixed-size kernels)
template <bool SW>
__device__ __forceinline__ int lslot(int i) { return SW ? sslot(i) : spad(i); }

template <bool SW, typename C>
__device__ __forceinline__ C dft_out(const C *buf, int k, int bluestein, const C *__restrict__ chp, float invM_f,
                                     double invM_d) {
  C v = buf[lslot<SW>(k)];
  if (bluestein) {
    v = cconj(v);
    const auto inv = sizeof(v.x) == 4 ? (decltype(v.x))invM_f : (decltype(v.x))invM_d;
    v.x *= inv;
    v.y *= inv;
    v = cmul(v, chp[k]);
  }
  return v;
}

// R: real type of the FFT and of the iteration maps (double or float); C its
// complex type.  User maps (in_map, out_user) are always FP64.  LR > 0: every
// ring of the launch has FFT size M = 2^LOGM and a lane is M / 2^LR threads
// running the fixed-size radix-2^LR transforms (twid then holds their pass
// tables); LR = 0: any size, blockDim.x threads per lane, radix-2^2 passes.
// Grid.x walks a list of rings with the same FFT size class; block =
// (blockDim.x threads per lane) x (blockDim.y lanes).  The lanes of a block are
// consecutive (RHS, Stokes) pairs of the same ring, so they run the same FFT in
// lockstep and share the ring's twiddles and quarter phase table in shared
// memory.  A lane works in place on M + 1 entries: the real-FFT packing and
// unpacking handle k and h - k in the same thread.  Lanes of finished RHS
// compute but write nothing.
template <typename R, typename C, int MODE, bool COMPACT, int LOGM, int LR, bool FUSE = false, bool CAPREG = false>
__global__ void __launch_bounds__(CAPREG ? 256 : 512,
                                  CAPREG ? 3 : ((LR == 0 || (LR == 3 && sizeof(R) == 4)) ? 2 : 1)) k_ring(const RingDev *__restrict__ rings, const int *__restrict__ order,
                                              const C *__restrict__ phase, const C *__restrict__ bhat,
                                              const C *__restrict__ twid, int tw_words, int ph_words,
                                              int buf_words, int lane_words, int nlanes, C *__restrict__ rc,
                                              int mmax, int npairs,
                                              int64_t npix, int nrings, const double *__restrict__ in_map,
                                              double *__restrict__ out_user, R *s_state, const R *__restrict__ w,
                                              const R *__restrict__ wd, double *__restrict__ norms,
                                              const SolveState *__restrict__ state,
                                              const R *__restrict__ s_anchor, const C *__restrict__ chirps) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ double red[16][8][2];  // [lane][warp]: up to 16 lanes of up to 8 warps
  const int g = threadIdx.y;
  // Paired kernels (fixed-size kernels whose lane is at most 256 threads, so
  // that two lanes fit a block): grid.x walks the northern (or the equatorial)
  // ring of each ring pair, and lanes 2q, 2q + 1 of a block are the northern
  // and southern rings for the same (RHS, field).  The fold of the
  // coefficients, the unpacking and the coefficient store then run once per
  // pair over the threads of both lanes, with one 16-byte access per m.
  constexpr bool pr = LR > 0 && ((1 << LOGM) >> LR) <= 256;
  const int Lv = blockIdx.y * blockDim.y + g;
  const int side = pr ? (Lv & 1) : 0;
  const int L = pr ? (Lv >> 1) : Lv;
  const int r0 = order[blockIdx.x];
  const bool has_pair = pr && (nrings - 1 - r0) != r0;  // the equator ring has no partner
  const int r = (pr && side) ? nrings - 1 - r0 : r0;
  const bool valid_pair = L < nlanes;
  const bool valid = valid_pair && (side == 0 || has_pair);
  const int b = valid_pair ? L / 3 : 0, f = valid_pair ? L % 3 : 0;
  bool plive = valid_pair;  // the pair's (RHS, field) is still iterating
  if ((MODE == RING_ITER || MODE == RING_INIT) && state != nullptr && valid_pair && state[b].done) plive = false;
  const bool live = plive && valid;
  if (!__syncthreads_or(live)) return;
  const RingDev Rg = rings[r];
  const int n = Rg.n, h = Rg.h, bl = Rg.bluestein;
  const int M = LR > 0 ? (1 << LOGM) : Rg.M;
  const int logM = LR > 0 ? LOGM : 31 - __clz(M);
  // Compact mode (COMPACT, rings too long for the full layout): twiddles
  // and phases are read from global memory (L1-cached) and the ring
  // coefficients are folded straight from global memory; shared memory holds
  // only the lane buffers.
  constexpr bool compact = COMPACT;
  // Fixed-size kernels fold the coefficients straight from global memory too
  // (each F_m is read once either way); dropping the staged copy halves the
  // shared memory of a lane, so more lanes stay resident.
  constexpr bool staged_S = !COMPACT && LR == 0;
  C *tws_s = reinterpret_cast<C *>(sm_raw);  // stage twiddles (M - 1 used)
  C *Tq_s = tws_s + tw_words;                // quarter phase table (n/2 + 1 used)
  C *buf = Tq_s + ph_words + (size_t)g * lane_words;  // slots lslot(0..M)
  C *bufN = Tq_s + ph_words + (size_t)(g & ~1) * lane_words, *bufS = bufN + lane_words;  // paired lanes
  C *S = buf + buf_words;                              // mmax + 1 staged coefficients (inverse modes)
  const C *tws = compact ? twid : tws_s;
  const C *Tq = compact ? phase + Rg.ph_off : Tq_s;
  const int tx = threadIdx.x, nt = LR > 0 ? ((1 << LOGM) >> LR) : (int)blockDim.x;
  const int tp = side * nt + tx, ntp = pr ? 2 * nt : nt;  // thread and thread count of a pair loop
  const int t0 = pr ? tp : tx;
  if (!compact) {
    const int tflat = threadIdx.y * nt + tx, nflat = nt * blockDim.y;
    for (int i = tflat; i < tw_words; i += nflat) tws_s[i] = twid[i];
    const C *ph = phase + Rg.ph_off;
    for (int i = tflat; i <= (n >> 1); i += nflat) Tq_s[i] = ph[i];
  }
  const int64_t moff = ((int64_t)b * 3 + f) * npix + Rg.start;
  const C *bh = bhat + (bl ? Rg.bh_off : 0);
  const C *chp = chirps + (bl ? Rg.ch_off : 0);  // Bluestein chirp e^{-i pi j^2 / h}, j < h
  const int64_t rbase = ((((int64_t)b * 3 + f) * (mmax + 1)) * npairs + Rg.pair) * 2 + Rg.side;
  const int64_t rbaseP = ((((int64_t)b * 3 + f) * (mmax + 1)) * npairs + Rg.pair) * 2;  // side 0
  const int64_t mstride = (int64_t)npairs * 2;
  if (MODE == RING_ITER && live && tx == 0) {
    // ring segments start on 16-byte boundaries: n = 4i pixels, starts and npix multiples of 4
    const uint32_t bytes = (uint32_t)(n * sizeof(R));
    prefetch_l2(s_state + moff, bytes);
    prefetch_l2(w + moff, bytes);
    prefetch_l2(s_anchor ? (const R *)s_anchor + moff : wd + moff, bytes);
  }
  const float invM_f = 1.0f / (float)M;
  const double invM_d = 1.0 / (double)M;
  __syncthreads();

  if (MODE == RING_INV_MAP || MODE == RING_ITER) {
    // Z_k = E_k + i O_k, E_k = C_k + conj(C_{h-k}), O_k = (C_k - conj(C_{h-k})) e^{2 pi i k/n},
    // stored conjugated (forward DFT + conjugation = inverse); one thread per (k, h - k).
    // stage S_m = F_m e^{i m phi0}: batches of independent loads per thread
    if (staged_S) {
      constexpr int U = sizeof(R) == 4 ? 8 : 4;
      const int n2 = 2 * n;
      for (int m0 = tx; m0 <= mmax; m0 += U * nt) {
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int m = m0 + u * nt;
          if (m <= mmax) v[u] = rc[rbase + (int64_t)m * mstride];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int m = m0 + u * nt;
          if (m <= mmax) S[m] = cmulc(v[u], phase_q(Tq, mod_small(m * Rg.shift, n2), n));
        }
      }
    }
    __syncthreads();
    // packed value of kk (t = 0: k, t = 1: h - k) into buffer x
    auto pack = [&](C *x, C ck, C ck2, int t, int kk) {
      const C a = t ? ck2 : ck, cc = cconj(t ? ck : ck2);
      const C E = cadd(a, cc), O = cmulc(csub(a, cc), phase_q(Tq, 2 * kk, n));
      C Z;  // conj(E + i O)
      Z.x = E.x - O.y;
      Z.y = -(E.y + O.x);
      if (bl)
        x[lslot<(LR > 0)>(kk)] = cmul(Z, chp[kk]);
      else
        x[lslot<(LR > 0)>(bitrev(kk, logM))] = Z;
    };
    for (int k = t0; k <= (h >> 1); k += ntp) {
      const int k2 = h - k;
      if (pr) {
        C ckN, ckS, ck2N, ck2S;
        fold_pair_g(rc, Tq, k, n, Rg.shift, mmax, rbaseP, mstride, ckN, ckS);
        if (k2 == k) {
          ck2N = ckN;
          ck2S = ckS;
        } else {
          fold_pair_g(rc, Tq, k2, n, Rg.shift, mmax, rbaseP, mstride, ck2N, ck2S);
        }
        for (int t = 0; t < 2; ++t) {
          if (t && (k2 >= h || k2 == k)) break;
          pack(bufN, ckN, ck2N, t, t ? k2 : k);
          pack(bufS, ckS, ck2S, t, t ? k2 : k);
        }
        continue;
      }
      const C ck = !staged_S ? fold_one_g(rc, Tq, k, n, Rg.shift, mmax, rbase, mstride) : fold_one(S, k, n, mmax);
      const C ck2 = (k2 == k) ? ck
                              : (!staged_S ? fold_one_g(rc, Tq, k2, n, Rg.shift, mmax, rbase, mstride)
                                         : fold_one(S, k2, n, mmax));
      for (int t = 0; t < 2; ++t) {
        if (t && (k2 >= h || k2 == k)) break;
        pack(buf, ck, ck2, t, t ? k2 : k);
      }
    }
    if (bl)
      for (int j = h + tx; j < bl_zero_end(M); j += nt) {
        buf[lslot<(LR > 0)>(j)].x = 0;
        buf[lslot<(LR > 0)>(j)].y = 0;
      }
    __syncthreads();
    if constexpr (LR > 0 && FUSE) {  // all but the last pass: that one is fused with the update below
      if (bl)
        bluesteinr_head<C, LOGM, LR>(buf, tws, bh, tx);
      else
        fftr_dit_head<C, LOGM, LR>(buf, tws, tx);
    } else if constexpr (LR > 0) {
      if (bl)
        bluesteinr<C, LOGM, LR>(buf, tws, bh, tx);
      else
        fftr_dit<C, LOGM, LR>(buf, tws, tx);
    } else {
      ring_dft(buf, M, bl, bh, tws);
    }
    // z_j = conj(D_j) = s_{2j} + i s_{2j+1}
    if (MODE == RING_INV_MAP) {
      if (live)
        for (int j = tx; j < h; j += nt) {
          const C z = dft_out<(LR > 0)>(buf, j, bl, chp, invM_f, invM_d);
          out_user[moff + 2 * j] = (double)z.x;
          out_user[moff + 2 * j + 1] = -(double)z.y;
        }
      return;
    }
    // RING_ITER: Cauchy partials, store s, form t - s = w d - w s and pack it.
    // With an anchor (mixed precision) the state is Y e, s = s_anchor + Y e, and
    // the data part w (d - s_anchor) is carried in FP64 by the anchor: r = -w Y e.
    // Each thread accumulates the Cauchy partials of its few pixels in the map
    // precision R (FP32 in the mixed mode, whose maps are FP32; FP64 arithmetic
    // runs at a small fraction of the FP32 rate on this GPU), the sums over
    // threads run in FP64.
    R dd_t = 0, ss_t = 0;
    // every thread reads and rewrites its own entries j only; plan-owned maps,
    // (s_{2j}, s_{2j+1}) read as one aligned pair, two j per batch
    C *sv = reinterpret_cast<C *>(s_state + moff);
    const C *wv = reinterpret_cast<const C *>(w + moff);
    const C *dv = reinterpret_cast<const C *>(wd + moff);
    const C *av = s_anchor ? reinterpret_cast<const C *>(s_anchor + moff) : nullptr;
    if constexpr (LR > 0 && FUSE) {
      // the fixed-size kernels: last inverse pass, this update and the first
      // forward pass in registers (fused_dit_dif); element j = tx + q M/2^LR
      const R invM = sizeof(R) == 4 ? (R)invM_f : (R)invM_d;
      auto upd = [&](int q, C y) -> C {
        const int j = tx + q * ((1 << LOGM) >> LR);
        C rr;
        rr.x = 0;
        rr.y = 0;
        if (j >= h) return rr;  // the Bluestein zero padding (direct rings: h = M)
        C z = y;
        if (bl) {
          z = cconj(z);
          z.x *= invM;
          z.y *= invM;
          z = cmul(z, chp[j]);
        }
        C sn;
        sn.x = z.x;
        sn.y = -z.y;
        if (live) {
          const C so = sv[j], ww = wv[j];
          const R d0 = sn.x - so.x, d1 = sn.y - so.y;
          dd_t += d0 * d0 + d1 * d1;
          sv[j] = sn;
          if (av) {
            const C sa = av[j];
            const R f0 = sa.x + sn.x, f1 = sa.y + sn.y;
            ss_t += f0 * f0 + f1 * f1;
            rr.x = -ww.x * sn.x;
            rr.y = -ww.y * sn.y;
          } else {
            const C dw = dv[j];
            ss_t += sn.x * sn.x + sn.y * sn.y;
            rr.x = dw.x - ww.x * sn.x;
            rr.y = dw.y - ww.y * sn.y;
          }
        }
        return bl ? cmul(rr, chp[j]) : rr;
      };
      if (bl)
        fused_dit_dif<C, LOGM, LR, true>(buf, tws, tx, upd);
      else
        fused_dit_dif<C, LOGM, LR, false>(buf, tws, tx, upd);
    } else
    for (int j0 = tx; j0 < h; j0 += 2 * nt) {
      C so[2], ww[2], dw[2], sa[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = j0 + u * nt;
        if (live && j < h) {
          so[u] = sv[j];
          ww[u] = wv[j];
          if (av)
            sa[u] = av[j];
          else
            dw[u] = dv[j];
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = j0 + u * nt;
        if (j >= h) break;
        const C z = dft_out<(LR > 0)>(buf, j, bl, chp, invM_f, invM_d);
        C s;
        s.x = z.x;
        s.y = -z.y;
        C rr;
        if (live) {
          const R d0 = s.x - so[u].x, d1 = s.y - so[u].y;
          dd_t += d0 * d0 + d1 * d1;
          sv[j] = s;
          if (av) {
            const R f0 = sa[u].x + s.x, f1 = sa[u].y + s.y;
            ss_t += f0 * f0 + f1 * f1;
            rr.x = -ww[u].x * s.x;
            rr.y = -ww[u].y * s.y;
          } else {
            ss_t += s.x * s.x + s.y * s.y;
            rr.x = dw[u].x - ww[u].x * s.x;
            rr.y = dw[u].y - ww[u].y * s.y;
          }
        } else {
          rr.x = 0;
          rr.y = 0;
        }
        buf[lslot<(LR > 0)>(j)] = bl ? cmul(rr, chp[j]) : rr;
      }
    }
    // warp sums in the map precision, the sums over warps and rings in FP64
    for (int o = 16; o > 0; o >>= 1) {
      dd_t += __shfl_down_sync(0xffffffffu, dd_t, o);
      ss_t += __shfl_down_sync(0xffffffffu, ss_t, o);
    }
    if ((tx & 31) == 0) {
      red[g][tx >> 5][0] = (double)dd_t;
      red[g][tx >> 5][1] = (double)ss_t;
    }
    __syncthreads();
    if (tx == 0 && live) {
      double a = 0.0, c = 0.0;
      for (int i = 0; i < (nt >> 5); ++i) {
        a += red[g][i][0];
        c += red[g][i][1];
      }
      const int64_t no = (((int64_t)b * 3 + f) * nrings + r) * 2;
      norms[no] = a;
      norms[no + 1] = c;
    }
  } else {
    // forward only: load the real ring (RING_INIT: t_0 - s_0 = d on observed pixels)
    for (int j = tx; j < h; j += nt) {
      double x0 = 0.0, x1 = 0.0;
      if (valid) {
        x0 = in_map[moff + 2 * j];
        x1 = in_map[moff + 2 * j + 1];
        if (MODE == RING_INIT) {
          x0 = (w[moff + 2 * j] > (R)0) ? x0 : 0.0;
          x1 = (w[moff + 2 * j + 1] > (R)0) ? x1 : 0.0;
        }
      }
      C v;
      v.x = (R)x0;
      v.y = (R)x1;
      buf[lslot<(LR > 0)>(j)] = bl ? cmul(v, chp[j]) : v;
    }
  }
  if (!FUSE && bl)  // (a fused pass wrote the padding itself)
    for (int j = h + tx; j < bl_zero_end(M); j += nt) {
      buf[lslot<(LR > 0)>(j)].x = 0;
      buf[lslot<(LR > 0)>(j)].y = 0;
    }
  __syncthreads();
  // forward: Z = DFT_h(z); direct rings take natural input to bit-reversed output
  if constexpr (LR > 0 && FUSE) {  // its first pass ran fused with the update
    if (bl)
      bluesteinr_tail<C, LOGM, LR>(buf, tws, bh, tx);
    else
      fftr_dif_tail<C, LOGM, LR>(buf, tws, tx);
  } else if constexpr (LR > 0) {
    if (bl)
      bluesteinr<C, LOGM, LR>(buf, tws, bh, tx);
    else
      fftr_dif<C, LOGM, LR>(buf, tws, tx);
  } else {
    if (bl)
      ring_dft(buf, M, 1, bh, tws);
    else
      fft_dif(buf, M, tws);
  }
  // X_k = E_k + e^{-2 pi i k/n} O_k, E_k = (Z_k + conj Z_{h-k}) / 2, O_k = (Z_k - conj Z_{h-k}) / 2i,
  // Z_h = Z_0; each thread reads and rewrites the slots of k and h - k; X_h goes to slot M (direct)
  // or slot h (Bluestein).
  const R half = (R)0.5;
  auto unpack = [&](C *x, int k) {
    const int k2 = h - k;
    const int sk = bl ? k : bitrev(k, logM);
    const int sk2 = (k == 0) ? sk : (bl ? k2 : bitrev(k2, logM));
    const C zk = dft_out<(LR > 0)>(x, sk, bl, chp, invM_f, invM_d);
    const C zk2 = (k == 0) ? zk : dft_out<(LR > 0)>(x, sk2, bl, chp, invM_f, invM_d);
    for (int t = 0; t < 2; ++t) {
      if (t && k2 == k) break;
      const C a = t ? zk2 : zk, c = cconj(t ? zk : zk2);
      const int kk = t ? k2 : k;
      C E, O;
      E.x = half * (a.x + c.x);
      E.y = half * (a.y + c.y);
      const C D = csub(a, c);
      O.x = half * D.y;
      O.y = -half * D.x;
      const C X = cadd(E, cmul(O, phase_q(Tq, 2 * kk, n)));
      const int slot = t ? ((k == 0) ? (bl ? h : M) : sk2) : sk;
      x[lslot<(LR > 0)>(slot)] = X;
    }
  };
  for (int k = t0; k <= (h >> 1); k += ntp) {
    if (pr) {
      unpack(bufN, k);
      unpack(bufS, k);
    } else {
      unpack(buf, k);
    }
  }
  __syncthreads();
  if (!(pr ? plive : live)) return;
  const int n2 = 2 * n;
  for (int m = t0; m <= mmax; m += ntp) {
    const int q = mod_small(m, n);
    const int qq = (q <= h) ? q : n - q;
    const int slot = bl ? qq : (qq == h ? M : bitrev(qq, logM));
    const C ph = phase_q(Tq, mod_small(m * Rg.shift, n2), n);
    if (pr) {
      C XN = bufN[lslot<(LR > 0)>(slot)], XS = bufS[lslot<(LR > 0)>(slot)];
      if (q > h) {
        XN = cconj(XN);
        XS = cconj(XS);
      }
      C *dst = rc + rbaseP + (int64_t)m * mstride;
      if (has_pair)
        st2(dst, cmul(XN, ph), cmul(XS, ph));
      else
        dst[0] = cmul(XN, ph);
    } else {
      C X = buf[lslot<(LR > 0)>(slot)];
      if (q > h) X = cconj(X);
      rc[rbase + (int64_t)m * mstride] = cmul(X, ph);
    }
  }
}

// Rings are launched by size class: one grid per class so that each gets the
// shared memory (twiddles, quarter phase table, G lanes of M + 1 entries) it needs.
// Iteration launches of classes with one FFT size M in [512, 4096] take the
// fixed-size kernel (LOGM = log2 M, radix 2^ring_lr, M / 2^ring_lr threads
// per lane) unless the plan's ring_lr is 0.
template <typename R, typename C, int MODE, int LR, bool FUSE, bool CAPREG = false>
static void pick_fixed(int logm, void (*&kern)(const RingDev *, const int *, const C *, const C *, const C *, int,
                                               int, int, int, int, C *, int, int, int64_t, int, const double *,
                                               double *, R *, const R *, const R *, double *, const SolveState *,
                                               const R *, const C *)) {
  switch (logm) {
    case 9: kern = k_ring<R, C, MODE, false, 9, LR, FUSE, CAPREG>; break;
    case 10: kern = k_ring<R, C, MODE, false, 10, LR, FUSE, CAPREG>; break;
    case 11: kern = k_ring<R, C, MODE, false, 11, LR, FUSE, CAPREG>; break;
    default: kern = k_ring<R, C, MODE, false, 12, LR, FUSE, CAPREG>; break;
  }
}

template <typename R, typename C, int MODE>
static cudaError_t launch_ring(dm_plan *p, const C *phase, const C *bhat, const C *chirps, const C *twid, C *rc,
                               const double *in_map, double *out_user, R *s_state, const R *w, const R *wd,
                               cudaStream_t st, const R *s_anchor = nullptr, const C *twr = nullptr,
                               const C *const *bhatT = nullptr) {
  using Kern = void (*)(const RingDev *, const int *, const C *, const C *, const C *, int, int, int, int, int, C *,
                        int, int, int64_t, int, const double *, double *, R *, const R *, const R *, double *,
                        const SolveState *, const R *, const C *);
  const int nlanes = 3 * p->batch;
  const SolveState *stp = (MODE == RING_ITER || MODE == RING_INIT) ? p->state : nullptr;
  for (int ci = 0; ci < (int)p->ring_classes.size(); ++ci) {
    const RingClass &rc_cls = p->ring_classes[ci];
    if (p->tune_only_class >= 0 && ci != p->tune_only_class) continue;
    const bool tcls = ci < DM_TUNE_MAX_CLASSES;
    const int lr = (tcls && p->tune_ring_lr[ci] >= 0) ? p->tune_ring_lr[ci] : p->ring_lr;
    int tw_words = std::max(1, rc_cls.M - 1);
    int ph_words = rc_cls.n / 2 + 1;
    int buf_words = rc_cls.M + rc_cls.M / 32 + 1;  // slots spad(0..M)
    const bool staged = (MODE == RING_ITER || MODE == RING_INV_MAP);
    int lane_words = buf_words + (staged ? p->mmax + 1 : 0);
    if (sizeof(C) * ((size_t)tw_words + ph_words + lane_words) > (227u << 10)) {  // compact mode
      tw_words = ph_words = 0;
      lane_words = buf_words;
      if (sizeof(C) * (size_t)lane_words > (227u << 10)) return cudaErrorInvalidValue;
    }
    const bool compact = (tw_words == 0);
    const int logm = 31 - __builtin_clz((unsigned)rc_cls.M);
    const bool fixed = MODE == RING_ITER && !compact && twr != nullptr && (lr == 3 || lr == 4) &&
                       rc_cls.M == (1 << logm) && logm >= 9 && logm <= 12 && p->twr_off[lr - 3][logm] >= 0 &&
                       (bhatT == nullptr || bhatT[lr - 3] != nullptr || p->bh_total == 0);
    Kern kern = compact ? k_ring<R, C, MODE, true, 0, 0> : k_ring<R, C, MODE, false, 0, 0>;
    int T = 128;
    const C *tws = twid;
    if constexpr (MODE == RING_ITER) {
      if (fixed) {
        // separate passes unless tuned otherwise (measured faster on the
        // bench workload: the fused pass spills at the 64-register cap)
        const bool fuse = tcls && p->tune_ring_fuse[ci] == 1;
        // variant 2: the FP32 radix-16 kernels of up to 2048 points compiled
        // for three blocks of 256 threads per SM (80 registers a thread)
        // instead of 128 registers and two blocks
        const bool cap = sizeof(R) == 4 && tcls && p->tune_ring_fuse[ci] == 2 && lr == 4 && logm <= 11;
        if (lr == 3) {
          fuse ? pick_fixed<R, C, MODE, 3, true>(logm, kern) : pick_fixed<R, C, MODE, 3, false>(logm, kern);
        } else if (cap) {
          if constexpr (sizeof(R) == 4) pick_fixed<R, C, MODE, 4, false, true>(logm, kern);
        } else {
          fuse ? pick_fixed<R, C, MODE, 4, true>(logm, kern) : pick_fixed<R, C, MODE, 4, false>(logm, kern);
        }
        if (tcls) p->ring_fuse_used[ci] = cap ? 2 : (fuse ? 1 : 0);
        T = rc_cls.M >> lr;
        tw_words = fftr_tw_words(logm, lr);
        tws = twr + p->twr_off[lr - 3][logm];
        lane_words = buf_words = rc_cls.M + 16;  // swizzled slots 0..M, no staged coefficients
      }
    }
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    // fixed-size kernels take both rings of a pair per block when two lanes
    // fit (the kernel's compile-time pr)
    const bool paired = fixed && T <= 256;
    const int vlanes = paired ? 2 * nlanes : nlanes;
    int G = ring_lanes_per_block(sizeof(C), tw_words, ph_words, lane_words, vlanes, fa.numRegs, T);
    if (tcls && p->tune_ring_G[ci] > 0) {  // tuned: clamp to what the launch allows
      int gmax = 1;
      while (gmax < 16 && (gmax + 1) * T <= 512 && (gmax + 1) * T <= fa.maxThreadsPerBlock &&
             sizeof(C) * ((size_t)tw_words + ph_words + (size_t)(gmax + 1) * lane_words) <= (227u << 10))
        ++gmax;
      G = std::min(std::min(p->tune_ring_G[ci], gmax), vlanes);
    }
    while (G > 1 && G * T > fa.maxThreadsPerBlock) --G;  // the register-capped kernels take 256 threads
    if (paired) G = std::max(2, G & ~1);
    if (MODE == RING_ITER && tcls) {
      p->ring_G_used[ci] = G;
      p->ring_lr_used[ci] = fixed ? lr : 0;
    }
    const size_t smem = sizeof(C) * ((size_t)tw_words + ph_words + (size_t)G * lane_words);
    dim3 grid(paired ? rc_cls.pcount : rc_cls.count, (vlanes + G - 1) / G);
    dim3 block(T, G);
    e = dyn_smem_allow(kern, smem);
    if (e != cudaSuccess) return e;
    const int *order = paired ? p->pair_order + rc_cls.poff : p->ring_order + rc_cls.off;
    // the fixed-size kernels read the Bluestein spectra transposed
    const C *bh_k = (fixed && bhatT != nullptr && bhatT[lr - 3] != nullptr) ? bhatT[lr - 3] : bhat;
    kern<<<grid, block, smem, st>>>(p->rings, order, phase, bh_k, tws, tw_words, ph_words, buf_words, lane_words,
                                    nlanes, rc, p->mmax, p->npairs, p->npix, p->nrings, in_map, out_user, s_state, w,
                                    wd, p->norms, stp, s_anchor, chirps);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Lanes per block: the G that keeps the most lanes resident on an SM (228 KB
// of shared memory with 1 KB reserved per block, 2048 threads, 64 K registers
// allocated per warp in units of 256), with G x nt <= 512 threads and G <= 16
// (the kernel's reduction array), ties to the larger G.
int ring_lanes_per_block(size_t word_bytes, int tw_words, int ph_words, int lane_words, int nlanes, int regs,
                         int nt) {
  int best = 1;
  long best_lanes = -1;
  const int warps = (nt + 31) / 32;
  for (int G = 1; G <= 16 && G * nt <= 512; ++G) {
    const size_t smem = word_bytes * ((size_t)tw_words + ph_words + (size_t)G * lane_words);
    if (smem > (227u << 10)) break;
    long blocks = (long)((228u << 10) / (smem + 1024));
    blocks = std::min<long>(blocks, 2048 / (nt * G));
    blocks = std::min<long>(blocks, 32);
    const long warp_regs = ((long)std::max(regs, 1) * 32 + 255) / 256 * 256;
    blocks = std::min<long>(blocks, 65536 / (warp_regs * warps * G));
    const long lanes = blocks * G;
    if (lanes >= best_lanes) {
      best_lanes = lanes;
      best = G;
    }
  }
  return std::max(1, std::min(best, nlanes));
}

// FP64 maps for the user-facing modes; the iteration state is s_iter (FP64:
// the caller's s buffer; FP32: the plan's s32).
cudaError_t ring_stage(dm_plan *p, int mode, const double *in_map, double *out_map, cudaStream_t st) {
  if (p->prec == DM_FP64) {
    switch (mode) {
      case RING_FWD_MAP:
        return launch_ring<double, double2, RING_FWD_MAP>(p, p->phase, p->bhat, p->chirp, p->twid, p->rc, in_map, nullptr,
                                                          nullptr, p->w, p->wd, st);
      case RING_INV_MAP:
        return launch_ring<double, double2, RING_INV_MAP>(p, p->phase, p->bhat, p->chirp, p->twid, p->rc, nullptr, out_map,
                                                          nullptr, p->w, p->wd, st);
      case RING_ITER:
        return launch_ring<double, double2, RING_ITER>(p, p->phase, p->bhat, p->chirp, p->twid, p->rc, nullptr, nullptr,
                                                       out_map, p->w, p->wd, st, nullptr, p->twr, p->bhatT);
      case RING_INIT:
        return launch_ring<double, double2, RING_INIT>(p, p->phase, p->bhat, p->chirp, p->twid, p->rc, in_map, nullptr,
                                                       nullptr, p->w, p->wd, st);
    }
  } else {
    switch (mode) {
      case RING_FWD_MAP:
        return launch_ring<float, float2, RING_FWD_MAP>(p, p->phase32, p->bhat32, p->chirp32, p->twid32, p->rc32, in_map,
                                                        nullptr, nullptr, p->w32, p->wd32, st);
      case RING_INV_MAP:
        return launch_ring<float, float2, RING_INV_MAP>(p, p->phase32, p->bhat32, p->chirp32, p->twid32, p->rc32, nullptr,
                                                        out_map, nullptr, p->w32, p->wd32, st);
      case RING_ITER:
        return launch_ring<float, float2, RING_ITER>(p, p->phase32, p->bhat32, p->chirp32, p->twid32, p->rc32, nullptr,
                                                     nullptr, p->s32, p->w32, p->wd32, st,
                                                     p->anchor_active ? p->shi32 : nullptr, p->twr32, p->bhatT32);
      case RING_INIT:
        return launch_ring<float, float2, RING_INIT>(p, p->phase32, p->bhat32, p->chirp32, p->twid32, p->rc32, in_map,
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
