// dm_fft.cuh -- shared-memory FFT building blocks for the ring transforms.
//
// Every HEALPix ring of n = 4i pixels is transformed as a real sequence packed
// into a complex one of length h = n / 2.  h is a power of two for the
// equatorial belt when nside is; the other lengths (h = 2i) go through
// Bluestein's chirp-z convolution (Bluestein 1970) on a power-of-two size M.
//
// Twiddles are stage-contiguous: tws[len - 1 + j] = e^{-i pi j / len} for the
// butterfly half-length len = 1, 2, 4, ... and j < len, so a transform of size
// M reads the first M - 1 entries and consecutive threads of a stage read
// consecutive entries.
//
// Two radix-2 forms avoid an explicit bit-reversal pass:
//   fft_dif: natural-order input -> bit-reversed output (Gentleman-Sande)
//   fft_dit: bit-reversed input  -> natural-order output (Cooley-Tukey)
// Both compute the forward transform X_k = sum_j x_j e^{-2 pi i jk/M}, and
// both fuse two radix-2 stages per pass (one closed quadruple per task), so a
// size-M transform takes ceil(log2 M / 2) barriers.  These generic forms take
// any M; the fixed-size family at the end of this file (fftr_*, radix 8 or
// 16 per pass in registers, XOR-swizzled slots) produces the same layouts for
// one compile-time M and serves the iteration's rings of 512 to 4096 points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dmwf {

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename T2>
__device__ __forceinline__ T2 cmulc(T2 a, T2 b) {  // a * conj(b)
  T2 r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename T2>
__device__ __forceinline__ T2 cconj(T2 a) {
  a.y = -a.y;
  return a;
}
template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
template <typename T2>
__device__ __forceinline__ T2 cmul_negi(T2 a) {  // a * (-i)
  T2 r;
  r.x = a.y;
  r.y = -a.x;
  return r;
}

// Shared-memory slot of element i of a transform buffer: one pad entry every 32
// elements, so that the power-of-two strides of the bit-reversed order and of
// the short butterflies do not all fall into the same bank.  A buffer of n
// elements takes spad(n - 1) + 1 entries.
__device__ __forceinline__ int spad(int i) { return i + (i >> 5); }

// index k of a size-2^logM transform in bit-reversed order
__device__ __forceinline__ int bitrev(int k, int logM) { return (int)(__brev((unsigned)k) >> (32 - logM)); }

// In place (slots spad(i)), natural order in, bit-reversed order out.  Threads threadIdx.x of
// blockDim.x take part (every y-slice of the block runs its own transform in
// lockstep); the caller syncs before, this ends with a block barrier.
template <typename T2>
__device__ void fft_dif(T2 *x, int M, const T2 *tws) {
  if (M <= 1) return;
  const int logM = 31 - __clz(M);
  const int tx = threadIdx.x, nt = blockDim.x;
  int L2 = M >> 1;  // half-length of the first stage of the pass
  for (; L2 >= 2; L2 >>= 2) {
    const int L = L2 >> 1;  // stages 2L then L on {B + j + {0, L, 2L, 3L}}, B a multiple of 4L
    for (int k = tx; k < (M >> 2); k += nt) {
      const int j = k & (L - 1);
      const int i0 = ((k - j) << 2) + j;
      const T2 a0 = x[spad(i0)], a1 = x[spad(i0 + L)], a2 = x[spad(i0 + 2 * L)], a3 = x[spad(i0 + 3 * L)];
      const T2 w2 = tws[2 * L - 1 + j], w1 = tws[L - 1 + j];
      const T2 b0 = cadd(a0, a2), b2 = cmul(csub(a0, a2), w2);
      const T2 b1 = cadd(a1, a3), b3 = cmul_negi(cmul(csub(a1, a3), w2));
      x[spad(i0)] = cadd(b0, b1);
      x[spad(i0 + L)] = cmul(csub(b0, b1), w1);
      x[spad(i0 + 2 * L)] = cadd(b2, b3);
      x[spad(i0 + 3 * L)] = cmul(csub(b2, b3), w1);
    }
    __syncthreads();
  }
  if (logM & 1) {  // last single stage, half-length 1 (twiddle 1)
    for (int k = tx; k < (M >> 1); k += nt) {
      const T2 u = x[spad(2 * k)], v = x[spad(2 * k + 1)];
      x[spad(2 * k)] = cadd(u, v);
      x[spad(2 * k + 1)] = csub(u, v);
    }
    __syncthreads();
  }
}

// In place, bit-reversed order in, natural order out; same conventions.
template <typename T2>
__device__ void fft_dit(T2 *x, int M, const T2 *tws) {
  if (M <= 1) return;
  const int logM = 31 - __clz(M);
  const int tx = threadIdx.x, nt = blockDim.x;
  int L = 1;
  if (logM & 1) {  // first single stage, half-length 1
    for (int k = tx; k < (M >> 1); k += nt) {
      const T2 u = x[spad(2 * k)], v = x[spad(2 * k + 1)];
      x[spad(2 * k)] = cadd(u, v);
      x[spad(2 * k + 1)] = csub(u, v);
    }
    __syncthreads();
    L = 2;
  }
  for (; L < M; L <<= 2) {  // stages L then 2L on {B + j + {0, L, 2L, 3L}}
    for (int k = tx; k < (M >> 2); k += nt) {
      const int j = k & (L - 1);
      const int i0 = ((k - j) << 2) + j;
      const T2 a0 = x[spad(i0)], a1 = x[spad(i0 + L)], a2 = x[spad(i0 + 2 * L)], a3 = x[spad(i0 + 3 * L)];
      const T2 w1 = tws[L - 1 + j], w2 = tws[2 * L - 1 + j];
      T2 v = cmul(a1, w1);
      const T2 b0 = cadd(a0, v), b1 = csub(a0, v);
      v = cmul(a3, w1);
      const T2 b2 = cadd(a2, v), b3 = csub(a2, v);
      v = cmul(b2, w2);
      x[spad(i0)] = cadd(b0, v);
      x[spad(i0 + 2 * L)] = csub(b0, v);
      v = cmul_negi(cmul(b3, w2));
      x[spad(i0 + L)] = cadd(b1, v);
      x[spad(i0 + 3 * L)] = csub(b1, v);
    }
    __syncthreads();
  }
}

// Bluestein convolution core of one ring, in place (slots spad(i)):
//   x <- FFT_M( conj( FFT_M(x) * bhat ) ),  bhat in bit-reversed order,
// for an input whose upper half [M/2, M) is zero (h <= M/2 chirped points,
// zero-filled up to M/2 by the caller; for M < 8 up to M) and of which only
// the lower half of the output is read.  The first DIF pass skips the zero
// half, the last DIF stage, the product with bhat and the first DIT stage run
// as one pass on the same slots (no barrier between them), and the last DIT
// pass computes only the lower half.  Same threading conventions as above.
template <typename T2>
__device__ void bluestein_conv(T2 *x, int M, const T2 *tws, const T2 *__restrict__ bhat) {
  const int logM = 31 - __clz(M);
  const int tx = threadIdx.x, nt = blockDim.x;
  const int lastL2 = (logM & 1) ? 1 : 2;  // half-length of the first stage of the last DIF pass
  // DIF passes before the last one
  for (int L2 = M >> 1; L2 > lastL2 && L2 >= 2; L2 >>= 2) {
    const int L = L2 >> 1;
    const bool zero_upper = (L2 == (M >> 1));
    for (int k = tx; k < (M >> 2); k += nt) {
      const int j = k & (L - 1);
      const int i0 = ((k - j) << 2) + j;
      const T2 w2 = tws[2 * L - 1 + j], w1 = tws[L - 1 + j];
      const T2 a0 = x[spad(i0)], a1 = x[spad(i0 + L)];
      T2 b0, b1, b2, b3;
      if (zero_upper) {
        b0 = a0;
        b2 = cmul(a0, w2);
        b1 = a1;
        b3 = cmul_negi(cmul(a1, w2));
      } else {
        const T2 a2 = x[spad(i0 + 2 * L)], a3 = x[spad(i0 + 3 * L)];
        b0 = cadd(a0, a2);
        b2 = cmul(csub(a0, a2), w2);
        b1 = cadd(a1, a3);
        b3 = cmul_negi(cmul(csub(a1, a3), w2));
      }
      x[spad(i0)] = cadd(b0, b1);
      x[spad(i0 + L)] = cmul(csub(b0, b1), w1);
      x[spad(i0 + 2 * L)] = cadd(b2, b3);
      x[spad(i0 + 3 * L)] = cmul(csub(b2, b3), w1);
    }
    __syncthreads();
  }
  // last DIF pass + pointwise product + first DIT pass on the same slots
  if (logM & 1) {
    for (int k = tx; k < (M >> 1); k += nt) {
      const int s0 = 2 * k, s1 = 2 * k + 1;
      const T2 u = x[spad(s0)], v = x[spad(s1)];
      const T2 y0 = cconj(cmul(cadd(u, v), bhat[s0])), y1 = cconj(cmul(csub(u, v), bhat[s1]));
      x[spad(s0)] = cadd(y0, y1);
      x[spad(s1)] = csub(y0, y1);
    }
  } else {
    for (int k = tx; k < (M >> 2); k += nt) {
      const int i0 = 4 * k;
      const T2 a0 = x[spad(i0)], a1 = x[spad(i0 + 1)], a2 = x[spad(i0 + 2)], a3 = x[spad(i0 + 3)];
      // DIF radix-4 (unit twiddles): outputs in slots i0 .. i0 + 3
      const T2 b0 = cadd(a0, a2), b2 = csub(a0, a2), b1 = cadd(a1, a3), b3 = cmul_negi(csub(a1, a3));
      const T2 y0 = cconj(cmul(cadd(b0, b1), bhat[i0])), y1 = cconj(cmul(csub(b0, b1), bhat[i0 + 1]));
      const T2 y2 = cconj(cmul(cadd(b2, b3), bhat[i0 + 2])), y3 = cconj(cmul(csub(b2, b3), bhat[i0 + 3]));
      // DIT radix-4 (unit twiddles) on the same slots
      const T2 c0 = cadd(y0, y1), c1 = csub(y0, y1), c2 = cadd(y2, y3), c3 = cmul_negi(csub(y2, y3));
      x[spad(i0)] = cadd(c0, c2);
      x[spad(i0 + 2)] = csub(c0, c2);
      x[spad(i0 + 1)] = cadd(c1, c3);
      x[spad(i0 + 3)] = csub(c1, c3);
    }
  }
  __syncthreads();
  // remaining DIT passes; the last one (L = M/4) writes only the lower half
  for (int L = (logM & 1) ? 2 : 4; L < M; L <<= 2) {
    const bool half_out = (4 * L == M);
    for (int k = tx; k < (M >> 2); k += nt) {
      const int j = k & (L - 1);
      const int i0 = ((k - j) << 2) + j;
      const T2 a0 = x[spad(i0)], a1 = x[spad(i0 + L)], a2 = x[spad(i0 + 2 * L)], a3 = x[spad(i0 + 3 * L)];
      const T2 w1 = tws[L - 1 + j], w2 = tws[2 * L - 1 + j];
      T2 v = cmul(a1, w1);
      const T2 b0 = cadd(a0, v), b1 = csub(a0, v);
      v = cmul(a3, w1);
      const T2 b2 = cadd(a2, v), b3 = csub(a2, v);
      const T2 v2 = cmul(b2, w2), v3 = cmul_negi(cmul(b3, w2));
      x[spad(i0)] = cadd(b0, v2);
      x[spad(i0 + L)] = cadd(b1, v3);
      if (!half_out) {
        x[spad(i0 + 2 * L)] = csub(b0, v2);
        x[spad(i0 + 3 * L)] = csub(b1, v3);
      }
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// Fixed-size transforms, M = 2^LOGM >= 512, radix R = 2^LR (LR = 3 or 4), one
// lane = M / R threads.
//
// Every pass gives each thread one group of R elements {base + r L, r < R} in
// registers (base = R L (t / L) + t mod L for thread t), so a transform takes
// ceil(LOGM / LR) shared-memory passes with compile-time strides instead of
// one pass per two radix-2 stages.  With j = t mod L and W_N = e^{-2 pi i/N}:
//   DIF pass (natural -> bit-reversed):  y_q = W_{RL}^{jq} sum_r a_r W_R^{rq},
//                                        stored at base + brev(q) L;
//   DIT pass (bit-reversed -> natural):  y_q = sum_r a_r W_{RL}^{j brev(r)} W_R^{brev(r) q},
//                                        stored at base + q L.
// DIF passes run with L = M/R, M/R^2, ... and a last pass of 2^(LOGM mod LR)
// points on L = 1 (several groups per thread); DIT passes run in the opposite
// order.  Both produce exactly the layouts of the radix-2 forms above (the
// same bit-reversed order), so the families are interchangeable.
// Twiddles of the pass with stride L > 1: tw[off(L) + (q - 1) L + j] = W_{RL}^{jq}
// (q = 1..R-1, j < L), tables of the passes in DIF order (fftr_tw_words entries).
// Element i of a buffer lives at slot sslot(i): the low four bits are XORed
// with bits 4-7 and 8-11, which spreads every access pattern of these kernels
// (passes of any stride, a thread's consecutive elements, bit-reversed and
// natural runs of consecutive indices) evenly over the 16 eight-byte bank
// pairs; a buffer of M elements takes M slots (M + 16 when slot M is used).

__device__ __forceinline__ int sslot(int i) { return (i & ~15) | ((i ^ (i >> 4) ^ (i >> 8)) & 15); }

__host__ __device__ constexpr int brev_bits(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// offset of the twiddle table of DIF pass P, and the total size
__host__ __device__ constexpr int fftr_tw_off(int LOGM, int LR, int P) {
  int o = 0;
  for (int i = 0; i < P; ++i) {
    const int L = (1 << LOGM) >> (LR * (i + 1));
    o += L > 1 ? ((1 << LR) - 1) * L : 0;
  }
  return o;
}
__host__ __device__ constexpr int fftr_tw_words(int LOGM, int LR) { return fftr_tw_off(LOGM, LR, LOGM / LR); }

template <typename T2>
__device__ __forceinline__ T2 cmk(decltype(T2::x) x, decltype(T2::x) y) {
  T2 r;
  r.x = x;
  r.y = y;
  return r;
}

// a * W_16^E for a compile-time E (cos and sin of multiples of pi/8)
template <int E, typename T2>
__device__ __forceinline__ T2 w16(T2 a) {
  using R = decltype(a.x);
  constexpr int e = E & 15;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 4) {
    return cmk<T2>(a.y, -a.x);
  } else if constexpr (e == 8) {
    return cmk<T2>(-a.x, -a.y);
  } else if constexpr (e == 12) {
    return cmk<T2>(-a.y, a.x);
  } else if constexpr ((e & 3) == 2) {  // |cos| = |sin| = sqrt(1/2)
    const R h = (R)0.70710678118654752440;
    constexpr int sc = (e == 2 || e == 14) ? 1 : -1;  // sign of cos(2 pi e / 16)
    constexpr int ss = (e == 2 || e == 6) ? 1 : -1;   // sign of sin(2 pi e / 16)
    const R u = sc > 0 ? a.x : -a.x, v = ss > 0 ? a.y : -a.y;      // c a.x, s a.y (over h)
    const R u2 = sc > 0 ? a.y : -a.y, v2 = ss > 0 ? a.x : -a.x;    // c a.y, s a.x (over h)
    return cmk<T2>(h * (u + v), h * (u2 - v2));
  } else {  // odd e: cos and sin are +-cos(pi/8), +-sin(pi/8)
    const R C8 = (R)0.92387953251128675613, S8 = (R)0.38268343236508977173;
    constexpr int q = e & 3;  // 1 or 3
    constexpr int quad = e >> 2;
    // angle 2 pi e / 16 = quad pi/2 + q pi/8
    R c = q == 1 ? C8 : S8, s = q == 1 ? S8 : C8;
    if constexpr (quad == 1) {
      const R t = c;
      c = -s;
      s = t;
    } else if constexpr (quad == 2) {
      c = -c;
      s = -s;
    } else if constexpr (quad == 3) {
      const R t = c;
      c = s;
      s = -t;
    }
    // a * (c - i s)
    return cmk<T2>(a.x * c + a.y * s, a.y * c - a.x * s);
  }
}

template <typename T2>
__device__ __forceinline__ void dft2r(T2 &x0, T2 &x1) {
  const T2 t = x0;
  x0 = cadd(t, x1);
  x1 = csub(t, x1);
}
template <typename T2>
__device__ __forceinline__ void dft4r(T2 &x0, T2 &x1, T2 &x2, T2 &x3) {
  const T2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = cmul_negi(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

// y = DFT_R(a) for R = 2, 4, 8, 16 (natural order in and out; a is clobbered)
template <int R, typename T2>
__device__ __forceinline__ void dft_nat(T2 *a, T2 *y) {
  if constexpr (R == 2) {
    dft2r(a[0], a[1]);
    y[0] = a[0];
    y[1] = a[1];
  } else if constexpr (R == 4) {
    dft4r(a[0], a[1], a[2], a[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) y[q] = a[q];
  } else if constexpr (R == 8) {  // n = 2 n1 + n2, k = k1 + 4 k2
    dft4r(a[0], a[2], a[4], a[6]);
    dft4r(a[1], a[3], a[5], a[7]);
    a[3] = w16<2>(a[3]);
    a[5] = w16<4>(a[5]);
    a[7] = w16<6>(a[7]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft2r(a[2 * k1], a[2 * k1 + 1]);
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = a[2 * (q & 3) + (q >> 2)];
  } else {  // R == 16: n = 4 n1 + n2, k = k1 + 4 k2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4r(a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]);
    a[5] = w16<1>(a[5]);
    a[9] = w16<2>(a[9]);
    a[13] = w16<3>(a[13]);
    a[6] = w16<2>(a[6]);
    a[10] = w16<4>(a[10]);
    a[14] = w16<6>(a[14]);
    a[7] = w16<3>(a[7]);
    a[11] = w16<6>(a[11]);
    a[15] = w16<9>(a[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4r(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
#pragma unroll
    for (int q = 0; q < 16; ++q) y[q] = a[4 * (q & 3) + (q >> 2)];
  }
}

// The twiddles w[q] = W_{RL}^{jq}, q = 1 .. R-1, of a pass: the rows q = 1, 2,
// 4 (and 8) are read from the pass table, the others are products of at most
// three of them, which trades shared-memory loads (the transforms' bound)
// for a few multiplications.
template <typename T2, int R, int L>
__device__ __forceinline__ void pass_twiddles(const T2 *tw, int j, T2 *w) {
  w[1] = tw[j];
  if constexpr (R >= 4) {
    w[2] = tw[L + j];
    w[3] = cmul(w[1], w[2]);
  }
  if constexpr (R >= 8) {
    w[4] = tw[3 * L + j];
    w[5] = cmul(w[1], w[4]);
    w[6] = cmul(w[2], w[4]);
    w[7] = cmul(w[3], w[4]);
  }
  if constexpr (R >= 16) {
    w[8] = tw[7 * L + j];
#pragma unroll
    for (int q = 9; q < 16; ++q) w[q] = cmul(w[q - 8], w[8]);
  }
}

// One DIF pass of radix 2^LR and stride L; ZERO_UPPER: the inputs r >= R/2 are zero (not read).
template <typename T2, int LR, int L, bool ZERO_UPPER>
__device__ __forceinline__ void difr_pass(T2 *x, const T2 *tw, int t) {
  constexpr int R = 1 << LR;
  const int j = t & (L - 1);
  const int base = ((t - j) << LR) + j;
  T2 a[R], y[R];
#pragma unroll
  for (int r = 0; r < R; ++r) a[r] = (ZERO_UPPER && r >= R / 2) ? cmk<T2>(0, 0) : x[sslot(base + r * L)];
  dft_nat<R>(a, y);
  if constexpr (L > 1) {
    T2 w[R];
    pass_twiddles<T2, R, L>(tw, j, w);
#pragma unroll
    for (int q = 1; q < R; ++q) y[q] = cmul(y[q], w[q]);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) x[sslot(base + brev_bits(q, LR) * L)] = y[q];
}

// One DIT pass of radix 2^LR and stride L; HALF: only the outputs q < R/2 are stored.
template <typename T2, int LR, int L, bool HALF>
__device__ __forceinline__ void ditr_pass(T2 *x, const T2 *tw, int t) {
  constexpr int R = 1 << LR;
  const int j = t & (L - 1);
  const int base = ((t - j) << LR) + j;
  T2 a[R], b[R], y[R];
#pragma unroll
  for (int r = 0; r < R; ++r) a[r] = x[sslot(base + r * L)];
  if constexpr (L > 1) {
    T2 w[R];
    pass_twiddles<T2, R, L>(tw, j, w);
#pragma unroll
    for (int r = 1; r < R; ++r) a[r] = cmul(a[r], w[brev_bits(r, LR)]);
  }
#pragma unroll
  for (int s = 0; s < R; ++s) b[s] = a[brev_bits(s, LR)];
  dft_nat<R>(b, y);
#pragma unroll
  for (int q = 0; q < (HALF ? R / 2 : R); ++q) x[sslot(base + q * L)] = y[q];
}

// The pass of 2^RB points on L = 1 over a thread's E consecutive elements
template <typename T2, int E, int RB>
__device__ __forceinline__ void dif_tail(T2 *v) {  // in registers, DIF: out q of group g -> v[gR + brev(q)]
  constexpr int R = 1 << RB;
#pragma unroll
  for (int g = 0; g < E / R; ++g) {
    T2 a[R], y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = v[g * R + r];
    dft_nat<R>(a, y);
#pragma unroll
    for (int q = 0; q < R; ++q) v[g * R + brev_bits(q, RB)] = y[q];
  }
}
template <typename T2, int E, int RB>
__device__ __forceinline__ void dit_tail(T2 *v) {  // in registers, DIT: bit-reversed group -> natural
  constexpr int R = 1 << RB;
#pragma unroll
  for (int g = 0; g < E / R; ++g) {
    T2 a[R], y[R];
#pragma unroll
    for (int s = 0; s < R; ++s) a[s] = v[g * R + brev_bits(s, RB)];
    dft_nat<R>(a, y);
#pragma unroll
    for (int q = 0; q < R; ++q) v[g * R + q] = y[q];
  }
}

template <typename T2, int LOGM, int LR, int P, bool ZERO_FIRST>
__device__ __forceinline__ void difr_passes(T2 *x, const T2 *tw, int t, int last) {
  if constexpr (P < LOGM / LR) {
    if (P < last) {
      difr_pass<T2, LR, ((1 << LOGM) >> (LR * (P + 1))), ZERO_FIRST && P == 0>(x, tw + fftr_tw_off(LOGM, LR, P), t);
      __syncthreads();
    }
    difr_passes<T2, LOGM, LR, P + 1, ZERO_FIRST>(x, tw, t, last);
  }
}
template <typename T2, int LOGM, int LR, int P, bool HALF_LAST, int PLO = 0>
__device__ __forceinline__ void ditr_passes(T2 *x, const T2 *tw, int t, int first) {
  // runs P = first, first - 1, ..., PLO (L ascending)
  if constexpr (P >= PLO) {
    if (P <= first) {
      ditr_pass<T2, LR, ((1 << LOGM) >> (LR * (P + 1))), HALF_LAST && P == 0>(x, tw + fftr_tw_off(LOGM, LR, P), t);
      __syncthreads();
    }
    ditr_passes<T2, LOGM, LR, P - 1, HALF_LAST, PLO>(x, tw, t, first);
  }
}

// Natural order in, bit-reversed order out (slots sslot(i)); ends with a block barrier.
template <typename T2, int LOGM, int LR>
__device__ void fftr_dif(T2 *x, const T2 *tw, int t) {
  constexpr int NP = LOGM / LR, RB = LOGM % LR, E = 1 << LR;
  difr_passes<T2, LOGM, LR, 0, false>(x, tw, t, NP);
  if constexpr (RB > 0) {
    T2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = x[sslot(E * t + i)];
    dif_tail<T2, E, RB>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) x[sslot(E * t + i)] = v[i];
    __syncthreads();
  }
}

// Bit-reversed order in, natural order out; ends with a block barrier.
template <typename T2, int LOGM, int LR>
__device__ void fftr_dit(T2 *x, const T2 *tw, int t) {
  constexpr int NP = LOGM / LR, RB = LOGM % LR, E = 1 << LR;
  if constexpr (RB > 0) {
    T2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = x[sslot(E * t + i)];
    dit_tail<T2, E, RB>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) x[sslot(E * t + i)] = v[i];
    __syncthreads();
  }
  ditr_passes<T2, LOGM, LR, NP - 1, false>(x, tw, t, NP - 1);
}

// Bluestein core with the conventions of bluestein_conv: x <- FFT_M(conj(FFT_M(x) * bhat)),
// upper input half zero, lower output half computed.  The middle (last DIF
// pass, product with bhat in bit-reversed order, conjugation, first DIT pass)
// runs on each thread's E consecutive slots in registers.  bhat is stored
// transposed for these kernels, entry E t + i at i (M / E) + t, so that the
// threads of a warp read consecutive entries.
template <typename T2, int LOGM, int LR>
__device__ void bluesteinr(T2 *x, const T2 *tw, const T2 *__restrict__ bhat, int t) {
  constexpr int NP = LOGM / LR, RB = LOGM % LR, E = 1 << LR;
  constexpr int nfull = RB > 0 ? NP : NP - 1;  // full DIF passes outside the middle
  difr_passes<T2, LOGM, LR, 0, true>(x, tw, t, nfull);
  {
    T2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = x[sslot(E * t + i)];
    dif_tail<T2, E, (RB > 0 ? RB : LR)>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = cconj(cmul(v[i], bhat[i * ((1 << LOGM) >> LR) + t]));
    dit_tail<T2, E, (RB > 0 ? RB : LR)>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) x[sslot(E * t + i)] = v[i];
  }
  __syncthreads();
  ditr_passes<T2, LOGM, LR, NP - 1, true>(x, tw, t, nfull - 1);
}

// ---------------------------------------------------------------------------
// An inverse transform, a pointwise map of its output and the next forward
// transform, with the last pass of the first and the first pass of the second
// fused in registers.  The last DIT pass (P = 0, stride L = M / R) leaves
// elements t + q L (q < R, natural order) in thread t, and the first DIF pass
// (P = 0) reads exactly those elements, with the same twiddle row, so the map
// runs between them without going through shared memory: one read and one
// write of the buffer instead of three of each.

// The DIT transform without its last pass: the register tail and the passes
// P = NP - 1 .. 1; ends with a block barrier.
template <typename T2, int LOGM, int LR>
__device__ void fftr_dit_head(T2 *x, const T2 *tw, int t) {
  constexpr int NP = LOGM / LR, RB = LOGM % LR, E = 1 << LR;
  if constexpr (RB > 0) {
    T2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = x[sslot(E * t + i)];
    dit_tail<T2, E, RB>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) x[sslot(E * t + i)] = v[i];
    __syncthreads();
  }
  ditr_passes<T2, LOGM, LR, NP - 1, false, 1>(x, tw, t, NP - 1);
}

// The DIF transform without its first pass: P = 1 .. NP - 1 and the register
// tail; ends with a block barrier.
template <typename T2, int LOGM, int LR>
__device__ void fftr_dif_tail(T2 *x, const T2 *tw, int t) {
  constexpr int NP = LOGM / LR, RB = LOGM % LR, E = 1 << LR;
  difr_passes<T2, LOGM, LR, 1, false>(x, tw, t, NP);
  if constexpr (RB > 0) {
    T2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = x[sslot(E * t + i)];
    dif_tail<T2, E, RB>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) x[sslot(E * t + i)] = v[i];
    __syncthreads();
  }
}

// bluesteinr without its last DIT pass (P = 0).
template <typename T2, int LOGM, int LR>
__device__ void bluesteinr_head(T2 *x, const T2 *tw, const T2 *__restrict__ bhat, int t) {
  constexpr int NP = LOGM / LR, RB = LOGM % LR, E = 1 << LR;
  constexpr int nfull = RB > 0 ? NP : NP - 1;
  difr_passes<T2, LOGM, LR, 0, true>(x, tw, t, nfull);
  {
    T2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = x[sslot(E * t + i)];
    dif_tail<T2, E, (RB > 0 ? RB : LR)>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = cconj(cmul(v[i], bhat[i * ((1 << LOGM) >> LR) + t]));
    dit_tail<T2, E, (RB > 0 ? RB : LR)>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) x[sslot(E * t + i)] = v[i];
  }
  __syncthreads();
  ditr_passes<T2, LOGM, LR, NP - 1, true, 1>(x, tw, t, nfull - 1);
}

// bluesteinr without its first DIF pass (P = 0).
template <typename T2, int LOGM, int LR>
__device__ void bluesteinr_tail(T2 *x, const T2 *tw, const T2 *__restrict__ bhat, int t) {
  constexpr int NP = LOGM / LR, RB = LOGM % LR, E = 1 << LR;
  constexpr int nfull = RB > 0 ? NP : NP - 1;
  difr_passes<T2, LOGM, LR, 1, false>(x, tw, t, nfull);
  {
    T2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = x[sslot(E * t + i)];
    dif_tail<T2, E, (RB > 0 ? RB : LR)>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = cconj(cmul(v[i], bhat[i * ((1 << LOGM) >> LR) + t]));
    dit_tail<T2, E, (RB > 0 ? RB : LR)>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) x[sslot(E * t + i)] = v[i];
  }
  __syncthreads();
  ditr_passes<T2, LOGM, LR, NP - 1, true>(x, tw, t, nfull - 1);
}

// The fused pass: DIT pass P = 0, y_q <- f(q, y_q) for the output element
// t + q L, DIF pass P = 0 on the mapped values.  HALF (Bluestein): only the
// outputs q < R/2 are mapped, and the forward input is zero for q >= R/2.
// Each thread writes back only the slots it read, so no barrier is needed
// inside; the caller syncs after it.
template <typename T2, int LOGM, int LR, bool HALF, typename F>
__device__ __forceinline__ void fused_dit_dif(T2 *x, const T2 *tw, int t, F f) {
  constexpr int R = 1 << LR, L = (1 << LOGM) >> LR;
  T2 a[R], b[R];
#pragma unroll
  for (int r = 0; r < R; ++r) a[r] = x[sslot(t + r * L)];
  {
    T2 w[R];
    pass_twiddles<T2, R, L>(tw, t, w);
#pragma unroll
    for (int r = 1; r < R; ++r) a[r] = cmul(a[r], w[brev_bits(r, LR)]);
  }
#pragma unroll
  for (int s = 0; s < R; ++s) b[s] = a[brev_bits(s, LR)];
  dft_nat<R>(b, a);  // a[q]: output element t + q L
  // two elements at a time: the compiler barrier keeps the loads of the map
  // from being hoisted all at once (they would not fit the register budget)
#pragma unroll
  for (int q = 0; q < R; q += 2) {
    a[q] = (HALF && q >= R / 2) ? cmk<T2>(0, 0) : f(q, a[q]);
    a[q + 1] = (HALF && q + 1 >= R / 2) ? cmk<T2>(0, 0) : f(q + 1, a[q + 1]);
    asm volatile("" ::: "memory");
  }
  dft_nat<R>(a, b);
  {  // the same twiddle row, read again rather than held across the map
    T2 w[R];
    pass_twiddles<T2, R, L>(tw, t, w);
#pragma unroll
    for (int q = 1; q < R; ++q) b[q] = cmul(b[q], w[q]);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) x[sslot(t + brev_bits(q, LR) * L)] = b[q];
}

}  // namespace dmwf
