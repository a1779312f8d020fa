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
// size-M transform takes ceil(log2 M / 2) barriers.
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

}  // namespace dmwf
