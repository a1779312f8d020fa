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

}  // namespace dmwf
