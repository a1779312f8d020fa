// dm_fft.cuh -- shared-memory FFT building blocks for the ring transforms.
//
// Every HEALPix ring of n = 4i pixels is transformed as a real sequence packed
// into a complex one of length h = n / 2.  h is a power of two for the
// equatorial belt when nside is; the other lengths (h = 2i) go through
// Bluestein's chirp-z convolution (Bluestein 1970) on a power-of-two size M.
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

template <typename T2, typename TW>
__device__ __forceinline__ T2 tw_cast(TW w) {
  T2 r;
  r.x = w.x;
  r.y = w.y;
  return r;
}

// In-place forward FFT (kernel e^{-2 pi i jk/M}) of length M = 2^k >= 1 held in
// shared memory, radix-2 decimation in time after a bit-reversal permutation.
// twid[k] = e^{-2 pi i k / Mtab}, k < Mtab / 2, Mtab a multiple of M.
// All threads of the block take part; the caller syncs before and after.
template <typename T2, typename TW>
__device__ void fft_pow2(T2 *x, int M, const TW *__restrict__ twid, int Mtab) {
  if (M <= 1) return;
  const int logM = 31 - __clz(M);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int j = (int)(__brev((unsigned)i) >> (32 - logM));
    if (j > i) {
      T2 t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  __syncthreads();
  for (int len = 1; len < M; len <<= 1) {
    const int tstride = Mtab / (2 * len);
    for (int k = threadIdx.x; k < (M >> 1); k += blockDim.x) {
      const int j = k & (len - 1);
      const int i0 = ((k - j) << 1) + j;
      const int i1 = i0 + len;
      T2 w = tw_cast<T2>(twid[j * tstride]);
      T2 u = x[i0];
      T2 v = cmul(x[i1], w);
      x[i0] = cadd(u, v);
      x[i1] = csub(u, v);
    }
    __syncthreads();
  }
}

// Forward DFT of length h (kernel e^{-2 pi i jk/h}) in place in x[0..h), x having
// room for M entries.  Power-of-two h: direct.  Otherwise Bluestein:
//   X_k = c_k sum_j (x_j c_j) conj(c_{k-j}),  c_j = e^{-i pi j^2 / h},
// the convolution done as IFFT_M(FFT_M(x c) * bhat) with bhat = FFT_M of the
// zero-padded conj(c) (precomputed).  ph[q] = e^{-i pi q / (2h)}, q < 4h, so
// c_j = ph[2 j^2 mod 4h].
template <typename T2, typename TW>
__device__ void dft_forward(T2 *x, int h, int M, int bluestein, const TW *__restrict__ ph,
                            const TW *__restrict__ bhat, const TW *__restrict__ twid, int Mtab) {
  if (!bluestein) {
    fft_pow2(x, h, twid, Mtab);
    return;
  }
  const int64_t n2 = 4LL * h;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    if (j < h) {
      T2 c = tw_cast<T2>(ph[(2LL * j * j) % n2]);
      x[j] = cmul(x[j], c);
    } else {
      x[j].x = 0;
      x[j].y = 0;
    }
  }
  __syncthreads();
  fft_pow2(x, M, twid, Mtab);
  for (int k = threadIdx.x; k < M; k += blockDim.x) x[k] = cconj(cmul(x[k], tw_cast<T2>(bhat[k])));
  __syncthreads();
  fft_pow2(x, M, twid, Mtab);
  const auto inv = (decltype(x[0].x))1 / (decltype(x[0].x))M;
  for (int k = threadIdx.x; k < h; k += blockDim.x) {
    T2 c = tw_cast<T2>(ph[(2LL * k * k) % n2]);
    T2 v = cconj(x[k]);
    v.x *= inv;
    v.y *= inv;
    x[k] = cmul(v, c);
  }
  __syncthreads();
}

}  // namespace dmwf
