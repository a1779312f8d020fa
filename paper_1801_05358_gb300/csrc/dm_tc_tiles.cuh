// dm_tc_tiles.cuh -- tile helpers shared by the tensor-core Legendre stages
// (stored tables in dm_legendre_tc.cu, tiles generated in the kernel in
// dm_legendre_otf.cu): the K-major core-matrix row stores, the three-product
// BF16 hi/lo MMA, the per-m step and tile counts, and the launch arithmetic.
#pragma once

#include "dm_internal.h"
#include "dm_tc.cuh"

namespace dmwf {
namespace {

using namespace tc;

constexpr int TILE_A = 4096;  // 128 x 16 BF16

__device__ __forceinline__ int64_t abase(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// byte offset of the 16-byte core-matrix row (row, k-octet ko) of a [rows x 16] K-major tile
__device__ __forceinline__ uint32_t crow(int row, int ko) {
  return (uint32_t)((row >> 3) * 256 + ko * 128 + (row & 7) * 16);
}

__device__ __forceinline__ void put_row(unsigned char *tile, int tile_bytes, int row, int ko, const float x[8]) {
  uint4 h, l;
  split8(x, h, l);
  *reinterpret_cast<uint4 *>(tile + crow(row, ko)) = h;
  *reinterpret_cast<uint4 *>(tile + tile_bytes + crow(row, ko)) = l;
}

__device__ __forceinline__ void mma3(uint32_t d, const unsigned char *a, const unsigned char *b, int tile_b,
                                     uint32_t idesc, uint32_t acc) {
  const uint64_t ah = smem_desc(smem_u32(a)), al = smem_desc(smem_u32(a + TILE_A));
  const uint64_t bh = smem_desc(smem_u32(b)), bl = smem_desc(smem_u32(b + tile_b));
  mma_bf16(d, ah, bh, idesc, acc);
  mma_bf16(d, ah, bl, idesc, 1u);
  mma_bf16(d, al, bh, idesc, 1u);
}

__device__ __forceinline__ void tc_teardown(uint32_t tbase, uint32_t ncols) {
  fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tbase, ncols);
}

}  // namespace

__host__ __device__ inline int syn_steps(int lmax, int m) { return (lmax - m + 1 + 31) / 32; }
__host__ __device__ inline int ana_nl(int lmax, int m, int par) { return (lmax - m + 1 - par + 1) / 2; }
__host__ __device__ inline int ana_tiles(int lmax, int m, int par) {
  const int nl = ana_nl(lmax, m, par);
  return nl > 0 ? (nl + 127) / 128 : 0;
}

// 8 ring pairs (north, south) of one field, as 16 float2; zero past npairs, no
// south ring at the equator pair.
__device__ __forceinline__ void load_pairs8(const float2 *__restrict__ g, int pair0, int npairs, float2 v[16]) {
  if (pair0 + 8 < npairs) {
    const float4 *g4 = reinterpret_cast<const float4 *>(g + 2 * (int64_t)pair0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 q = g4[i];
      v[2 * i] = make_float2(q.x, q.y);
      v[2 * i + 1] = make_float2(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int pair = pair0 + i;
      v[2 * i] = pair < npairs ? g[2 * (int64_t)pair] : make_float2(0.f, 0.f);
      v[2 * i + 1] = pair < npairs - 1 ? g[2 * (int64_t)pair + 1] : make_float2(0.f, 0.f);
    }
  }
}

// Analysis B operand, split in two so that the loads of step c + 1 are in
// flight while step c is converted and multiplied.  One task per thread at
// most (PART 0: 2B tasks, PART 1: 4B tasks, B <= 64).
//  PART 0 task = (b / 4) * 8 + (b & 3) * 2 + ko: rows 2b, 2b + 1
//  PART 1 task = (b / 2) * 8 + (b & 1) * 4 + f * 2 + ko, f = 0 (Q) / 1 (U)
template <int PART>
__device__ __forceinline__ void load_ana_b(int task, const float2 *__restrict__ rc, int m, int c, int mmax,
                                           int npairs, float2 v[16]) {
  const int ko = task & 1;
  const int b = PART == 0 ? (task >> 3) * 4 + ((task >> 1) & 3) : (task >> 3) * 2 + ((task >> 2) & 1);
  const int f = PART == 0 ? 0 : 1 + ((task >> 1) & 1);
  load_pairs8(rc + (((int64_t)b * 3 + f) * (mmax + 1) + m) * npairs * 2, 16 * c + 8 * ko, npairs, v);
}

template <int PART>
__device__ __forceinline__ void convert_ana_b(int task, unsigned char *Bbuf, int tileB, int par, const float2 v[16]) {
  const float sgn = par == 0 ? 1.f : -1.f;  // G_par = G_N + sgn G_S
  const int ko = task & 1;
  if (PART == 0) {
    const int b = (task >> 3) * 4 + ((task >> 1) & 3);
    float re[8], im[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      re[i] = v[2 * i].x + sgn * v[2 * i + 1].x;
      im[i] = v[2 * i].y + sgn * v[2 * i + 1].y;
    }
    put_row(Bbuf, tileB, 2 * b + ko, ko, ko ? im : re);
    put_row(Bbuf, tileB, 2 * b + (ko ^ 1), ko, ko ? re : im);
  } else {
    const int f = (task >> 1) & 1, b = (task >> 3) * 2 + ((task >> 2) & 1);
    float a0[8], a1[8], b0[8], b1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float pr = v[2 * i].x + sgn * v[2 * i + 1].x, pi = v[2 * i].y + sgn * v[2 * i + 1].y;  // this parity
      const float orr = v[2 * i].x - sgn * v[2 * i + 1].x, oi = v[2 * i].y - sgn * v[2 * i + 1].y;  // opposite
      // B1: Q -> rows 4b (-Qp.re), 4b+1 (-Qp.im); U -> rows 4b+2 (-Up.re), 4b+3 (-Up.im)
      a0[i] = -pr;
      a1[i] = -pi;
      // B2: U -> rows 4b (Uo.im), 4b+1 (-Uo.re); Q -> rows 4b+2 (-Qo.im), 4b+3 (Qo.re)
      b0[i] = f == 1 ? oi : -oi;
      b1[i] = f == 1 ? -orr : orr;
    }
    unsigned char *B1 = Bbuf, *B2 = Bbuf + 2 * tileB;
    const int r1 = 4 * b + 2 * f, r2 = 4 * b + 2 * (1 - f);
    put_row(B1, tileB, r1 + ko, ko, ko ? a1 : a0);
    put_row(B1, tileB, r1 + (ko ^ 1), ko, ko ? a0 : a1);
    put_row(B2, tileB, r2 + ko, ko, ko ? b1 : b0);
    put_row(B2, tileB, r2 + (ko ^ 1), ko, ko ? b0 : b1);
  }
}

static inline uint32_t pow2_cols(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

// smem per CTA for NS stages, raised when needed so that the CTAs sharing an
// SM never ask for more tensor memory than its 512 columns
static inline size_t tc_smem_n(int stage_bytes, int ns, uint32_t ncols) {
  size_t s = (size_t)ns * stage_bytes + 1024;
  const int per_sm = (int)(512 / ncols);
  const size_t floor_bytes = (232448 / (per_sm + 1)) + 1024;
  return s > floor_bytes ? s : floor_bytes;
}

}  // namespace dmwf
