// dm_legendre_otf.cu -- the tensor-core Legendre stages with the Legendre
// tiles generated inside the kernels, in place of the stored BF16 tables.
//
// The contractions are those of dm_legendre_tc.cu: the same GEMM shapes, the
// same BF16 hi/lo three-product scheme with FP32 accumulation in tensor
// memory, the same epilogues.  Only the A operand changes.  For every
// (m, block of CKL = 64 multipoles, ring pair) the set-up stores the state of
// the FP64 recurrence at the block's first multipole (two consecutive values
// of lambda, of 2lambda / 2 and of -2lambda / 2), rounded to FP32 with a
// power-of-two scale 2^-S for the values that FP32 cannot hold.  The kernels
// restart the recurrence there and advance it in FP32.  Two forms of the
// step keep the FP32 drift over a block to a few units in the sixth digit or
// less, below the ~16 bits that the BF16 hi/lo split carries:
// - rings with x = cos(theta) < 3/4 advance lambda_{l+1} = al x lambda_l -
//   bl lambda_{l-1} with x lambda_l in float-float (x = x_hi + x_lo), so that
//   the rounding of x does not perturb every step the same way;
// - nearer the poles the two roots of the recurrence's characteristic
//   equation approach each other (a double root at x = 1) and step rounding
//   grows quadratically over a block (1e-4 at the polar rings in 64 steps).
//   There the state is (lambda_l, D_l = lambda_l - lambda_{l-1}) and
//   D_{l+1} = bl D_l + (al - 1 - bl - al u) lambda_l, lambda_{l+1} =
//   lambda_l + D_{l+1}, u = 1 - x taken without cancellation: every rounding
//   then enters at the size of the (small) increment.  The spin-2 recurrences
//   take the same two forms with (a x +- ac, b).
// The form is chosen per octet of ring pairs by the first pair's x.  The
// checkpoints take 32 bytes per (m, block, pair), about 1/64 of the tables
// they replace.
//
// Synthesis (grid: pair tiles x m): four generator warps, one thread per ring
// pair, continue the recurrence through the K steps in order and store each
// parity tile's 8 consecutive multipoles as one 16-byte core-matrix row; one
// thread bulk-copies the B operand (the iterate, converted once per iteration
// by k_syn_b) and issues the MMAs.
// Analysis (grid: l-tile groups x parity x m): the contraction runs over ring
// pairs, so the recurrence direction is the MMA's M dimension.  A worker warp
// takes one K step (16 ring pairs) at a time: each lane restarts the
// recurrence of 8 pairs at one checkpoint block and stores the block's 32
// rows of this parity, one 16-byte row (8 pairs) per multipole, and the warp
// converts the step's ring coefficients into the B operand.  Spin 2 uses
// p = 2lambda / 2 and q = -2lambda / 2 as its two A tiles with B operands
// B1 + B2 and B1 - B2, since lam+ B1 + lam- B2 = p (B1 + B2) + q (B1 - B2).
#include <algorithm>
#include <vector>

#include "dm_internal.h"
#include "dm_rec.cuh"
#include "dm_tc.cuh"
#include "dm_tc_tiles.cuh"

namespace dmwf {

using namespace tc;

namespace {

constexpr int CKL = 64;  // multipoles per checkpoint block

// 2^-S as a float for 0 <= S <= 126; zero beyond (a value below 2^-126 of the
// functions' O(1) range is negligible, and the stored tables flush it too)
__device__ __forceinline__ float scale_of(int S) {
  return S <= 0 ? 1.f : (S < 127 ? __int_as_float((127 - S) << 23) : 0.f);
}

// An FP64 state v[0..n) carried as v 2^-S64 -> FP32 values out and a scale
// S32 >= 0 with true = out 2^-S32; out is normalised to [1, 2) in magnitude
// whenever a scale is needed.
__device__ void to_fp32_state(const double *v, int n, int S64, float *out, int &S32) {
  double M = 0.0;
  for (int i = 0; i < n; ++i) M = fmax(M, fabs(v[i]));
  S32 = 0;
  if (M == 0.0) {
    for (int i = 0; i < n; ++i) out[i] = 0.f;
    return;
  }
  const int e = ilogb(M);
  if (S64 == 0 && e >= -60) {
    for (int i = 0; i < n; ++i) out[i] = (float)v[i];
    return;
  }
  if (S64 - e <= 0) {  // representable after all
    for (int i = 0; i < n; ++i) out[i] = (float)ldexp(v[i], -S64);
    return;
  }
  S32 = S64 - e;
  for (int i = 0; i < n; ++i) out[i] = (float)ldexp(v[i], -e);
}

// Ring pairs whose octet starts at x >= 3/4 run the difference form.
__host__ __device__ __forceinline__ bool pair_dform(const PairDev *pairs, int p) { return pairs[p & ~7].x >= 0.75; }

// Per-pair constants of the step: x = xh + xl and u = 1 - x.
struct Xs {
  float xh, xl, u;
};
__device__ __forceinline__ Xs xs_of(const PairDev *pairs, int p) {
  const PairDev q = pairs[p];
  Xs r;
  r.xh = (float)q.x;
  r.xl = (float)(q.x - (double)r.xh);
  r.u = (float)q.omz;
  return r;
}

// Checkpoints: one thread per (pair, m) runs the FP64 recurrence of every
// Legendre kernel (dm_rec.cuh) from l = m and stores its state at the start
// of each block, l = m + CKL j.  The spin-2 state of block 0 is taken at
// l = max(m, 2), where its recurrence starts.
__global__ void __launch_bounds__(128) k_ckpt(const PairDev *__restrict__ pairs, const RecCoef *__restrict__ rec,
                                              const double *__restrict__ seed, const int *__restrict__ seed_exp,
                                              const int64_t *__restrict__ cko, float4 *__restrict__ ck0,
                                              float4 *__restrict__ ck2, int lmax, int npairs) {
  const int m = blockIdx.y, p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const double x = pairs[p].x;
  const bool dform = pair_dform(pairs, p);
  Rec s;
  rec_init(s, seed, seed_exp, m, p, npairs);
  const int64_t base = abase(lmax, m);
  for (int l = m; l <= lmax; ++l) {
    const int j = (l - m) / CKL;
    const int64_t o = (cko[m] + j) * (int64_t)npairs + p;
    if (l == m + CKL * j) {
      const double v[2] = {s.l0, dform ? s.l0 - s.l1 : s.l1};
      float f[2];
      int S0;
      to_fp32_state(v, 2, s.S, f, S0);
      ck0[o] = make_float4(f[0], f[1], __int_as_float(S0), __int_as_float(0));
    }
    if (l == (j == 0 ? max(m, 2) : m + CKL * j)) {
      const double v[4] = {0.5 * s.p0, 0.5 * (dform ? s.p0 - s.p1 : s.p1), 0.5 * s.q0,
                           0.5 * (dform ? s.q0 - s.q1 : s.q1)};
      float f[4];
      int S2;
      to_fp32_state(v, 4, s.S, f, S2);
      ck2[o] = make_float4(f[0], f[1], f[2], f[3]);
      reinterpret_cast<float *>(ck0 + o)[3] = __int_as_float(S2);
    }
    if (l < lmax) rec_advance(s, rec[base + l + 1], x, m, l, seed, p, npairs);
  }
}

// FP32 coefficients of target l: (al, bl, al - 1 - bl), (a, ac, b) and
// (a + ac - 1 - b, a - ac - 1 - b), the differences formed in FP64
__global__ void k_rec32(const RecCoef *__restrict__ rec, float4 *__restrict__ rq0, float4 *__restrict__ rq2,
                        float2 *__restrict__ rq2d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const RecCoef c = rec[i];
    rq0[i] = make_float4((float)c.al, (float)c.bl, (float)(c.al - 1.0 - c.bl), 0.f);
    rq2[i] = make_float4((float)c.a, (float)c.ac, (float)c.b, 0.f);
    rq2d[i] = make_float2((float)(c.a + c.ac - 1.0 - c.b), (float)(c.a - c.ac - 1.0 - c.b));
  }
}

// One step of one recurrence to target l + 1.  Standard form, state
// (v_l, v_{l-1}): v_{l+1} = (c x + k) v_l - b v_{l-1} with the product by x in
// float-float.  Difference form, state (v_l, D_l): D_{l+1} = b D_l +
// (d - c u) v_l, v_{l+1} = v_l + D_{l+1}.  Spin 0: c = al, k = 0, b = bl,
// d = al - 1 - bl; spin 2: c = a, k = +-ac, b = b, d = a +- ac - 1 - b.
template <bool DF>
__device__ __forceinline__ void step(float &v0, float &v1, float c, float k, float b, float d, const Xs &x) {
  if (DF) {
    const float g = fmaf(-c, x.u, d);
    v1 = fmaf(b, v1, g * v0);
    v0 = v0 + v1;
  } else {
    const float n = fmaf(fmaf(c, x.xh, k), v0, fmaf(c * x.xl, v0, -b * v1));
    v1 = v0;
    v0 = n;
  }
}

// Scaled state (S > 0, values far below FP32 range): once the running value
// has grown past 2^32, move 2^32 of it (or all of the scale) into the values.
__device__ __forceinline__ void rescale(float &a0, float &a1, float &b0, float &b1, int &S, float &sc) {
  if (S > 32) {
    a0 *= 0x1p-32f;
    a1 *= 0x1p-32f;
    b0 *= 0x1p-32f;
    b1 *= 0x1p-32f;
    S -= 32;
  } else {
    const float f = scale_of(S);
    a0 *= f;
    a1 *= f;
    b0 *= f;
    b1 *= f;
    S = 0;
  }
  sc = scale_of(S);
}


// ------------------------------------------------------------------ analysis
// A tiles of the analysis: 128 multipoles x 16 ring pairs, K-major core
// matrices, 8-row groups ASBO = 272 bytes apart instead of 256 and each tile
// of a stage 16 bytes further along: the lanes of a worker warp store rows
// 32 q + x of several tiles at once, and these offsets spread them over all
// eight 16-byte bank groups (four stores per wavefront, the minimum).
constexpr int ASBO = 272;
constexpr int ATILE = 16 * ASBO;         // one of hi / lo
constexpr int ATS = 2 * ATILE + 16;      // hi + lo + the 16-byte shift
constexpr int AGEN_THREADS = 192;        // 5 worker warps at most + the MMA warp
constexpr int AGEN_MAX_S = 5;

__device__ __forceinline__ uint64_t smem_desc_sbo(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;  // next K core matrix
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;   // next 8-row group
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void mma3_a(uint32_t d, const unsigned char *a, const unsigned char *b, int tile_b,
                                       uint32_t idesc, uint32_t acc) {
  const uint64_t ah = smem_desc_sbo(smem_u32(a), ASBO), al = smem_desc_sbo(smem_u32(a + ATILE), ASBO);
  const uint64_t bh = smem_desc(smem_u32(b)), bl = smem_desc(smem_u32(b + tile_b));
  mma_bf16(d, ah, bh, idesc, acc);
  mma_bf16(d, ah, bl, idesc, 1u);
  mma_bf16(d, al, bh, idesc, 1u);
}

// Spin-2 B operands of one task (RHS b, k-octet ko) in the p / q form:
// rows 4b + k of B1' = B1 + B2 and B2' = B1 - B2, with (P = this parity,
// O = the opposite one, of the fields Q and U)
//   k = 0: -Qp.re + Uo.im | -Qp.re - Uo.im      k = 1: -Qp.im - Uo.re | -Qp.im + Uo.re
//   k = 2: -Up.re - Qo.im | -Up.re + Qo.im      k = 3: -Up.im + Qo.re | -Up.im - Qo.re
// The four rows go out in an order rotated by (b >> 1) & 3, so that the lanes
// of a warp hit all eight bank groups.
__device__ __forceinline__ void convert_b_pq(int b, int ko, unsigned char *B1, unsigned char *B2, int tileB,
                                             int par, const float2 vq[16], const float2 vu[16]) {
  const float sgn = par == 0 ? 1.f : -1.f;
  const int rot = (b >> 1) & 3;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int kk = (k + rot) & 3;
    const bool qrow = kk < 2, im = (kk & 1) != 0;
    const float s2 = (kk == 0 || kk == 3) ? 1.f : -1.f;
    float r1[8], r2[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 n1 = qrow ? vq[2 * i] : vu[2 * i], s1 = qrow ? vq[2 * i + 1] : vu[2 * i + 1];
      const float2 n2 = qrow ? vu[2 * i] : vq[2 * i], s2v = qrow ? vu[2 * i + 1] : vq[2 * i + 1];
      const float first = -((im ? n1.y : n1.x) + sgn * (im ? s1.y : s1.x));  // -(this parity).comp
      const float sec = s2 * ((im ? n2.x : n2.y) - sgn * (im ? s2v.x : s2v.y));  // +-(opposite).other comp
      r1[i] = first + sec;
      r2[i] = first - sec;
    }
    put_row(B1, tileB, 4 * b + kk, ko, r1);
    put_row(B2, tileB, 4 * b + kk, ko, r2);
  }
}

// BF16 hi / lo of N consecutive values (N = 1, 2, 4, 8 ring pairs of one
// core-matrix row), stored at byte offset o of the hi tile and of the lo tile.
template <int N>
__device__ __forceinline__ void put_vals(unsigned char *tile, uint32_t o, const float *x) {
  if (N == 1) {
    uint16_t h, l;
    split1(x[0], h, l);
    *reinterpret_cast<uint16_t *>(tile + o) = h;
    *reinterpret_cast<uint16_t *>(tile + ATILE + o) = l;
  } else {
    constexpr int H = N > 1 ? N / 2 : 1;
    uint32_t h[H], l[H];
#pragma unroll
    for (int i = 0; i < N / 2; ++i) split2(x[2 * i], x[2 * i + 1], h[i], l[i]);
    if (N == 2) {
      *reinterpret_cast<uint32_t *>(tile + o) = h[0];
      *reinterpret_cast<uint32_t *>(tile + ATILE + o) = l[0];
    } else if (N == 4) {
      *reinterpret_cast<uint2 *>(tile + o) = make_uint2(h[0], h[1]);
      *reinterpret_cast<uint2 *>(tile + ATILE + o) = make_uint2(l[0], l[1]);
    } else {
      *reinterpret_cast<uint4 *>(tile + o) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4 *>(tile + ATILE + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
}

__device__ __forceinline__ uint32_t arow(int row) { return (uint32_t)((row >> 3) * ASBO + (row & 7) * 16); }

// Slot of the k-th staged coefficient: one slot of padding every 64, so that
// lanes on different checkpoint blocks (64 targets apart) read different
// bank groups.
__device__ __forceinline__ int cpad(int k) { return k + (k >> 6); }
__host__ __device__ inline int coef_slots(int LT) { return 256 * LT + 4 * LT + 1; }

// One lane's share of a K step's A operand: the rows of parity PAR of
// checkpoint block J (l0 = its first multipole, tile rows 32 q ..) for the
// PPL ring pairs p0 .. p0 + PPL - 1, at byte offset obase of each row; f
// selects the spin-2 function (p or q).  Rows past lmax are left as they
// are: they only reach accumulator rows that the epilogue drops.  The
// coefficients of the next step are loaded one step ahead.
template <int PART, bool DF, int PAR, int PPL>
__device__ __forceinline__ void ana_task(unsigned char *At, int q, uint32_t obase, int l0, int lmax, int ls, int f,
                                         const float4 *__restrict__ ck0, const float4 *__restrict__ ck2,
                                         int64_t orow, const PairDev *__restrict__ pairs, int p0, int npairs,
                                         const float4 *sA, const float2 *sD, int tlo) {
  float v0[PPL], v1[PPL], sc[PPL];
  Xs xs[PPL];
  int Sk[PPL];
  int anyS = 0;
#pragma unroll
  for (int i = 0; i < PPL; ++i) {
    const int pp = min(p0 + i, npairs - 1);
    xs[i] = xs_of(pairs, pp);
    const float4 r0 = ck0[orow + pp];
    if (PART == 0) {
      v0[i] = r0.x;
      v1[i] = r0.y;
      Sk[i] = __float_as_int(r0.z);
    } else {
      const float4 r2 = ck2[orow + pp];
      v0[i] = f == 0 ? r2.x : r2.z;
      v1[i] = f == 0 ? r2.y : r2.w;
      Sk[i] = __float_as_int(r0.w);
    }
    sc[i] = scale_of(Sk[i]);
    anyS |= Sk[i];
  }
  const int nv = min(CKL, lmax - l0 + 1);  // multipoles of the block up to lmax
  const int t0 = max(0, ls - l0);          // spin 2 starts at l = 2
  for (int t = PAR; t < t0 && t < nv; t += 2) {
    const float z[PPL] = {};
    put_vals<PPL>(At, arow(32 * q + (t >> 1)) + obase, z);
  }
  auto coef = [&](int l, float &c, float &k, float &b, float &d) {  // coefficients of target l + 1 (shared memory)
    const int q = cpad(l + 1 - tlo);
    const float4 cf = sA[q];
    if (PART == 0) {
      c = cf.x;
      k = 0.f;
      b = cf.y;
      d = cf.z;
    } else {
      c = cf.x;
      k = f ? -cf.y : cf.y;
      b = cf.z;
      d = 0.f;
      if (DF) {
        const float2 dd = sD[q];
        d = f ? dd.y : dd.x;
      }
    }
  };
  float c = 0.f, k = 0.f, b = 0.f, d = 0.f;
  if (t0 + 1 < nv) coef(l0 + t0, c, k, b, d);
  for (int t = t0; t < nv; ++t) {
    float cn = 0.f, kn = 0.f, bn = 0.f, dn = 0.f;
    if (t + 2 < nv) coef(l0 + t + 1, cn, kn, bn, dn);
    if ((t & 1) == PAR) {
      float x[PPL];
#pragma unroll
      for (int i = 0; i < PPL; ++i) x[i] = v0[i] * sc[i];
      put_vals<PPL>(At, arow(32 * q + (t >> 1)) + obase, x);
    }
    if (t + 1 < nv) {
#pragma unroll
      for (int i = 0; i < PPL; ++i) step<DF>(v0[i], v1[i], c, k, b, d, xs[i]);
      if (anyS) {
        anyS = 0;
#pragma unroll
        for (int i = 0; i < PPL; ++i) {
          if (Sk[i] > 0 && fabsf(v0[i]) > 0x1p32f) {
            float d0 = 0.f, d1 = 0.f;
            rescale(v0[i], v1[i], d0, d1, Sk[i], sc[i]);
          }
          anyS |= Sk[i];
        }
      }
    }
    c = cn;
    k = kn;
    b = bn;
    d = dn;
  }
}

template <int PART, bool DF, int PAR>
__device__ __forceinline__ void ana_task_ppl(int PPL, unsigned char *At, int q, uint32_t obase, int l0, int lmax,
                                             int ls, int f, const float4 *ck0, const float4 *ck2, int64_t orow,
                                             const PairDev *pairs, int p0, int npairs, const float4 *sA,
                                             const float2 *sD, int tlo) {
  switch (PPL) {
    case 8:
      ana_task<PART, DF, PAR, 8>(At, q, obase, l0, lmax, ls, f, ck0, ck2, orow, pairs, p0, npairs, sA, sD,
                                 tlo);
      break;
    case 4:
      ana_task<PART, DF, PAR, 4>(At, q, obase, l0, lmax, ls, f, ck0, ck2, orow, pairs, p0, npairs, sA, sD,
                                 tlo);
      break;
    case 2:
      ana_task<PART, DF, PAR, 2>(At, q, obase, l0, lmax, ls, f, ck0, ck2, orow, pairs, p0, npairs, sA, sD,
                                 tlo);
      break;
    default:
      ana_task<PART, DF, PAR, 1>(At, q, obase, l0, lmax, ls, f, ck0, ck2, orow, pairs, p0, npairs, sA, sD,
                                 tlo);
  }
}

// Worker warps 0 .. S-1 own stage w and K steps c = w, w + S, ...; warp 5
// issues the MMAs; warps 0-3 read the accumulators after the single-use
// barrier fin.  PART 0: LT <= 4 l tiles, lane = (tile j, octet g, block q);
// PART 1: LT <= 2, lane = (j, g, q, function f: p or q).
template <int PART>
__global__ void __launch_bounds__(AGEN_THREADS, 1) k_ana_gen(
    const float4 *__restrict__ ck0, const float4 *__restrict__ ck2, const int64_t *__restrict__ cko,
    const float4 *__restrict__ rq0, const float4 *__restrict__ rq2, const float2 *__restrict__ rq2d,
    const PairDev *__restrict__ pairs,
    const float2 *__restrict__ rc, float2 *__restrict__ out, int lmax, int mmax, int npairs, int64_t nalm, int B,
    int LT, uint32_t ncols, int S, int *err, int withhold) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bars[2 * AGEN_MAX_S + 1];
  __shared__ uint32_t tslot;
  uint64_t *full = bars, *done = bars + AGEN_MAX_S, *fin = bars + 2 * AGEN_MAX_S;
  const int m = blockIdx.z, par = blockIdx.y;
  const int nl = ana_nl(lmax, m, par);
  const int lt0 = blockIdx.x * LT;
  const int nt = min(LT, (nl > 0 ? (nl + 127) / 128 : 0) - lt0);
  if (nt <= 0) return;  // uniform over the block
  const int NC = (PART == 0) ? 2 * B : 4 * B;
  constexpr int nA = (PART == 0) ? 1 : 2;
  const int tileB = NC * 32;
  const int a_area = ((LT * nA * ATS) + 1023) & ~1023;
  const int stage = a_area + nA * 2 * tileB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the recurrence coefficients of this CTA's multipoles, staged once: every
  // worker walks the same range for every K step (targets tlo .. tlo + 256 nt - 1)
  const int ncs = coef_slots(LT);
  float4 *sA = reinterpret_cast<float4 *>(sm);
  float2 *sD = reinterpret_cast<float2 *>(sm + 16 * ncs);
  const int coef_bytes = ((ncs * (PART == 0 ? 16 : 24)) + 1023) & ~1023;
  unsigned char *stg = sm + coef_bytes;
  const int tlo = m + 256 * lt0 + 1;
  {
    const int64_t b0 = abase(lmax, m);
    for (int k = tid; k < 256 * nt; k += blockDim.x) {
      const int T = tlo + k;
      if (T > lmax) break;
      if (PART == 0) {
        sA[cpad(k)] = rq0[b0 + T];
      } else {
        sA[cpad(k)] = rq2[b0 + T];
        sD[cpad(k)] = rq2d[b0 + T];
      }
    }
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 32);
      mbar_init(&done[i], 1);
    }
    mbar_init(fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tslot, ncols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tslot;
  const int64_t base = abase(lmax, m);
  const int nsteps = (npairs + 15) / 16;
  const int nblk = (lmax - m + 1 + CKL - 1) / CKL;
  if (warp < S) {
    // This CTA's checkpoint blocks: J = 4 lt0 + bi for bi < nvalid.  A lane
    // takes PPL pairs of one octet g of one block bi (and one spin-2 function
    // f); PPL is the fewest pairs per lane that still covers every block with
    // the warp's 32 lanes: 8 at low m, down to 1 when few blocks remain.
    constexpr int nf = PART == 0 ? 1 : 2;
    const int nvalid = max(0, min(4 * nt, nblk - 4 * lt0));
    int PPL = 1;
    while (PPL < 8 && nvalid * 2 * (8 / PPL) * nf > 32) PPL *= 2;
    const int sub = 8 / PPL;
    const int sl = lane % sub, g = (lane / sub) & 1, f = PART == 0 ? 0 : (lane / (2 * sub)) & 1;
    const int bi = lane / (2 * sub * nf);
    const bool gen = bi < nvalid;
    const int J = 4 * lt0 + bi, j = bi >> 2, q = bi & 3;
    const int ls = (PART == 1 && m < 2 && J == 0) ? 2 : 0;
    const uint32_t obase = (uint32_t)(g * 128 + sl * PPL * 2);
    for (int c = warp; c < nsteps; c += S) {
      const int s = warp, k = c / S;
      if (k > 0 && !mbar_wait(&done[s], (k - 1) & 1, err)) break;
      unsigned char *Ast = stg + s * stage, *Bst = Ast + a_area;
      // B operand of this K step
      if (PART == 0) {
        for (int task = lane; task < 2 * B; task += 32) {
          float2 v[16];
          load_ana_b<0>(task, rc, m, c, mmax, npairs, v);
          convert_ana_b<0>(task, Bst, tileB, par, v);
        }
      } else {
        for (int task = lane; task < 2 * B; task += 32) {
          const int b = task >> 1, ko = task & 1;
          float2 vq[16], vu[16];
          const int64_t fq = (((int64_t)b * 3 + 1) * (mmax + 1) + m) * npairs * 2;
          const int64_t fu = (((int64_t)b * 3 + 2) * (mmax + 1) + m) * npairs * 2;
          load_pairs8(rc + fq, 16 * c + 8 * ko, npairs, vq);
          load_pairs8(rc + fu, 16 * c + 8 * ko, npairs, vu);
          convert_b_pq(b, ko, Bst, Bst + 2 * tileB, tileB, par, vq, vu);
        }
      }
      // A tile rows of block J, pairs 16 c + 8 g + PPL sl ..
      if (gen) {
        unsigned char *At = Ast + (j * nA + f) * ATS;
        const int p0 = 16 * c + 8 * g + PPL * sl;
        const int64_t orow = (cko[m] + J) * (int64_t)npairs;
        const bool df = pair_dform(pairs, min(16 * c + 8 * g, npairs - 1));
        const int l0 = m + CKL * J;
        if (df) {
          if (par == 0)
            ana_task_ppl<PART, true, 0>(PPL, At, q, obase, l0, lmax, ls, f, ck0, ck2, orow, pairs, p0, npairs, sA,
                                        sD, tlo);
          else
            ana_task_ppl<PART, true, 1>(PPL, At, q, obase, l0, lmax, ls, f, ck0, ck2, orow, pairs, p0, npairs, sA,
                                        sD, tlo);
        } else {
          if (par == 0)
            ana_task_ppl<PART, false, 0>(PPL, At, q, obase, l0, lmax, ls, f, ck0, ck2, orow, pairs, p0, npairs, sA,
                                         sD, tlo);
          else
            ana_task_ppl<PART, false, 1>(PPL, At, q, obase, l0, lmax, ls, f, ck0, ck2, orow, pairs, p0, npairs, sA,
                                         sD, tlo);
        }
      }
      fence_proxy_async();  // generic-proxy writes -> tensor-core reads
      // test hook (dm_test_tc_withhold): lane 0 of the first worker of the
      // first CTA withholds its arrival for the first K step; the MMA warp's
      // bounded wait then gives up with nothing asynchronous in flight
      if (!(withhold && c == 0 && lane == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0))
        mbar_arrive(&full[s]);
    }
  } else if (warp == 5 && lane == 0) {
    const uint32_t idesc = idesc_bf16(128, NC);
    for (int c = 0; c < nsteps; ++c) {
      const int s = c % S, k = c / S;
      if (!mbar_wait(&full[s], k & 1, err)) break;
      fence_after_sync();
      const unsigned char *Ast = stg + s * stage, *Bst = Ast + a_area;
      const uint32_t acc = c > 0 ? 1u : 0u;
      for (int j = 0; j < nt; ++j) {
        const uint32_t dj = tbase + (uint32_t)(j * NC);
        mma3_a(dj, Ast + (j * nA) * ATS, Bst, tileB, idesc, acc);
        if (PART == 1) mma3_a(dj, Ast + (j * nA + 1) * ATS, Bst + 2 * tileB, tileB, idesc, 1u);
      }
      commit(&done[s]);
    }
    commit(fin);
  }
  if (warp < 4) {
    mbar_wait(fin, 0, err);
    __syncwarp();
    fence_after_sync();
    const int row = warp * 32 + lane;
    const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);
    for (int j = 0; j < nt; ++j) {
      const int i = (lt0 + j) * 128 + row;
      const bool ok = i < nl;
      const int64_t idx = base + m + par + 2 * i;
      for (int c0 = 0; c0 < NC; c0 += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)(j * NC) + c0, v);
        if (!ok) continue;
        if (PART == 0) {
          for (int qq = 0; qq < 8; ++qq) {
            const int b = (c0 >> 1) + qq;
            out[((int64_t)b * 3 + 0) * nalm + idx] = make_float2(v[2 * qq], v[2 * qq + 1]);
          }
        } else {
          for (int qq = 0; qq < 4; ++qq) {
            const int b = (c0 >> 2) + qq;
            out[((int64_t)b * 3 + 1) * nalm + idx] = make_float2(v[4 * qq], v[4 * qq + 1]);
            out[((int64_t)b * 3 + 2) * nalm + idx] = make_float2(v[4 * qq + 2], v[4 * qq + 3]);
          }
        }
      }
    }
  }
  tc_teardown(tbase, ncols);
}

// ----------------------------------------------------------------- synthesis
constexpr int SGEN_MAX_NS = 8;

// One K step of the synthesis generator (thread = ring pair row r): the 32
// multipoles l = lb .. lb + 31, stored as the rows of the parity tiles (spin 0:
// lambda e, o in unit Ae; spin 2: {lam+ e, lam- o} in Ae, {lam+ o, lam- e} in
// Ao), the recurrence state carried on to the next step.
template <int PART>
__device__ __forceinline__ void syn_step(unsigned char *Ae, unsigned char *Ao, int r, int lb, int lmax, int ls,
                                         bool act, float &a0, float &a1, float &b0, float &b1, int &S, float &sc,
                                         const Xs &xs, bool df, float4 cA, float2 cD) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float ve[8], vo[8], we[8], wo[8];  // spin 0: lambda; spin 2: v = lam+, w = lam-
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int l = lb + 16 * h + t;
      const bool live = act && l <= lmax && l >= ls;
      float v, w = 0.f;
      if (PART == 0) {
        v = live ? a0 * sc : 0.f;
      } else {
        v = live ? (a0 + b0) * sc : 0.f;
        w = live ? (a0 - b0) * sc : 0.f;
      }
      if (t & 1) {
        vo[t >> 1] = v;
        wo[t >> 1] = w;
      } else {
        ve[t >> 1] = v;
        we[t >> 1] = w;
      }
      // the coefficients of target l + 1, held by lane 16 h + t of the warp;
      // every lane takes part in the shuffles (the form is chosen after them,
      // per lane: a warp can hold ring pairs of both forms)
      const int src = 16 * h + t;
      const float c0 = __shfl_sync(0xffffffffu, cA.x, src), c1 = __shfl_sync(0xffffffffu, cA.y, src);
      const float c2 = __shfl_sync(0xffffffffu, cA.z, src);
      float dp = c2, dq = 0.f;
      if (PART == 1) {
        dp = __shfl_sync(0xffffffffu, cD.x, src);
        dq = __shfl_sync(0xffffffffu, cD.y, src);
      }
      if (l < lmax && l >= ls) {
        if (PART == 0) {
          if (df)
            step<true>(a0, a1, c0, 0.f, c1, dp, xs);
          else
            step<false>(a0, a1, c0, 0.f, c1, 0.f, xs);
          if (S > 0 && fabsf(a0) > 0x1p32f) rescale(a0, a1, b0, b1, S, sc);
        } else {
          if (df) {
            step<true>(a0, a1, c0, c1, c2, dp, xs);
            step<true>(b0, b1, c0, -c1, c2, dq, xs);
          } else {
            step<false>(a0, a1, c0, c1, c2, 0.f, xs);
            step<false>(b0, b1, c0, -c1, c2, 0.f, xs);
          }
          if (S > 0 && fabsf(a0) + fabsf(b0) > 0x1p32f) rescale(a0, a1, b0, b1, S, sc);
        }
      }
    }
    if (PART == 0) {
      put_row(Ae, TILE_A, r, h, ve);
      put_row(Ae + 2 * TILE_A, TILE_A, r, h, vo);
    } else {
      put_row(Ae, TILE_A, r, h, ve);
      put_row(Ae + 2 * TILE_A, TILE_A, r, h, wo);
      put_row(Ao, TILE_A, r, h, vo);
      put_row(Ao + 2 * TILE_A, TILE_A, r, h, we);
    }
  }
}

// Warps 0-3: generators (thread = ring pair row) and epilogue; warp 4 lane 0:
// bulk copies of the B operand and the MMAs.  Units and tiles as in k_syn_tc:
// a unit is a K step for spin 0 and half of one for spin 2 (parity e:
// {lam+ e, lam- o}, parity o: {lam+ o, lam- e}); a generator fills both
// units of its K step.  full_a counts the 128 generator arrivals, full_b the
// copy's bytes, done the MMA commit that frees the stage.
template <int PART>
__global__ void __launch_bounds__(160, 1) k_syn_gen(
    const float4 *__restrict__ ck0, const float4 *__restrict__ ck2, const int64_t *__restrict__ cko,
    const float4 *__restrict__ rq0, const float4 *__restrict__ rq2, const float2 *__restrict__ rq2d,
    const PairDev *__restrict__ pairs,
    const unsigned char *__restrict__ bt, const int64_t *__restrict__ soff, float2 *__restrict__ rc, int lmax,
    int mmax, int npairs, int B, int NS, uint32_t ncols, int *err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar[3 * SGEN_MAX_NS];
  __shared__ uint32_t tslot;
  uint64_t *done = mbar, *full_a = mbar + SGEN_MAX_NS, *full_b = mbar + 2 * SGEN_MAX_NS;
  const int NC = (PART == 0) ? 2 * B : 4 * B;
  constexpr int nA = (PART == 0) ? 2 : 4;
  constexpr int UPS = (PART == 0) ? 1 : 2;
  constexpr int nU = nA / UPS;
  const int tileB = NC * 32;
  const int bbytes = nA * 2 * tileB;
  const int uabytes = nU * 2 * TILE_A, ubbytes = nU * 2 * tileB;
  const int stage = uabytes + ubbytes;
  const int m = blockIdx.y, pt = blockIdx.x, p0 = pt * 128;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&done[i], 1);
      mbar_init(&full_a[i], 128);
      mbar_init(&full_b[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tslot, ncols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tslot;
  const int nsteps = syn_steps(lmax, m);
  const int nunits = nsteps * UPS;
  if (warp < 4) {
    const int r = tid, pair = p0 + r;
    const bool act = pair < npairs;
    const int pp = act ? pair : npairs - 1;
    const Xs xs = xs_of(pairs, pp);
    const bool df = pair_dform(pairs, pp);
    const int64_t base = abase(lmax, m);
    const int64_t ckb = cko[m] * (int64_t)npairs + pp;
    const int ls = (PART == 1 && m < 2) ? 2 : 0;  // spin 2 starts at l = 2
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f, sc = 1.f;
    int S = 0;
    // lane t holds the coefficients of target l = m + 32 c + t + 1 for the
    // current K step c (cA, cD) and the next one (nA, nD), loaded a step ahead;
    // the checkpoint of the next block is loaded a block ahead (k0, k2)
    auto coef = [&](int c, float4 &ca, float2 &cd) {
      const int l1 = m + 32 * c + lane + 1;
      ca = make_float4(0.f, 0.f, 0.f, 0.f);
      cd = make_float2(0.f, 0.f);
      if (l1 <= lmax) {
        ca = PART == 0 ? rq0[base + l1] : rq2[base + l1];
        if (PART == 1) cd = rq2d[base + l1];
      }
    };
    float4 cA, nA, k0 = ck0[ckb], k2 = PART == 1 ? ck2[ckb] : make_float4(0.f, 0.f, 0.f, 0.f);
    float2 cD, nD;
    coef(0, cA, cD);
    for (int c = 0; c < nsteps; ++c) {
      if (c + 1 < nsteps) coef(c + 1, nA, nD);
      bool ok = true;
      for (int h = 0; h < UPS; ++h) {
        const int u = c * UPS + h;
        if (u >= NS && !mbar_wait(&done[u % NS], ((u - NS) / NS) & 1, err)) ok = false;
      }
      if (!ok) break;
      if ((c & 1) == 0) {  // restart at the checkpoint of block c / 2
        if (PART == 0) {
          a0 = k0.x;
          a1 = k0.y;
          S = __float_as_int(k0.z);
        } else {
          a0 = k2.x;
          a1 = k2.y;
          b0 = k2.z;
          b1 = k2.w;
          S = __float_as_int(k0.w);
        }
        sc = scale_of(S);
        if (c + 2 < nsteps) {
          const int64_t o = ckb + (int64_t)((c >> 1) + 1) * npairs;
          k0 = ck0[o];
          if (PART == 1) k2 = ck2[o];
        }
      }
      unsigned char *Ae = sm + ((c * UPS) % NS) * stage;
      unsigned char *Ao = PART == 0 ? Ae : sm + ((c * UPS + 1) % NS) * stage;
      syn_step<PART>(Ae, Ao, r, m + 32 * c, lmax, ls, act, a0, a1, b0, b1, S, sc, xs, df, cA, cD);
      cA = nA;
      cD = nD;
      fence_proxy_async();
      for (int h = 0; h < UPS; ++h) mbar_arrive(&full_a[(c * UPS + h) % NS]);
    }
  } else if (warp == 4 && lane == 0) {
    const unsigned char *btm = bt + soff[m] * (int64_t)bbytes;
    const uint32_t idesc = idesc_bf16(128, NC);
    auto tile = [&](int u, int j) { return PART == 0 ? j : ((u & 1) == 0 ? 3 * j : 1 + j); };
    auto issue = [&](int u) {
      const int s = u % NS, c = u / UPS;
      unsigned char *dst = sm + s * stage + uabytes;
      mbar_expect_tx(&full_b[s], (uint32_t)ubbytes);
      for (int j = 0; j < nU; ++j)
        bulk_g2s(dst + j * 2 * tileB, btm + (int64_t)c * bbytes + tile(u, j) * 2 * tileB, (uint32_t)(2 * tileB),
                 &full_b[s]);
    };
    for (int u = 0; u < NS && u < nunits; ++u) issue(u);
    int issued = min(NS, nunits), landed = 0, committed = 0;
    bool bad = false;
    for (int u = 0; u < nunits; ++u) {
      const int s = u % NS, c = u / UPS;
      unsigned char *Abuf = sm + s * stage, *Bbuf = Abuf + uabytes;
      if (!mbar_wait(&full_b[s], (u / NS) & 1, err)) {
        bad = true;
        break;
      }
      landed = u + 1;
      if (!mbar_wait(&full_a[s], (u / NS) & 1, err)) {
        bad = true;
        break;
      }
      fence_after_sync();
      const uint32_t acc = c > 0 ? 1u : 0u;
      if (PART == 0) {
        mma3(tbase, Abuf, Bbuf, tileB, idesc, acc);
        mma3(tbase + NC, Abuf + 2 * TILE_A, Bbuf + 2 * tileB, tileB, idesc, acc);
      } else {
        const uint32_t d = (u & 1) ? tbase + NC : tbase;
        mma3(d, Abuf, Bbuf, tileB, idesc, acc);
        mma3(d, Abuf + 2 * TILE_A, Bbuf + 2 * tileB, tileB, idesc, 1u);
      }
      commit(&done[s]);
      committed = u + 1;
      if (u >= 1 && u - 1 + NS < nunits) {
        if (!mbar_wait(&done[(u - 1) % NS], ((u - 1) / NS) & 1, err)) {
          bad = true;
          break;
        }
        issue(u - 1 + NS);
        issued = u + NS;
      }
    }
    // after a failed wait no more work is issued; the copies in flight land
    // before the CTA's shared memory goes away (their barriers count bytes only)
    if (bad)
      for (int v = landed; v < issued; ++v) mbar_wait(&full_b[v % NS], (v / NS) & 1, err);
    if (committed > 0) mbar_wait(&done[(committed - 1) % NS], ((committed - 1) / NS) & 1, err);
  }
  __syncthreads();
  fence_after_sync();
  if (warp < 4) {
    const int row = warp * 32 + lane, pair = p0 + row;
    const bool ok = pair < npairs, equator = (pair == npairs - 1);
    const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < NC; c0 += 16) {
      float ve[16], vo[16];
      tmem_ld16(trow + c0, ve);
      tmem_ld16(trow + NC + c0, vo);
      if (!ok) continue;
      if (PART == 0) {
        for (int i = 0; i < 8; ++i) {
          const int b = (c0 >> 1) + i;
          float2 *o = rc + ((((int64_t)b * 3 + 0) * (mmax + 1) + m) * npairs + pair) * 2;
          o[0] = make_float2(ve[2 * i] + vo[2 * i], ve[2 * i + 1] + vo[2 * i + 1]);
          if (!equator) o[1] = make_float2(ve[2 * i] - vo[2 * i], ve[2 * i + 1] - vo[2 * i + 1]);
        }
      } else {
        for (int i = 0; i < 4; ++i) {
          const int b = (c0 >> 2) + i;
          float2 *oq = rc + ((((int64_t)b * 3 + 1) * (mmax + 1) + m) * npairs + pair) * 2;
          float2 *ou = rc + ((((int64_t)b * 3 + 2) * (mmax + 1) + m) * npairs + pair) * 2;
          const float *e = ve + 4 * i, *d = vo + 4 * i;
          oq[0] = make_float2(e[0] + d[0], e[1] + d[1]);
          ou[0] = make_float2(e[2] + d[2], e[3] + d[3]);
          if (!equator) {
            oq[1] = make_float2(e[0] - d[0], e[1] - d[1]);
            ou[1] = make_float2(e[2] - d[2], e[3] - d[3]);
          }
        }
      }
    }
  }
  tc_teardown(tbase, ncols);
}

}  // namespace

// --------------------------------------------------------------------- host
// Checkpoints and FP32 recurrence coefficients, made on first use; all or
// nothing (a failure frees what was allocated here).
cudaError_t gen_setup(dm_plan *p) {
  if (p->ck0) return cudaSuccess;
  std::vector<int64_t> cko(p->mmax + 2, 0);
  for (int m = 0; m <= p->mmax; ++m) cko[m + 1] = cko[m] + (p->lmax - m + 1 + CKL - 1) / CKL;
  const size_t nrec = (size_t)cko[p->mmax + 1] * p->npairs;
  float4 *ck0 = nullptr, *ck2 = nullptr, *rq0 = nullptr, *rq2 = nullptr;
  float2 *rq2d = nullptr;
  int64_t *ckod = nullptr;
  auto fail = [&](cudaError_t e) {
    cudaFree(ck0);
    cudaFree(ck2);
    cudaFree(rq0);
    cudaFree(rq2);
    cudaFree(rq2d);
    cudaFree(ckod);
    return e;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&ck0, sizeof(float4) * nrec))) return fail(e);
  if ((e = cudaMalloc(&ck2, sizeof(float4) * nrec))) return fail(e);
  if ((e = cudaMalloc(&rq0, sizeof(float4) * (size_t)p->nalm))) return fail(e);
  if ((e = cudaMalloc(&rq2, sizeof(float4) * (size_t)p->nalm))) return fail(e);
  if ((e = cudaMalloc(&rq2d, sizeof(float2) * (size_t)p->nalm))) return fail(e);
  if ((e = cudaMalloc(&ckod, sizeof(int64_t) * cko.size()))) return fail(e);
  cudaMemset(ck0, 0, sizeof(float4) * nrec);
  cudaMemset(ck2, 0, sizeof(float4) * nrec);
  cudaMemcpy(ckod, cko.data(), sizeof(int64_t) * cko.size(), cudaMemcpyHostToDevice);
  k_rec32<<<512, 256>>>(p->rec, rq0, rq2, rq2d, p->nalm);
  k_ckpt<<<dim3((p->npairs + 127) / 128, p->mmax + 1), 128>>>(p->pairs, p->rec, p->seed, p->seed_exp, ckod, ck0,
                                                              ck2, p->lmax, p->npairs);
  if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize())) return fail(e);
  p->ck0 = ck0;
  p->ck2 = ck2;
  p->rq0 = rq0;
  p->rq2 = rq2;
  p->rq2d = rq2d;
  p->cko = ckod;
  p->bytes += (int64_t)(2 * sizeof(float4) * nrec + (2 * sizeof(float4) + sizeof(float2)) * (size_t)p->nalm +
                        sizeof(int64_t) * cko.size());
  return cudaSuccess;
}

// Stored tiles when they and the FP32 tables they are cut from take at most
// 40 GiB (nside 512 / lmax 1024: 26 GB); generated tiles beyond, where the
// tables would crowd out the batch (nside 1024 / lmax 2048: about 210 GB).
bool tc_tables_fit(int lmax, int mmax, int npairs, int B) {
  const int64_t nalm = (int64_t)(mmax + 1) * (2 * lmax + 2 - mmax) / 2;
  const double bytes = (double)tc_table_bytes(lmax, mmax, npairs, B) + 24.0 * (double)nalm * npairs;
  return bytes <= 40.0 * (1u << 30);
}

bool tc_generate(dm_plan *p) {
  if (p->tc_gen >= 0) return p->tc_gen != 0;
  if (p->tc_gen_used < 0) p->tc_gen_used = tc_tables_fit(p->lmax, p->mmax, p->npairs, p->batch) ? 0 : 1;
  return p->tc_gen_used != 0;
}

size_t gen_bytes(int lmax, int mmax, int npairs) {
  int64_t nck = 0;
  for (int m = 0; m <= mmax; ++m) nck += (lmax - m + 1 + CKL - 1) / CKL;
  const int64_t nalm = (int64_t)(mmax + 1) * (2 * lmax + 2 - mmax) / 2;
  return (size_t)(2 * 16 * nck * npairs + 40 * nalm);
}

// stages of the generated synthesis: as many as fit in one CTA's shared memory,
// or in half of it when two CTAs can share an SM's tensor memory (2 .. 8)
static int sgen_stages(int want, int stage_bytes, uint32_t ncols) {
  const int fit = (int)(((227u << 10) - 1024u) / (unsigned)stage_bytes);
  if (want > 0) return std::max(2, std::min(want, std::min(fit, SGEN_MAX_NS)));
  const int per_sm = ncols <= 256 ? 2 : 1;
  const int ns = (int)(((227u << 10) - 1024u * per_sm) / per_sm) / stage_bytes;
  return std::max(2, std::min(ns, SGEN_MAX_NS));
}

cudaError_t syn_gen_launch(dm_plan *p, bool run0, bool run1, cudaStream_t st) {
  cudaError_t e = gen_setup(p);
  if (e) return e;
  const int B = p->batch, npt = (p->npairs + 127) / 128;
  dim3 g(npt, p->mmax + 1);
  if (run0) {
    const int stage = 2 * 2 * TILE_A + 2 * 2 * (2 * B * 32);
    const uint32_t nc = pow2_cols(4 * B);
    const int ns = sgen_stages(p->tune_syn_ns[0], stage, nc);
    p->syn_ns_used[0] = ns;
    const size_t sm = tc_smem_n(stage, ns, nc);
    dyn_smem_allow(k_syn_gen<0>, sm);
    k_syn_gen<0><<<g, 160, sm, st>>>(p->ck0, p->ck2, p->cko, p->rq0, p->rq2, p->rq2d, p->pairs, p->tc_synB[0], p->tc_soff,
                                     p->rc32, p->lmax, p->mmax, p->npairs, B, ns, nc, p->tc_err);
  }
  if (run1) {
    const int stage = 2 * 2 * TILE_A + 2 * 2 * (4 * B * 32);
    const uint32_t nc = pow2_cols(8 * B);
    const int ns = sgen_stages(p->tune_syn_ns[1], stage, nc);
    p->syn_ns_used[1] = ns;
    const size_t sm = tc_smem_n(stage, ns, nc);
    dyn_smem_allow(k_syn_gen<1>, sm);
    k_syn_gen<1><<<g, 160, sm, st>>>(p->ck0, p->ck2, p->cko, p->rq0, p->rq2, p->rq2d, p->pairs, p->tc_synB[1], p->tc_soff,
                                     p->rc32, p->lmax, p->mmax, p->npairs, B, ns, nc, p->tc_err);
  }
  return cudaGetLastError();
}

// l tiles per CTA (tensor memory: LT x NC <= 512 columns; the lane map holds
// 4 for spin 0, 2 for spin 2) and worker warps = stages (2 .. 5, as many as
// fit in shared memory)
static int agen_stage_bytes(int part, int LT, int B) {
  const int nA = part == 0 ? 1 : 2, NC = part == 0 ? 2 * B : 4 * B;
  return (((LT * nA * ATS) + 1023) & ~1023) + nA * 2 * NC * 32;
}

cudaError_t ana_gen_launch(dm_plan *p, cudaStream_t st) {
  cudaError_t e = gen_setup(p);
  if (e) return e;
  const int B = p->batch;
  const int ltiles = ana_tiles(p->lmax, 0, 0);
  for (int part = 0; part < 2; ++part) {
    if (p->tune_only_part == 1 - part) continue;
    const int NC = part == 0 ? 2 * B : 4 * B;
    const int ltmax = std::max(1, std::min(part == 0 ? 4 : 2, 512 / (int)pow2_cols(NC)));
    const int LT = p->tune_ana_lt[part] > 0 ? std::min(p->tune_ana_lt[part], ltmax) : ltmax;
    const int stage = agen_stage_bytes(part, LT, B);
    const int coef_bytes = ((coef_slots(LT) * (part == 0 ? 16 : 24)) + 1023) & ~1023;
    const int fit = (int)(((227u << 10) - 1024u - (unsigned)coef_bytes) / (unsigned)stage);
    const int want = p->tune_ana_S[part] > 0 ? p->tune_ana_S[part] : AGEN_MAX_S;
    const int S = std::max(1, std::min(want, std::min(fit, AGEN_MAX_S)));
    if (fit < 1) return cudaErrorInvalidConfiguration;
    p->ana_lt_used[part] = LT;
    p->ana_S_used[part] = S;
    const uint32_t nc = pow2_cols(LT * NC);
    const size_t sm = tc_smem_n(stage, S, nc) + coef_bytes;
    dim3 g((ltiles + LT - 1) / LT, 2, p->mmax + 1);
    if (part == 0) {
      dyn_smem_allow(k_ana_gen<0>, sm);
      k_ana_gen<0><<<g, AGEN_THREADS, sm, st>>>(p->ck0, p->ck2, p->cko, p->rq0, p->rq2, p->rq2d, p->pairs, p->rc32,
                                                p->apart32, p->lmax, p->mmax, p->npairs, p->nalm, B, LT, nc, S,
                                                p->tc_err, p->tc_withhold);
    } else {
      dyn_smem_allow(k_ana_gen<1>, sm);
      k_ana_gen<1><<<g, AGEN_THREADS, sm, st>>>(p->ck0, p->ck2, p->cko, p->rq0, p->rq2, p->rq2d, p->pairs, p->rc32,
                                                p->apart32, p->lmax, p->mmax, p->npairs, p->nalm, B, LT, nc, S,
                                                p->tc_err, 0);
    }
  }
  return cudaGetLastError();
}

}  // namespace dmwf
