// dm_legendre_tc.cu -- the Legendre stages of a batch of right-hand sides as
// dense contractions on the tcgen05 tensor cores (mixed precision).
//
// For one order m the synthesis is, per parity class of l (l - m even / odd),
//   T_p[pair][b]  = sum_{l in p} lambda_l(pair) aT_l[b]
//   QU_p[pair][b] = sum_{l in p} lam+_l(pair) X1_l[b] + sum_{l in p'} lam-_l(pair) X2_l[b]
// with X1 = (-aE, -aB) and X2 = (-i aB, +i aE) (re, im columns), and the
// mirror ring from F_N = F_e + F_o, F_S = F_e - F_o.  The analysis is the
// transposed contraction over ring pairs:
//   aT_l[b] = sum_pairs lambda_l G^T_p,   (aE, aB)_l[b] = -sum_pairs (lam+_l (G^Q, G^U)_p
//             + lam-_l (i G^U, -i G^Q)_p').
// Both are GEMMs with M = 128 (ring pairs or multipoles), N = 2B or 4B columns
// (B right-hand sides x re/im x fields), K over multipoles or ring pairs.
// Operands: the FP32 Legendre tables (generated once by the FP64 recurrence)
// and the FP32 iterate, each split into BF16 hi + lo in shared memory; three
// kind::f16 MMAs per K step (hi*hi + hi*lo + lo*hi) accumulate in FP32 in
// tensor memory.  The FP64 anchors of the mixed mode carry the last digits.
// Two shared-memory stages: threads stage step c+1 while the MMAs of step c run.
#include "dm_internal.h"
#include "dm_tc.cuh"

namespace dmwf {

using namespace tc;

namespace {

constexpr int TC_THREADS = 256;
constexpr int TILE_A = 4096;  // 128 x 16 BF16

__device__ __forceinline__ int64_t abase(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

__device__ __forceinline__ void put_split(unsigned char *hi, int tile_bytes, int row, int k, float x) {
  __nv_bfloat16 h, l;
  split_bf16(x, h, l);
  const uint32_t off = kmajor_off(row, k);
  *reinterpret_cast<__nv_bfloat16 *>(hi + off) = h;
  *reinterpret_cast<__nv_bfloat16 *>(hi + tile_bytes + off) = l;
}

__device__ __forceinline__ void mma3(uint32_t d, const unsigned char *a, const unsigned char *b, int tile_b,
                                     uint32_t idesc, uint32_t acc) {
  const uint64_t ah = smem_desc(smem_u32(a)), al = smem_desc(smem_u32(a + TILE_A));
  const uint64_t bh = smem_desc(smem_u32(b)), bl = smem_desc(smem_u32(b + tile_b));
  mma_bf16(d, ah, bh, idesc, acc);
  mma_bf16(d, ah, bl, idesc, 1u);
  mma_bf16(d, al, bh, idesc, 1u);
}

__device__ __forceinline__ float2 e_of(const double2 *a, const double2 *ahi, int64_t i) {
  double2 v = a[i];
  if (ahi != nullptr) {
    const double2 h = ahi[i];
    v.x -= h.x;
    v.y -= h.y;
  }
  return make_float2((float)v.x, (float)v.y);
}

__device__ __forceinline__ void tc_setup(uint64_t *mbar, uint32_t *slot, uint32_t ncols) {
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(slot, ncols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

__device__ __forceinline__ void tc_drain(uint64_t *mbar, int n, int *err) {
  if (n >= 2) mbar_wait(&mbar[(n - 2) & 1], ((n - 2) >> 1) & 1, err);
  mbar_wait(&mbar[(n - 1) & 1], ((n - 1) >> 1) & 1, err);
  fence_after_sync();
}

__device__ __forceinline__ void tc_teardown(uint32_t tbase, uint32_t ncols) {
  fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tbase, ncols);
}

}  // namespace

// ---------------------------------------------------------------- synthesis
// PART 0: T (2 A tiles: lambda even / odd; D columns [0, 2B) even, [2B, 4B) odd)
// PART 1: Q, U (A tiles lam+ e, lam+ o, lam- e, lam- o with B tiles X1 e, X1 o,
//          X2 e, X2 o; D_e = [0, 4B), D_o = [4B, 8B))
// grid (pair tiles of 128, m); K steps of 32 consecutive multipoles (16 + 16).
template <int PART>
__global__ void __launch_bounds__(TC_THREADS, 1) k_syn_tc(const float *__restrict__ ptab,
                                                         const double2 *__restrict__ alm,
                                                         const double2 *__restrict__ a_hi, float2 *__restrict__ rc,
                                                         int lmax, int mmax, int npairs, int64_t nalm, int B,
                                                         uint32_t ncols, int *err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tslot;
  const int NC = (PART == 0) ? 2 * B : 4 * B;  // D columns per parity
  const int nA = (PART == 0) ? 2 : 4;
  const int tileB = NC * 32;
  const int stage = nA * 2 * TILE_A + nA * 2 * tileB;
  const int m = blockIdx.y, p0 = blockIdx.x * 128;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  tc_setup(mbar, &tslot, ncols);
  const uint32_t tbase = tslot;
  const int64_t base = abase(lmax, m);
  const int64_t plane = nalm * (int64_t)npairs;
  const int nsteps = (lmax - m + 1 + 31) / 32;
  const uint32_t idesc = idesc_bf16(128, NC);
  for (int c = 0; c < nsteps; ++c) {
    const int s = c & 1;
    unsigned char *st = sm + s * stage;
    if (c >= 2) mbar_wait(&mbar[s], ((c - 2) >> 1) & 1, err);
    unsigned char *Abuf = st, *Bbuf = st + nA * 2 * TILE_A;
    // A tiles: row = pair (coalesced), k = l step within the parity class
    for (int idx = tid; idx < nA * 2048; idx += TC_THREADS) {
      const int t = idx >> 11, r = idx & 2047, k = r >> 7, row = r & 127;
      const int par = t & 1, func = (PART == 0) ? 0 : 1 + (t >> 1);
      const int l = m + 32 * c + par + 2 * k, pair = p0 + row;
      const float x = (l <= lmax && pair < npairs) ? ptab[func * plane + (base + l) * npairs + pair] : 0.f;
      put_split(Abuf + t * 2 * TILE_A, TILE_A, row, k, x);
    }
    // B tiles from the iterate (correction e = a - a_hi in the anchored mixed mode)
    for (int idx = tid; idx < 2 * B * 16; idx += TC_THREADS) {
      const int par = idx / (B * 16), rem = idx % (B * 16), b = rem >> 4, k = rem & 15;
      const int l = m + 32 * c + par + 2 * k;
      const int64_t ib = (int64_t)b * 3 * nalm + base + l;
      if (PART == 0) {
        float2 t = (l <= lmax) ? e_of(alm, a_hi, ib) : make_float2(0.f, 0.f);
        unsigned char *T = Bbuf + par * 2 * tileB;
        put_split(T, tileB, 2 * b, k, t.x);
        put_split(T, tileB, 2 * b + 1, k, t.y);
      } else {
        float2 e = make_float2(0.f, 0.f), bb = make_float2(0.f, 0.f);
        if (l <= lmax) {
          e = e_of(alm, a_hi, ib + nalm);
          bb = e_of(alm, a_hi, ib + 2 * nalm);
        }
        unsigned char *X1 = Bbuf + par * 2 * tileB, *X2 = Bbuf + (2 + par) * 2 * tileB;
        put_split(X1, tileB, 4 * b + 0, k, -e.x);   // Q.re <- -aE.re
        put_split(X1, tileB, 4 * b + 1, k, -e.y);   // Q.im <- -aE.im
        put_split(X1, tileB, 4 * b + 2, k, -bb.x);  // U.re <- -aB.re
        put_split(X1, tileB, 4 * b + 3, k, -bb.y);  // U.im <- -aB.im
        put_split(X2, tileB, 4 * b + 0, k, bb.y);   // Q.re <- (-i aB).re
        put_split(X2, tileB, 4 * b + 1, k, -bb.x);  // Q.im <- (-i aB).im
        put_split(X2, tileB, 4 * b + 2, k, -e.y);   // U.re <- (+i aE).re
        put_split(X2, tileB, 4 * b + 3, k, e.x);    // U.im <- (+i aE).im
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t acc = c > 0 ? 1u : 0u;
      if (PART == 0) {
        mma3(tbase, Abuf, Bbuf, tileB, idesc, acc);
        mma3(tbase + NC, Abuf + 2 * TILE_A, Bbuf + 2 * tileB, tileB, idesc, acc);
      } else {
        // D_e += lam+_e X1_e + lam-_o X2_o ;  D_o += lam+_o X1_o + lam-_e X2_e
        mma3(tbase, Abuf + 0 * 2 * TILE_A, Bbuf + 0 * 2 * tileB, tileB, idesc, acc);
        mma3(tbase, Abuf + 3 * 2 * TILE_A, Bbuf + 3 * 2 * tileB, tileB, idesc, 1u);
        mma3(tbase + NC, Abuf + 1 * 2 * TILE_A, Bbuf + 1 * 2 * tileB, tileB, idesc, acc);
        mma3(tbase + NC, Abuf + 2 * 2 * TILE_A, Bbuf + 2 * 2 * tileB, tileB, idesc, 1u);
      }
      commit(&mbar[s]);
    }
  }
  tc_drain(mbar, nsteps, err);
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

// ----------------------------------------------------------------- analysis
// PART 0: aT    (A = lambda [128 l x 16 pairs], B rows (b, re/im))
// PART 1: aE,aB (A = lam+ with B1 rows (b; E.re, E.im, B.re, B.im) and
//                A = lam- with B2, over 16 pairs per K step)
// grid (l tiles of 128 multipoles of one parity, parity, m); rows l = m + p + 2 i.
// Output: out[b][f][alm] (FP32 partial sums with a single chunk).
template <int PART>
__global__ void __launch_bounds__(TC_THREADS, 1) k_ana_tc(const float *__restrict__ ptab,
                                                         const float2 *__restrict__ rc, float2 *__restrict__ out,
                                                         int lmax, int mmax, int npairs, int64_t nalm, int B,
                                                         uint32_t ncols, int *err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tslot;
  const int m = blockIdx.z, par = blockIdx.y, lt = blockIdx.x;
  const int nl = (lmax - m + 1 - par + 1) / 2;  // multipoles of this parity
  if (nl <= 0 || lt * 128 >= nl) return;        // uniform over the block
  const int NC = (PART == 0) ? 2 * B : 4 * B;
  const int nA = (PART == 0) ? 1 : 2;
  const int tileB = NC * 32;
  const int stage = nA * 2 * TILE_A + nA * 2 * tileB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  tc_setup(mbar, &tslot, ncols);
  const uint32_t tbase = tslot;
  const int64_t base = abase(lmax, m);
  const int64_t plane = nalm * (int64_t)npairs;
  const int nsteps = (npairs + 15) / 16;
  const uint32_t idesc = idesc_bf16(128, NC);
  const int opp = par ^ 1;
  for (int c = 0; c < nsteps; ++c) {
    const int s = c & 1;
    unsigned char *st = sm + s * stage;
    if (c >= 2) mbar_wait(&mbar[s], ((c - 2) >> 1) & 1, err);
    unsigned char *Abuf = st, *Bbuf = st + nA * 2 * TILE_A;
    const int pair0 = 16 * c;
    // A tiles: row = multipole, k = pair (16 consecutive floats per row)
    for (int idx = tid; idx < nA * 2048; idx += TC_THREADS) {
      const int t = idx >> 11, r = idx & 2047, row = r >> 4, k = r & 15;
      const int func = (PART == 0) ? 0 : 1 + t;
      const int i = lt * 128 + row, l = m + par + 2 * i, pair = pair0 + k;
      const float x = (i < nl && pair < npairs) ? ptab[func * plane + (base + l) * npairs + pair] : 0.f;
      put_split(Abuf + t * 2 * TILE_A, TILE_A, row, k, x);
    }
    // B tiles from the ring coefficients (parity combinations of the ring pair)
    for (int idx = tid; idx < B * 16; idx += TC_THREADS) {
      const int b = idx >> 4, k = idx & 15, pair = pair0 + k;
      const bool ok = pair < npairs, eq = (pair == npairs - 1);
      if (PART == 0) {
        float2 gp = make_float2(0.f, 0.f);
        if (ok) {
          const float2 *g = rc + ((((int64_t)b * 3 + 0) * (mmax + 1) + m) * npairs + pair) * 2;
          const float2 gn = g[0], gs = eq ? make_float2(0.f, 0.f) : g[1];
          gp = par == 0 ? make_float2(gn.x + gs.x, gn.y + gs.y) : make_float2(gn.x - gs.x, gn.y - gs.y);
        }
        put_split(Bbuf, tileB, 2 * b, k, gp.x);
        put_split(Bbuf, tileB, 2 * b + 1, k, gp.y);
      } else {
        float2 qp = make_float2(0.f, 0.f), up = qp, qo = qp, uo = qp;
        if (ok) {
          const float2 *gq = rc + ((((int64_t)b * 3 + 1) * (mmax + 1) + m) * npairs + pair) * 2;
          const float2 *gu = rc + ((((int64_t)b * 3 + 2) * (mmax + 1) + m) * npairs + pair) * 2;
          const float2 qn = gq[0], qs = eq ? make_float2(0.f, 0.f) : gq[1];
          const float2 un = gu[0], us = eq ? make_float2(0.f, 0.f) : gu[1];
          const float2 qe = make_float2(qn.x + qs.x, qn.y + qs.y), qd = make_float2(qn.x - qs.x, qn.y - qs.y);
          const float2 ue = make_float2(un.x + us.x, un.y + us.y), ud = make_float2(un.x - us.x, un.y - us.y);
          qp = par == 0 ? qe : qd;
          up = par == 0 ? ue : ud;
          qo = opp == 0 ? qe : qd;
          uo = opp == 0 ? ue : ud;
        }
        unsigned char *B1 = Bbuf, *B2 = Bbuf + 2 * tileB;
        put_split(B1, tileB, 4 * b + 0, k, -qp.x);  // aE.re <- -lam+ GQ.re
        put_split(B1, tileB, 4 * b + 1, k, -qp.y);  // aE.im
        put_split(B1, tileB, 4 * b + 2, k, -up.x);  // aB.re <- -lam+ GU.re
        put_split(B1, tileB, 4 * b + 3, k, -up.y);  // aB.im
        put_split(B2, tileB, 4 * b + 0, k, uo.y);   // aE.re <- +lam- GU_opp.im
        put_split(B2, tileB, 4 * b + 1, k, -uo.x);  // aE.im <- -lam- GU_opp.re
        put_split(B2, tileB, 4 * b + 2, k, -qo.y);  // aB.re <- -lam- GQ_opp.im
        put_split(B2, tileB, 4 * b + 3, k, qo.x);   // aB.im <- +lam- GQ_opp.re
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t acc = c > 0 ? 1u : 0u;
      if (PART == 0) {
        mma3(tbase, Abuf, Bbuf, tileB, idesc, acc);
      } else {
        mma3(tbase, Abuf, Bbuf, tileB, idesc, acc);
        mma3(tbase, Abuf + 2 * TILE_A, Bbuf + 2 * tileB, tileB, idesc, 1u);
      }
      commit(&mbar[s]);
    }
  }
  tc_drain(mbar, nsteps, err);
  if (warp < 4) {
    const int row = warp * 32 + lane, i = lt * 128 + row;
    const bool ok = i < nl;
    const int64_t idx = base + m + par + 2 * i;
    const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < NC; c0 += 16) {
      float v[16];
      tmem_ld16(trow + c0, v);
      if (!ok) continue;
      if (PART == 0) {
        for (int j = 0; j < 8; ++j) {
          const int b = (c0 >> 1) + j;
          out[((int64_t)b * 3 + 0) * nalm + idx] = make_float2(v[2 * j], v[2 * j + 1]);
        }
      } else {
        for (int j = 0; j < 4; ++j) {
          const int b = (c0 >> 2) + j;
          out[((int64_t)b * 3 + 1) * nalm + idx] = make_float2(v[4 * j], v[4 * j + 1]);
          out[((int64_t)b * 3 + 2) * nalm + idx] = make_float2(v[4 * j + 2], v[4 * j + 3]);
        }
      }
    }
  }
  tc_teardown(tbase, ncols);
}

// ------------------------------------------------------------------ launch
static uint32_t pow2_cols(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

// smem per CTA, raised when needed so that the CTAs sharing an SM never ask
// for more tensor memory than its 512 columns
static size_t tc_smem(int stage_bytes, uint32_t ncols) {
  size_t s = 2 * (size_t)stage_bytes + 1024;
  const int per_sm = (int)(512 / ncols);
  const size_t floor_bytes = (232448 / (per_sm + 1)) + 1024;
  return s > floor_bytes ? s : floor_bytes;
}

bool tc_batch_ok(int B) { return B == 8 || B == 16 || B == 32 || B == 64; }

cudaError_t legendre_synthesis_tc(dm_plan *p, const double2 *alm, cudaStream_t st) {
  const int B = p->batch;
  const double2 *ahi = p->anchor_active ? p->a_hi : nullptr;
  dim3 g((p->npairs + 127) / 128, p->mmax + 1);
  {
    const uint32_t nc = pow2_cols(4 * B);
    const size_t sm = tc_smem(2 * 2 * TILE_A + 2 * 2 * (2 * B * 32), nc);
    cudaFuncSetAttribute(k_syn_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_syn_tc<0><<<g, TC_THREADS, sm, st>>>(p->ptab, alm, ahi, p->rc32, p->lmax, p->mmax, p->npairs, p->nalm, B, nc,
                                           p->tc_err);
  }
  {
    const uint32_t nc = pow2_cols(8 * B);
    const size_t sm = tc_smem(4 * 2 * TILE_A + 4 * 2 * (4 * B * 32), nc);
    cudaFuncSetAttribute(k_syn_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_syn_tc<1><<<g, TC_THREADS, sm, st>>>(p->ptab, alm, ahi, p->rc32, p->lmax, p->mmax, p->npairs, p->nalm, B, nc,
                                           p->tc_err);
  }
  return cudaGetLastError();
}

cudaError_t legendre_analysis_tc(dm_plan *p, cudaStream_t st) {
  const int B = p->batch;
  const int ltiles = ((p->lmax + 2) / 2 + 127) / 128;
  dim3 g(ltiles, 2, p->mmax + 1);
  {
    const uint32_t nc = pow2_cols(2 * B);
    const size_t sm = tc_smem(1 * 2 * TILE_A + 1 * 2 * (2 * B * 32), nc);
    cudaFuncSetAttribute(k_ana_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_ana_tc<0><<<g, TC_THREADS, sm, st>>>(p->ptab, p->rc32, p->apart32, p->lmax, p->mmax, p->npairs, p->nalm, B,
                                           nc, p->tc_err);
  }
  {
    const uint32_t nc = pow2_cols(4 * B);
    const size_t sm = tc_smem(2 * 2 * TILE_A + 2 * 2 * (4 * B * 32), nc);
    cudaFuncSetAttribute(k_ana_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_ana_tc<1><<<g, TC_THREADS, sm, st>>>(p->ptab, p->rc32, p->apart32, p->lmax, p->mmax, p->npairs, p->nalm, B,
                                           nc, p->tc_err);
  }
  return cudaGetLastError();
}

}  // namespace dmwf
