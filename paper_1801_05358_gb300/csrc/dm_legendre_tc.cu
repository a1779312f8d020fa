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
// Operands: the Legendre tables, split once into BF16 hi + lo and stored in
// HBM in the K-major core-matrix tile order of each kernel, are streamed into
// shared memory with bulk asynchronous copies (cp.async.bulk, completion by
// mbarrier transaction count); the iterate (synthesis) or the ring
// coefficients (analysis) are split into BF16 hi + lo by the threads, whole
// 16-byte core-matrix rows per store.  Three kind::f16 MMAs per K step
// (hi*hi + hi*lo + lo*hi) accumulate in FP32 in tensor memory; the FP64
// anchors of the mixed mode carry the last digits.  Two shared-memory stages:
// while the MMAs of step c run, the copy of step c+1's tables and the
// conversion of its other operand proceed.
#include <algorithm>
#include <vector>

#include "dm_internal.h"
#include "dm_tc.cuh"
#include "dm_tc_tiles.cuh"

namespace dmwf {

using namespace tc;

namespace {

constexpr int TC_THREADS = 256;

__device__ __forceinline__ float2 e_of(const double2 *a, const double2 *ahi, int64_t i) {
  double2 v = a[i];
  if (ahi != nullptr) {
    const double2 h = ahi[i];
    v.x -= h.x;
    v.y -= h.y;
  }
  return make_float2((float)v.x, (float)v.y);
}

}  // namespace

// ------------------------------------------------------------ table layouts
// Synthesis: per (m, pair tile pt, K step c) one block of nA tiles, each
// 128 pairs x 16 multipoles of one parity (l = m + 32 c + par + 2 k), hi then
// lo.  PART 0 tiles {lambda e, lambda o}; PART 1 {lam+ e, lam+ o, lam- e,
// lam- o}.  Blocks of one CTA (m, pt) are consecutive in c.
// Analysis: per (m, parity, l tile lt, K step c) one block of nA tiles, each
// 128 multipoles (l = m + par + 2 i, i = 128 lt + row) x 16 ring pairs, hi
// then lo.  PART 0 tile {lambda}; PART 1 {lam+, lam-}.

template <int PART>
__global__ void k_tab_syn(const float *__restrict__ ptab, unsigned char *__restrict__ out,
                          const int64_t *__restrict__ soff, int lmax, int npairs, int64_t nalm, int npt) {
  constexpr int nA = PART == 0 ? 2 : 4;
  const int c = blockIdx.x, pt = blockIdx.y, m = blockIdx.z;
  const int ns = syn_steps(lmax, m);
  if (c >= ns) return;
  const int64_t plane = nalm * (int64_t)npairs, base = abase(lmax, m);
  unsigned char *blk = out + (soff[m] * npt + (int64_t)pt * ns + c) * (int64_t)(nA * 2 * TILE_A);
  for (int idx = threadIdx.x; idx < nA * 256; idx += blockDim.x) {
    const int t = idx >> 8, q = idx & 255, row = q & 127, ko = q >> 7;
    const int par = t & 1, func = PART == 0 ? 0 : 1 + (t >> 1);
    const int pair = pt * 128 + row;
    float x[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int l = m + 32 * c + par + 2 * (8 * ko + kk);
      x[kk] = (l <= lmax && pair < npairs) ? ptab[func * plane + (base + l) * npairs + pair] : 0.f;
    }
    put_row(blk + t * 2 * TILE_A, TILE_A, row, ko, x);
  }
}

template <int PART>
__global__ void k_tab_ana(const float *__restrict__ ptab, unsigned char *__restrict__ out,
                          const int64_t *__restrict__ aoff, int lmax, int npairs, int64_t nalm, int nps) {
  constexpr int nA = PART == 0 ? 1 : 2;
  const int c = blockIdx.x, lt = blockIdx.y, m = blockIdx.z >> 1, par = blockIdx.z & 1;
  const int nl = ana_nl(lmax, m, par);
  if (lt * 128 >= nl) return;
  const int64_t plane = nalm * (int64_t)npairs, base = abase(lmax, m);
  unsigned char *blk = out + ((aoff[2 * m + par] + lt) * nps + c) * (int64_t)(nA * 2 * TILE_A);
  for (int idx = threadIdx.x; idx < nA * 256; idx += blockDim.x) {
    const int t = idx >> 8, q = idx & 255, row = q >> 1, ko = q & 1;
    const int func = PART == 0 ? 0 : 1 + t;
    const int i = lt * 128 + row, l = m + par + 2 * i, pair0 = 16 * c + 8 * ko;
    float x[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
      x[kk] = (i < nl && pair0 + kk < npairs) ? ptab[func * plane + (base + l) * npairs + pair0 + kk] : 0.f;
    put_row(blk + t * 2 * TILE_A, TILE_A, row, ko, x);
  }
}

// ---------------------------------------------------------------- synthesis
// PART 0: T (2 A tiles: lambda even / odd; D columns [0, 2B) even, [2B, 4B) odd)
// PART 1: Q, U (A tiles lam+ e, lam+ o, lam- e, lam- o with B tiles X1 e, X1 o,
//          X2 e, X2 o; D_e = [0, 4B), D_o = [4B, 8B))
// grid (pair tiles of 128, m); K steps of 32 consecutive multipoles (16 + 16).
// The B rows are written so that the 8 threads of a quarter warp fill the 8
// rows of one core matrix (row order rotated by the k-octet): no bank conflicts.
// iterate value: the FP32 state e when given, else a - a_hi (a_hi may be null)
__device__ __forceinline__ float2 iter_of(const float2 *__restrict__ e32, const double2 *__restrict__ alm,
                                          const double2 *__restrict__ a_hi, int64_t i) {
  return e32 != nullptr ? e32[i] : e_of(alm, a_hi, i);
}

template <int PART>
__device__ __forceinline__ void stage_syn_b(unsigned char *Bbuf, int tileB, const double2 *__restrict__ alm,
                                            const double2 *__restrict__ a_hi, const float2 *__restrict__ e32,
                                            int64_t base, int m, int c, int lmax, int64_t nalm, int B) {
  if (PART == 0) {
    // task = ((par * B/4 + b/4) * 8) + (b & 3) * 2 + ko: rows 2b, 2b + 1 of parity tile par
    for (int task = threadIdx.x; task < 4 * B; task += TC_THREADS) {
      const int ko = task & 1, b = ((task >> 3) % (B >> 2)) * 4 + ((task >> 1) & 3), par = task / (2 * B);
      float re[8], im[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int l = m + 32 * c + par + 2 * (8 * ko + kk);
        const float2 v =
            l <= lmax ? iter_of(e32, alm, a_hi, (int64_t)b * 3 * nalm + base + l) : make_float2(0.f, 0.f);
        re[kk] = v.x;
        im[kk] = v.y;
      }
      unsigned char *T = Bbuf + par * 2 * tileB;
      put_row(T, tileB, 2 * b + ko, ko, ko ? im : re);
      put_row(T, tileB, 2 * b + (ko ^ 1), ko, ko ? re : im);
    }
  } else {
    // task = ((par * B/2 + b/2) * 8) + (b & 1) * 4 + f * 2 + ko, f = 0 (E) / 1 (B)
    for (int task = threadIdx.x; task < 8 * B; task += TC_THREADS) {
      const int ko = task & 1, f = (task >> 1) & 1, b = ((task >> 3) % (B >> 1)) * 2 + ((task >> 2) & 1);
      const int par = task / (4 * B);
      float re[8], im[8], nre[8], nim[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int l = m + 32 * c + par + 2 * (8 * ko + kk);
        const float2 v =
            l <= lmax ? iter_of(e32, alm, a_hi, ((int64_t)b * 3 + 1 + f) * nalm + base + l) : make_float2(0.f, 0.f);
        re[kk] = v.x;
        im[kk] = v.y;
        nre[kk] = -v.x;
        nim[kk] = -v.y;
      }
      unsigned char *X1 = Bbuf + par * 2 * tileB, *X2 = Bbuf + (2 + par) * 2 * tileB;
      // X1: E -> rows 4b (-E.re), 4b+1 (-E.im); B -> rows 4b+2 (-B.re), 4b+3 (-B.im)
      const int r1 = 4 * b + 2 * f;
      put_row(X1, tileB, r1 + ko, ko, ko ? nim : nre);
      put_row(X1, tileB, r1 + (ko ^ 1), ko, ko ? nre : nim);
      // X2: E -> rows 4b+2 (-E.im), 4b+3 (E.re); B -> rows 4b (B.im), 4b+1 (-B.re)
      const int r2 = 4 * b + 2 * (1 - f);
      const float *x2a = f == 0 ? nim : im, *x2b = f == 0 ? re : nre;  // rows r2, r2 + 1
      put_row(X2, tileB, r2 + ko, ko, ko ? x2b : x2a);
      put_row(X2, tileB, r2 + (ko ^ 1), ko, ko ? x2a : x2b);
    }
  }
}

// The B operand of every (m, K step) once per synthesis, in the tile order of
// the shared-memory stage: block (m, c) at (soff[m] + c) * nA * 2 * tileB.
template <int PART>
__global__ void __launch_bounds__(TC_THREADS) k_syn_b(unsigned char *__restrict__ out, const int64_t *__restrict__ soff,
                                                      const double2 *__restrict__ alm,
                                                      const double2 *__restrict__ a_hi,
                                                      const float2 *__restrict__ e32, int lmax, int64_t nalm,
                                                      int B) {
  const int c = blockIdx.x, m = blockIdx.y;
  if (c >= syn_steps(lmax, m)) return;
  constexpr int nA = (PART == 0) ? 2 : 4;
  const int tileB = ((PART == 0) ? 2 * B : 4 * B) * 32;
  stage_syn_b<PART>(out + (soff[m] + c) * (int64_t)(nA * 2 * tileB), tileB, alm, a_hi, e32, abase(lmax, m), m, c,
                    lmax, nalm, B);
}

constexpr int TC_MAX_STAGES = 8;

// Both operands arrive by bulk copy: thread 0 keeps NS stages in flight and
// issues the MMAs; the four warps read the accumulators out at the end.  A
// stage holds one unit of work: a whole K step for spin 0, and for spin 2 the
// half of a K step that feeds one parity accumulator (lam+_e X1_e + lam-_o X2_o
// into D_e, lam+_o X1_o + lam-_e X2_e into D_o), so that twice as many stages
// fit in shared memory.
template <int PART>
__global__ void __launch_bounds__(128, 1) k_syn_tc(const unsigned char *__restrict__ tab,
                                                   const unsigned char *__restrict__ bt,
                                                   const int64_t *__restrict__ soff, float2 *__restrict__ rc,
                                                   int lmax, int mmax, int npairs, int B, int NS, uint32_t ncols,
                                                   int *err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar[2 * TC_MAX_STAGES];  // done[NS] (MMAs of the stage finished), full[NS] (operands landed)
  __shared__ uint32_t tslot;
  uint64_t *done = mbar, *full = mbar + TC_MAX_STAGES;
  const int NC = (PART == 0) ? 2 * B : 4 * B;  // D columns per parity
  constexpr int nA = (PART == 0) ? 2 : 4;
  constexpr int UPS = (PART == 0) ? 1 : 2;     // stage units per K step
  constexpr int nU = nA / UPS;                 // tiles per unit
  const int tileB = NC * 32;
  const int abytes = nA * 2 * TILE_A, bbytes = nA * 2 * tileB;   // per K step in global memory
  const int uabytes = nU * 2 * TILE_A, ubbytes = nU * 2 * tileB;  // per unit in shared memory
  const int stage = uabytes + ubbytes;
  const int m = blockIdx.y, pt = blockIdx.x, npt = gridDim.x, p0 = pt * 128;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < 2 * TC_MAX_STAGES; ++i) mbar_init(&mbar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tslot, ncols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tslot;
  const int nsteps = syn_steps(lmax, m);
  const int nunits = nsteps * UPS;
  if (tid == 0) {
    const unsigned char *tabm = tab + (soff[m] * npt + (int64_t)pt * nsteps) * (int64_t)abytes;
    const unsigned char *btm = bt + soff[m] * (int64_t)bbytes;
    const uint32_t idesc = idesc_bf16(128, NC);
    // tile j of unit u: spin 0 tiles {0, 1}; spin 2 parity e tiles {0, 3}, parity o tiles {1, 2}
    auto tile = [&](int u, int j) { return PART == 0 ? j : ((u & 1) == 0 ? 3 * j : 1 + j); };
    auto issue = [&](int u) {
      const int s = u % NS, c = u / UPS;
      unsigned char *dst = sm + s * stage;
      mbar_expect_tx(&full[s], (uint32_t)stage);
      for (int j = 0; j < nU; ++j)
        bulk_g2s(dst + j * 2 * TILE_A, tabm + (int64_t)c * abytes + tile(u, j) * 2 * TILE_A, 2u * TILE_A, &full[s]);
      for (int j = 0; j < nU; ++j)
        bulk_g2s(dst + uabytes + j * 2 * tileB, btm + (int64_t)c * bbytes + tile(u, j) * 2 * tileB,
                 (uint32_t)(2 * tileB), &full[s]);
    };
    for (int u = 0; u < NS && u < nunits; ++u) issue(u);
    // units whose copies were issued, whose operands were waited for, whose MMAs were committed
    int issued = min(NS, nunits), landed = 0, committed = 0;
    bool bad = false;
    for (int u = 0; u < nunits; ++u) {
      const int s = u % NS, c = u / UPS;
      unsigned char *Abuf = sm + s * stage, *Bbuf = Abuf + uabytes;
      if (!mbar_wait(&full[s], (u / NS) & 1, err)) {
        bad = true;
        break;
      }
      landed = u + 1;
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
      // refill the stage of unit u - 1 (its MMAs precede those just issued)
      if (u >= 1 && u - 1 + NS < nunits) {
        if (!mbar_wait(&done[(u - 1) % NS], ((u - 1) / NS) & 1, err)) {
          bad = true;
          break;
        }
        issue(u - 1 + NS);
        issued = u + NS;
      }
    }
    // after a failed wait no more work is issued; copies still in flight (one
    // phase per stage at most) land before the CTA's shared memory goes away
    if (bad)
      for (int v = landed; v < issued; ++v) mbar_wait(&full[v % NS], (v / NS) & 1, err);
    // the last commit covers every MMA issued before it
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

// ----------------------------------------------------------------- analysis
// PART 0: aT    (A = lambda [128 l x 16 pairs], B rows (b, re/im))
// PART 1: aE,aB (A = lam+ with B1 rows (b; E.re, E.im, B.re, B.im) and
//                A = lam- with B2, over 16 pairs per K step)
// grid (groups of LT l tiles of 128 multipoles of one parity, parity, m); rows
// l = m + p + 2 i.  The LT tiles of a CTA share each converted B tile, one
// tensor-memory accumulator of NC columns per tile.
// Output: out[b][f][alm] (FP32 partial sums with a single chunk).

// Warp roles: warps 0 .. 7 convert the ring-coefficient operand of each K
// step into its stage, in ngroups groups of nconv warps that take the steps in
// turn (every thread of the group arrives on full_b), warp 8
// bulk-copies the table tiles (full_a, transaction bytes), warp 9 issues the
// MMAs once both halves of a stage are in and commits them to done, which
// frees the stage; S stages in a ring.  Warps 0-3 read the accumulators after
// the single-use barrier fin that the MMA thread commits last.
constexpr int ANA_THREADS = 320;
constexpr int ANA_MAX_STAGES = 4;

template <int PART>
__global__ void __launch_bounds__(ANA_THREADS, 1) k_ana_tc(const unsigned char *__restrict__ tab,
                                                          const int64_t *__restrict__ aoff,
                                                          const float2 *__restrict__ rc, float2 *__restrict__ out,
                                                          int lmax, int mmax, int npairs, int64_t nalm, int B,
                                                          int LT, uint32_t ncols, int S, int *err, int withhold) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bars[3 * ANA_MAX_STAGES + 1];
  __shared__ uint32_t tslot;
  __shared__ int cta_bad;  // some wait of this CTA gave up
  uint64_t *full_a = bars, *full_b = bars + ANA_MAX_STAGES, *done = bars + 2 * ANA_MAX_STAGES;
  uint64_t *fin = bars + 3 * ANA_MAX_STAGES;  // one phase: every MMA of the CTA has completed
  const int m = blockIdx.z, par = blockIdx.y;
  const int nl = ana_nl(lmax, m, par);
  const int lt0 = blockIdx.x * LT;                                   // first l tile of this CTA
  const int nt = min(LT, (nl > 0 ? (nl + 127) / 128 : 0) - lt0);    // l tiles it takes
  if (nt <= 0) return;  // uniform over the block
  const int NC = (PART == 0) ? 2 * B : 4 * B;
  constexpr int nA = (PART == 0) ? 1 : 2;
  const int tileB = NC * 32;
  const int abytes = nA * 2 * TILE_A;
  const int stage = LT * abytes + nA * 2 * tileB;  // A tiles of the LT l tiles, then B
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntask = (PART == 0) ? 2 * B : 4 * B;  // converter threads with a row pair
  const int nconv = (ntask + 31) / 32;            // warps of one converter group (<= 8)
  // groups of converter warps take the K steps in turn, so that the loads of
  // several steps are in flight when a group alone would wait on each
  const int ngroups = max(1, min(S, 8 / nconv));
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full_a[i], 1);
      mbar_init(&full_b[i], 32 * nconv);
      mbar_init(&done[i], 1);
    }
    mbar_init(fin, 1);
    cta_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tslot, ncols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tslot;
  const int64_t base = abase(lmax, m);
  const int nsteps = (npairs + 15) / 16;
  int issued = 0;  // K steps whose A copies the producer issued
  if (warp < nconv * ngroups) {
    const int grp = warp / nconv, task = tid - grp * 32 * nconv;
    const bool has = task < ntask;
    float2 v[16];
    if (has && grp < nsteps) load_ana_b<PART>(task, rc, m, grp, mmax, npairs, v);
    for (int c = grp; c < nsteps; c += ngroups) {
      const int s = c % S, k = c / S;
      if (c >= S && !mbar_wait(&done[s], (k - 1) & 1, err)) {
        cta_bad = 1;
        break;
      }
      if (has) {
        convert_ana_b<PART>(task, sm + s * stage + LT * abytes, tileB, par, v);
        if (c + ngroups < nsteps) load_ana_b<PART>(task, rc, m, c + ngroups, mmax, npairs, v);
      }
      fence_proxy_async();  // generic-proxy writes -> tensor-core reads
      // test hook (dm_test_tc_withhold): the first converter thread of the
      // first CTA withholds its plain arrival for the first K step, so that the
      // MMA warp's bounded wait gives up with nothing asynchronous in flight
      // that targets the withheld barrier
      if (!(withhold && c == 0 && task == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0))
        mbar_arrive(&full_b[s]);
    }
  } else if (warp == 8 && lane == 0) {
    const unsigned char *tabm = tab + (aoff[2 * m + par] + lt0) * nsteps * (int64_t)abytes;
    const int64_t tstride = (int64_t)nsteps * abytes;  // next l tile
    for (int c = 0; c < nsteps; ++c) {
      const int s = c % S, k = c / S;
      if (c >= S && !mbar_wait(&done[s], (k - 1) & 1, err)) {
        cta_bad = 1;
        break;
      }
      mbar_expect_tx(&full_a[s], (uint32_t)(nt * abytes));
      for (int j = 0; j < nt; ++j)
        bulk_g2s(sm + s * stage + j * abytes, tabm + j * tstride + (int64_t)c * abytes, (uint32_t)abytes, &full_a[s]);
      issued = c + 1;
    }
  } else if (warp == 9 && lane == 0) {
    const uint32_t idesc = idesc_bf16(128, NC);
    for (int c = 0; c < nsteps; ++c) {
      const int s = c % S, k = c / S;
      if (!mbar_wait(&full_a[s], k & 1, err) || !mbar_wait(&full_b[s], k & 1, err)) {
        cta_bad = 1;
        break;
      }
      fence_after_sync();
      const unsigned char *Abuf = sm + s * stage, *Bbuf = Abuf + LT * abytes;
      const uint32_t acc = c > 0 ? 1u : 0u;
      for (int j = 0; j < nt; ++j) {  // one accumulator of NC columns per l tile, the same B
        const unsigned char *Aj = Abuf + j * abytes;
        const uint32_t dj = tbase + (uint32_t)(j * NC);
        mma3(dj, Aj, Bbuf, tileB, idesc, acc);
        if (PART == 1) mma3(dj, Aj + 2 * TILE_A, Bbuf + 2 * tileB, tileB, idesc, 1u);
      }
      commit(&done[s]);
    }
    commit(fin);
  }
  if (warp < 4) {
    // A stage barrier may be several phases behind a warp that did not
    // convert; fin completes exactly once.
    mbar_wait(fin, 0, err);
    __syncwarp();  // converged for the warp-wide tcgen05.ld
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
          for (int q = 0; q < 8; ++q) {
            const int b = (c0 >> 1) + q;
            out[((int64_t)b * 3 + 0) * nalm + idx] = make_float2(v[2 * q], v[2 * q + 1]);
          }
        } else {
          for (int q = 0; q < 4; ++q) {
            const int b = (c0 >> 2) + q;
            out[((int64_t)b * 3 + 1) * nalm + idx] = make_float2(v[4 * q], v[4 * q + 1]);
            out[((int64_t)b * 3 + 2) * nalm + idx] = make_float2(v[4 * q + 2], v[4 * q + 3]);
          }
        }
      }
    }
  }
  // Step c was issued only after the MMAs of step c - S, which waited for its
  // copies, so each stage has at most its last issued phase outstanding.  When
  // any wait of the CTA gave up, those copies land before its shared memory
  // goes away.
  __syncthreads();
  if (cta_bad && warp == 8 && lane == 0)
    for (int c = max(0, issued - S); c < issued; ++c) mbar_wait(&full_a[c % S], (c / S) & 1, err);
  tc_teardown(tbase, ncols);
}

// ------------------------------------------------------------------ launch

bool tc_batch_ok(int B) { return B == 8 || B == 16 || B == 32 || B == 64; }

// Bytes of the four tiled BF16 table copies of a plan and of the synthesis
// operand scratch for B right-hand sides (for memory estimates).
size_t tc_table_bytes(int lmax, int mmax, int npairs, int B) {
  const int64_t npt = (npairs + 127) / 128, nps = (npairs + 15) / 16;
  int64_t ssteps = 0, atiles = 0;
  for (int m = 0; m <= mmax; ++m) {
    ssteps += syn_steps(lmax, m);
    atiles += ana_tiles(lmax, m, 0) + ana_tiles(lmax, m, 1);
  }
  return (size_t)(ssteps * npt * (2 + 4) * 2 * TILE_A + atiles * nps * (1 + 2) * 2 * TILE_A +
                  ssteps * (int64_t)B * (2 * 2 * 64 + 4 * 2 * 128));
}

// Block offsets per m (synthesis) and per (m, parity) (analysis), and the
// per-iteration B operand of the synthesis: needed by both the stored-table
// and the generated-tile kernels.
static cudaError_t tc_scratch(dm_plan *p) {
  if (p->tc_synB[1]) return cudaSuccess;
  std::vector<int64_t> soff(p->mmax + 2, 0), aoff(2 * (p->mmax + 1) + 1, 0);
  for (int m = 0; m <= p->mmax; ++m) {
    soff[m + 1] = soff[m] + syn_steps(p->lmax, m);
    for (int par = 0; par < 2; ++par) aoff[2 * m + par + 1] = aoff[2 * m + par] + ana_tiles(p->lmax, m, par);
  }
  cudaError_t e;
  if (!p->tc_soff) {
    if ((e = cudaMalloc(&p->tc_soff, sizeof(int64_t) * soff.size()))) return e;
    cudaMemcpy(p->tc_soff, soff.data(), sizeof(int64_t) * soff.size(), cudaMemcpyHostToDevice);
  }
  if (!p->tc_aoff) {
    if ((e = cudaMalloc(&p->tc_aoff, sizeof(int64_t) * aoff.size()))) return e;
    cudaMemcpy(p->tc_aoff, aoff.data(), sizeof(int64_t) * aoff.size(), cudaMemcpyHostToDevice);
  }
  const size_t b0 = (size_t)soff[p->mmax + 1] * 2 * 2 * (2 * p->batch * 32);
  const size_t b1 = (size_t)soff[p->mmax + 1] * 4 * 2 * (4 * p->batch * 32);
  if (!p->tc_synB[0]) {
    if ((e = cudaMalloc(&p->tc_synB[0], b0))) return e;
    p->bytes += (int64_t)b0;
  }
  if ((e = cudaMalloc(&p->tc_synB[1], b1))) return e;
  p->bytes += (int64_t)b1;
  return cudaSuccess;
}

// The tiled BF16 hi/lo copies of the FP32 Legendre tables, made on first use.
static cudaError_t tc_tables(dm_plan *p) {
  if (p->tc_synA[1] && p->tc_anaA[1]) return cudaSuccess;
  cudaError_t e = tc_scratch(p);
  if (!e) e = ensure_ptab(p);  // the tiles are cut from the FP32 tables
  if (e) return e;
  const int npt = (p->npairs + 127) / 128, nps = (p->npairs + 15) / 16;
  int64_t ssteps = 0, atiles = 0;
  int max_lt = 0;
  for (int m = 0; m <= p->mmax; ++m) {
    ssteps += syn_steps(p->lmax, m);
    for (int par = 0; par < 2; ++par) {
      atiles += ana_tiles(p->lmax, m, par);
      max_lt = std::max(max_lt, ana_tiles(p->lmax, m, par));
    }
  }
  const size_t sbytes[2] = {(size_t)ssteps * npt * 2 * 2 * TILE_A, (size_t)ssteps * npt * 4 * 2 * TILE_A};
  const size_t abytes[2] = {(size_t)atiles * nps * 1 * 2 * TILE_A, (size_t)atiles * nps * 2 * 2 * TILE_A};
  for (int part = 0; part < 2; ++part) {
    if (!p->tc_synA[part]) {
      if ((e = cudaMalloc(&p->tc_synA[part], sbytes[part]))) return e;
      p->bytes += (int64_t)sbytes[part];
    }
    if (!p->tc_anaA[part]) {
      if ((e = cudaMalloc(&p->tc_anaA[part], abytes[part]))) return e;
      p->bytes += (int64_t)abytes[part];
    }
  }
  dim3 gs(syn_steps(p->lmax, 0), npt, p->mmax + 1);
  k_tab_syn<0><<<gs, 256>>>(p->ptab, p->tc_synA[0], p->tc_soff, p->lmax, p->npairs, p->nalm, npt);
  k_tab_syn<1><<<gs, 256>>>(p->ptab, p->tc_synA[1], p->tc_soff, p->lmax, p->npairs, p->nalm, npt);
  if (max_lt > 0) {
    dim3 ga(nps, max_lt, 2 * (p->mmax + 1));
    k_tab_ana<0><<<ga, 256>>>(p->ptab, p->tc_anaA[0], p->tc_aoff, p->lmax, p->npairs, p->nalm, nps);
    k_tab_ana<1><<<ga, 256>>>(p->ptab, p->tc_anaA[1], p->tc_aoff, p->lmax, p->npairs, p->nalm, nps);
  }
  if ((e = cudaGetLastError())) return e;
  return cudaDeviceSynchronize();
}

// stages per CTA: as many as fit in the shared memory of one CTA, or of two
// when their tensor memory lets two CTAs share an SM (2..TC_MAX_STAGES)
static int tc_stages(int stage_bytes, uint32_t ncols) {
  const int per_sm = ncols <= 256 ? 2 : 1;
  const int ns = (int)(((227u << 10) - 1024u * per_sm) / per_sm) / stage_bytes;
  return ns < 2 ? 2 : (ns > TC_MAX_STAGES ? TC_MAX_STAGES : ns);
}

// a requested stage count within what one CTA's shared memory holds, else the heuristic
static int syn_stages_pick(int want, int stage_bytes, uint32_t ncols) {
  if (want <= 0) return tc_stages(stage_bytes, ncols);
  const int fit = (int)(((227u << 10) - 1024u) / (unsigned)stage_bytes);
  return std::max(2, std::min(want, std::min(fit, TC_MAX_STAGES)));
}

cudaError_t legendre_synthesis_tc(dm_plan *p, const double2 *alm, cudaStream_t st) {
  cudaError_t e = tc_generate(p) ? tc_scratch(p) : tc_tables(p);
  if (e) return e;
  const int B = p->batch;
  const double2 *ahi = p->anchor_active ? p->a_hi : nullptr;
  const int npt = (p->npairs + 127) / 128;
  dim3 gb(syn_steps(p->lmax, 0), p->mmax + 1);
  const float2 *e32 = p->anchor_active ? p->e32 : nullptr;  // iteration: the FP32 state e
  const bool run0 = p->tune_only_part != 1, run1 = p->tune_only_part != 0;
  if (run0) k_syn_b<0><<<gb, TC_THREADS, 0, st>>>(p->tc_synB[0], p->tc_soff, alm, ahi, e32, p->lmax, p->nalm, B);
  if (run1) k_syn_b<1><<<gb, TC_THREADS, 0, st>>>(p->tc_synB[1], p->tc_soff, alm, ahi, e32, p->lmax, p->nalm, B);
  if (tc_generate(p)) return syn_gen_launch(p, run0, run1, st);
  dim3 g(npt, p->mmax + 1);
  if (run0) {
    const int stage = 2 * 2 * TILE_A + 2 * 2 * (2 * B * 32);
    const uint32_t nc = pow2_cols(4 * B);
    const int ns = syn_stages_pick(p->tune_syn_ns[0], stage, nc);
    p->syn_ns_used[0] = ns;
    const size_t sm = tc_smem_n(stage, ns, nc);
    dyn_smem_allow(k_syn_tc<0>, sm);
    k_syn_tc<0><<<g, 128, sm, st>>>(p->tc_synA[0], p->tc_synB[0], p->tc_soff, p->rc32, p->lmax, p->mmax,
                                    p->npairs, B, ns, nc, p->tc_err);
  }
  if (run1) {
    const int stage = 2 * 2 * TILE_A + 2 * 2 * (4 * B * 32);  // half a K step (one parity)
    const uint32_t nc = pow2_cols(8 * B);
    const int ns = syn_stages_pick(p->tune_syn_ns[1], stage, nc);
    p->syn_ns_used[1] = ns;
    const size_t sm = tc_smem_n(stage, ns, nc);
    dyn_smem_allow(k_syn_tc<1>, sm);
    k_syn_tc<1><<<g, 128, sm, st>>>(p->tc_synA[1], p->tc_synB[1], p->tc_soff, p->rc32, p->lmax, p->mmax,
                                    p->npairs, B, ns, nc, p->tc_err);
  }
  return cudaGetLastError();
}

// l tiles per CTA: as many accumulators of NC columns as tensor memory holds (at most 4)
static int ana_tiles_per_cta(int NC) {
  const int nc = (int)pow2_cols(NC);
  const int lt = 512 / nc;
  return lt < 1 ? 1 : (lt > 4 ? 4 : lt);
}

// Stages of the analysis ring: as many as fit (2 to 4), and at least the
// shared memory that keeps the CTAs of an SM within its tensor memory.
static int ana_stages(int stage_bytes) {
  const int fit = (int)(((227u << 10) - 1024) / (size_t)stage_bytes);
  return fit < 2 ? 2 : (fit > ANA_MAX_STAGES ? ANA_MAX_STAGES : fit);
}

// requested l tiles per CTA within tensor memory (LT x NC columns <= 512), else the heuristic
static int ana_lt_pick(int want, int NC) {
  const int mx = ana_tiles_per_cta(NC);
  return want <= 0 ? mx : std::max(1, std::min(want, mx));
}
// requested stages within one CTA's shared memory (2 .. ANA_MAX_STAGES), else the heuristic
static int ana_S_pick(int want, int stage_bytes) {
  if (want <= 0) return ana_stages(stage_bytes);
  const int fit = (int)(((227u << 10) - 1024) / (size_t)stage_bytes);
  return std::max(2, std::min(want, std::min(fit, ANA_MAX_STAGES)));
}

cudaError_t legendre_analysis_tc(dm_plan *p, cudaStream_t st) {
  if (tc_generate(p)) return ana_gen_launch(p, st);
  cudaError_t e = tc_tables(p);
  if (e) return e;
  const int B = p->batch;
  const int ltiles = ana_tiles(p->lmax, 0, 0);
  if (p->tune_only_part != 1) {
    const int NC = 2 * B, LT = ana_lt_pick(p->tune_ana_lt[0], NC);
    const uint32_t nc = pow2_cols(LT * NC);
    const int stage = LT * 1 * 2 * TILE_A + 1 * 2 * (NC * 32);
    const int S = ana_S_pick(p->tune_ana_S[0], stage);
    p->ana_lt_used[0] = LT;
    p->ana_S_used[0] = S;
    const size_t sm = tc_smem_n(stage, S, nc);
    dim3 g((ltiles + LT - 1) / LT, 2, p->mmax + 1);
    dyn_smem_allow(k_ana_tc<0>, sm);
    k_ana_tc<0><<<g, ANA_THREADS, sm, st>>>(p->tc_anaA[0], p->tc_aoff, p->rc32, p->apart32, p->lmax, p->mmax,
                                            p->npairs, p->nalm, B, LT, nc, S, p->tc_err, p->tc_withhold);
  }
  if (p->tune_only_part != 0) {
    const int NC = 4 * B, LT = ana_lt_pick(p->tune_ana_lt[1], NC);
    const uint32_t nc = pow2_cols(LT * NC);
    const int stage = LT * 2 * 2 * TILE_A + 2 * 2 * (NC * 32);
    const int S = ana_S_pick(p->tune_ana_S[1], stage);
    p->ana_lt_used[1] = LT;
    p->ana_S_used[1] = S;
    const size_t sm = tc_smem_n(stage, S, nc);
    dim3 g((ltiles + LT - 1) / LT, 2, p->mmax + 1);
    dyn_smem_allow(k_ana_tc<1>, sm);
    k_ana_tc<1><<<g, ANA_THREADS, sm, st>>>(p->tc_anaA[1], p->tc_aoff, p->rc32, p->apart32, p->lmax, p->mmax,
                                            p->npairs, p->nalm, B, LT, nc, S, p->tc_err, 0);
  }
  return cudaGetLastError();
}

}  // namespace dmwf
