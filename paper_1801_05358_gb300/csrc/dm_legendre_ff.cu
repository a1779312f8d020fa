// dm_legendre_ff.cu -- the Legendre synthesis and analysis (Eq. 2-5 of the
// spin-weighted transforms: F_m(ring) = sum_l lambda_lm(theta) a_lm and its
// transpose over rings) in float-float arithmetic on the FP32 pipe.
//
// A value is carried as an unevaluated sum h + l of two FP32 numbers (about 48
// significant bits).  Tables: the FP64 recurrence values v give h = fl32(v)
// (ptab) and l = fl32(v - h) (ptab_lo).  A product of two such values takes
// the exact rounding error of h1 h2 from one FMA (Dekker / Kahan) plus the two
// cross terms; sums use Knuth's two-sum, so the accumulation loses no more
// than about 2^-48 per term.  The inputs (FP64 a_lm or FP64 ring
// coefficients) are split the same way and the results returned in FP64.
//
// The FP32 pipe of this GPU runs several tens of times faster than its FP64
// pipe, so these kernels give FP64-class results (relative error near 1e-13)
// for the anchors of the mixed mode and for DM_FLOAT_FLOAT at a fraction of
// the FP64 cost.  Products and sums are written with __fmul_rn / __fadd_rn so
// that the compiler does not contract them into FMAs, which would break the
// error-free transformations.
#include <algorithm>

#include "dm_internal.h"

namespace dmwf {

namespace {

constexpr int FF_SYN_THREADS = 128;
constexpr int FF_SYN_CH = 32;
constexpr int FF_ANA_P = 64;
constexpr int FF_ANA_L = 16;
constexpr int FF_ANA_PARTS = FF_ANA_P / FF_ANA_L;

__device__ __forceinline__ int64_t ff_alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }
__device__ __forceinline__ int64_t ff_rc_index(int b, int f, int m, int mmax, int pair, int npairs) {
  return ((((int64_t)b * 3 + f) * (mmax + 1) + m) * npairs + pair) * 2;
}

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_split(double x) {
  const float h = (float)x;
  return ff{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

// s += a * b (a, b float-float), s float-float with a lazily renormalised tail
__device__ __forceinline__ void ff_mac(ff &s, ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float pe = fmaf(a.h, b.h, -p);               // exact: a.h b.h = p + pe
  pe = fmaf(a.h, b.l, fmaf(a.l, b.h, pe));     // cross terms (a.l b.l dropped)
  const float t = __fadd_rn(s.h, p);           // two-sum s.h + p = t + e
  const float bp = __fadd_rn(t, -s.h);
  const float e = __fadd_rn(__fadd_rn(s.h, -__fadd_rn(t, -bp)), __fadd_rn(p, -bp));
  s.h = t;
  s.l = __fadd_rn(s.l, __fadd_rn(e, pe));
}

// s += a (float-float)
__device__ __forceinline__ void ff_add(ff &s, ff a) {
  const float t = __fadd_rn(s.h, a.h);
  const float bp = __fadd_rn(t, -s.h);
  const float e = __fadd_rn(__fadd_rn(s.h, -__fadd_rn(t, -bp)), __fadd_rn(a.h, -bp));
  s.h = t;
  s.l = __fadd_rn(s.l, __fadd_rn(e, a.l));
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }

// One multipole of the synthesis for one RHS; Q = parity of l - m (compile time,
// so that the accumulators stay in registers).
template <int Q>
__device__ __forceinline__ void syn_ff_step(ff (&acc)[2][6], ff lam, ff lp, ff lq, const ff *a) {
  constexpr int QO = Q ^ 1;
  const ff tr = a[0], ti = a[1], ner = a[2], nei = a[3], nbr = a[4], nbi = a[5];
  // T_q += lam aT; Q_q += lam+ (-aE); U_q += lam+ (-aB)
  ff_mac(acc[Q][0], lam, tr);
  ff_mac(acc[Q][1], lam, ti);
  ff_mac(acc[Q][2], lp, ner);
  ff_mac(acc[Q][3], lp, nei);
  ff_mac(acc[Q][4], lp, nbr);
  ff_mac(acc[Q][5], lp, nbi);
  // opposite parity: Q += lam- (-i)(-aB) ; U += lam- (+i)(-aE)
  ff_mac(acc[QO][2], lq, ff_neg(nbi));
  ff_mac(acc[QO][3], lq, nbr);
  ff_mac(acc[QO][4], lq, nei);
  ff_mac(acc[QO][5], lq, ff_neg(ner));
}

// Synthesis: one thread per ring pair, NB right-hand sides; the a_lm of a chunk
// of FF_SYN_CH multipoles are staged in shared memory as float-float.
// Output: ring coefficients rc[b][f][m][pair][side] in FP64.
// Tables: entry (idx(l, m) - base0) * npairs + pair of each function plane
// (plane entries apart), for the orders m0 + blockIdx.z.
template <int NB>
__global__ void __launch_bounds__(FF_SYN_THREADS) k_leg_syn_ff(const float *__restrict__ ptab,
                                                              const float *__restrict__ ptab_lo,
                                                              const double2 *__restrict__ alm,
                                                              double2 *__restrict__ rc, int lmax, int mmax,
                                                              int npairs, int64_t nalm, int batch,
                                                              const SolveState *__restrict__ state, int m0,
                                                              int64_t base0, int64_t plane) {
  // per RHS and l: T (re, im), -E (re, im), -B (re, im), each float-float
  __shared__ ff sA[NB][FF_SYN_CH][6];
  const int b0 = blockIdx.x * NB, m = m0 + blockIdx.z;
  bool any = false;
  for (int k = 0; k < NB; ++k) any = any || (b0 + k < batch && (state == nullptr || !state[b0 + k].done));
  if (!any) return;
  const int p = blockIdx.y * FF_SYN_THREADS + threadIdx.x;
  const bool act = p < npairs;
  const int pp = act ? p : npairs - 1;
  // accumulators [k][parity][T re, T im, Q re, Q im, U re, U im]
  ff acc[NB][2][6];
#pragma unroll
  for (int k = 0; k < NB; ++k)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int i = 0; i < 6; ++i) acc[k][q][i] = ff{0.f, 0.f};
  const int64_t base = ff_alm_base(lmax, m), tbase = base - base0;
  for (int lc = m; lc <= lmax; lc += FF_SYN_CH) {
    const int cnt = min(FF_SYN_CH, lmax + 1 - lc);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * NB; i += FF_SYN_THREADS) {
      const int k = i / cnt, j = i % cnt;
      const int b = min(b0 + k, batch - 1);
      const int64_t ob = (int64_t)b * 3 * nalm + base + lc + j;
      const double2 t = alm[ob], e = alm[ob + nalm], bb = alm[ob + 2 * nalm];
      sA[k][j][0] = ff_split(t.x);
      sA[k][j][1] = ff_split(t.y);
      sA[k][j][2] = ff_split(-e.x);
      sA[k][j][3] = ff_split(-e.y);
      sA[k][j][4] = ff_split(-bb.x);
      sA[k][j][5] = ff_split(-bb.y);
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const int l = lc + j;
      const int64_t o = (tbase + l) * (int64_t)npairs + pp;
      const ff lam{ptab[o], ptab_lo[o]}, lp{ptab[plane + o], ptab_lo[plane + o]},
          lq{ptab[2 * plane + o], ptab_lo[2 * plane + o]};
      if (((l - m) & 1) == 0) {
#pragma unroll
        for (int k = 0; k < NB; ++k) syn_ff_step<0>(acc[k], lam, lp, lq, sA[k][j]);
      } else {
#pragma unroll
        for (int k = 0; k < NB; ++k) syn_ff_step<1>(acc[k], lam, lp, lq, sA[k][j]);
      }
    }
  }
  if (!act) return;
  const bool equator = (p == npairs - 1);
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = b0 + k;
    if (b >= batch || (state != nullptr && state[b].done)) continue;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      double2 *o = rc + ff_rc_index(b, f, m, mmax, p, npairs);
      const double er = ff_to_double(acc[k][0][2 * f]), ei = ff_to_double(acc[k][0][2 * f + 1]);
      const double orr = ff_to_double(acc[k][1][2 * f]), oi = ff_to_double(acc[k][1][2 * f + 1]);
      o[0] = make_double2(er + orr, ei + oi);
      if (!equator) o[1] = make_double2(er - orr, ei - oi);
    }
  }
}

// Analysis partial sums over one chunk of FF_ANA_P ring pairs: thread = ring
// pair while loading, then (l, quarter of the pairs) while contracting.
// Output: apart[b][chunk][f][alm] in FP64.
template <int NB>
__global__ void __launch_bounds__(FF_ANA_P) k_leg_ana_ff(const float *__restrict__ ptab,
                                                        const float *__restrict__ ptab_lo,
                                                        const double2 *__restrict__ rc, double2 *__restrict__ apart,
                                                        int lmax, int mmax, int npairs, int64_t nalm, int c0,
                                                        int slot0, int nslot, int batch,
                                                        const SolveState *__restrict__ state, int m0, int64_t base0,
                                                        int64_t plane) {
  __shared__ ff P[3][FF_ANA_P][FF_ANA_L + 1];
  // per pair and RHS: (T, Q, U) x (even, odd) x (re, im)
  __shared__ ff G[FF_ANA_P][NB][12];
  __shared__ ff red[FF_ANA_PARTS][FF_ANA_L][NB][6];
  const int b0 = blockIdx.x * NB, chunk = c0 + blockIdx.y, slot = slot0 + blockIdx.y, m = m0 + blockIdx.z;
  bool any = false;
  for (int k = 0; k < NB; ++k) any = any || (b0 + k < batch && (state == nullptr || !state[b0 + k].done));
  if (!any) return;
  const int t = threadIdx.x;
  const int p = chunk * FF_ANA_P + t;
  const bool act = p < npairs;
  const int pp = act ? p : npairs - 1;
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = min(b0 + k, batch - 1);
    for (int f = 0; f < 3; ++f) {
      const double2 *g = rc + ff_rc_index(b, f, m, mmax, pp, npairs);
      const double2 gn = act ? g[0] : make_double2(0.0, 0.0);
      const double2 gs = (act && p != npairs - 1) ? g[1] : make_double2(0.0, 0.0);
      G[t][k][4 * f + 0] = ff_split(gn.x + gs.x);
      G[t][k][4 * f + 1] = ff_split(gn.y + gs.y);
      G[t][k][4 * f + 2] = ff_split(gn.x - gs.x);
      G[t][k][4 * f + 3] = ff_split(gn.y - gs.y);
    }
  }
  const int64_t base = ff_alm_base(lmax, m), tbase = base - base0;
  const int lj = t % FF_ANA_L, part = t / FF_ANA_L;
  for (int lc = m; lc <= lmax; lc += FF_ANA_L) {
    const int cnt = min(FF_ANA_L, lmax + 1 - lc);
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const int64_t o = (tbase + lc + j) * (int64_t)npairs + pp;
#pragma unroll
      for (int fn = 0; fn < 3; ++fn)
        P[fn][t][j] = act ? ff{ptab[fn * plane + o], ptab_lo[fn * plane + o]} : ff{0.f, 0.f};
    }
    __syncthreads();
    ff acc[NB][6];
#pragma unroll
    for (int k = 0; k < NB; ++k)
#pragma unroll
      for (int i = 0; i < 6; ++i) acc[k][i] = ff{0.f, 0.f};
    if (lj < cnt) {
      const int l = lc + lj;
      const int par = (l - m) & 1, opp = par ^ 1;
      for (int q = part * FF_ANA_L; q < (part + 1) * FF_ANA_L; ++q) {
        const ff lam = P[0][q][lj], lp = P[1][q][lj], lq = P[2][q][lj];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          const ff *g = G[q][k];
          // aT += lam GT_par ; aE += -lam+ GQ_par + lam- (GU_opp im, -GU_opp re) ;
          // aB += -lam+ GU_par + lam- (-GQ_opp im, GQ_opp re)
          ff_mac(acc[k][0], lam, g[0 + 2 * par]);
          ff_mac(acc[k][1], lam, g[1 + 2 * par]);
          ff_mac(acc[k][2], ff_neg(lp), g[4 + 2 * par]);
          ff_mac(acc[k][2], lq, g[9 + 2 * opp]);
          ff_mac(acc[k][3], ff_neg(lp), g[5 + 2 * par]);
          ff_mac(acc[k][3], ff_neg(lq), g[8 + 2 * opp]);
          ff_mac(acc[k][4], ff_neg(lp), g[8 + 2 * par]);
          ff_mac(acc[k][4], ff_neg(lq), g[5 + 2 * opp]);
          ff_mac(acc[k][5], ff_neg(lp), g[9 + 2 * par]);
          ff_mac(acc[k][5], lq, g[4 + 2 * opp]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NB; ++k)
#pragma unroll
      for (int i = 0; i < 6; ++i) red[part][lj][k][i] = acc[k][i];
    __syncthreads();
    if (part == 0 && lj < cnt) {
      const int l = lc + lj;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const int b = b0 + k;
        if (b >= batch) continue;
        double v[6];
        for (int i = 0; i < 6; ++i) {
          ff a = red[0][lj][k][i];
          for (int q = 1; q < FF_ANA_PARTS; ++q) ff_add(a, red[q][lj][k][i]);
          v[i] = ff_to_double(a);
        }
        double2 *o = apart + ((int64_t)b * nslot + slot) * 3 * nalm + base + l;
        o[0] = make_double2(v[0], v[1]);
        o[nalm] = make_double2(v[2], v[3]);
        o[2 * nalm] = make_double2(v[4], v[5]);
      }
    }
  }
}

}  // namespace

constexpr int FF_NB = 2;

// Slabs of orders whose tables (3 functions, hi and lo) take at most
// p->ffs_cap bytes (one order at least):
// the float-float stages of a plan without the full FP32 tables generate each
// slab's tables (FP64 recurrence) and then contract it.
static cudaError_t ff_slabs(dm_plan *p) {
  if (!p->ffs_m.empty()) return cudaSuccess;
  const size_t cap = (size_t)p->ffs_cap, per_entry = 3 * 2 * sizeof(float) * (size_t)p->npairs;
  std::vector<int> mb{0};
  size_t cur = 0, most = 0;
  for (int m = 0; m <= p->mmax; ++m) {
    const size_t e = (size_t)(p->lmax - m + 1) * per_entry;
    if (cur > 0 && cur + e > cap) {
      mb.push_back(m);
      most = std::max(most, cur);
      cur = 0;
    }
    cur += e;
  }
  mb.push_back(p->mmax + 1);
  most = std::max(most, cur);
  const size_t n = most / (2 * sizeof(float));
  cudaError_t e = cudaMalloc(&p->ffs, sizeof(float) * n);
  if (!e) e = cudaMalloc(&p->ffs_lo, sizeof(float) * n);
  if (e) {
    cudaFree(p->ffs);
    cudaFree(p->ffs_lo);
    p->ffs = p->ffs_lo = nullptr;
    return e;
  }
  p->bytes += (int64_t)(2 * sizeof(float) * n);
  p->ffs_m = mb;
  return cudaSuccess;
}

// Full tables instead of slabs when they are cheap to keep: when they fit in
// one slab, and, unless the slab size was set (dm_set_ff_slab_bytes), in
// DM_FLOAT_FLOAT (which reads them every iteration, not only at the mixed
// mode's anchors) when they take at most 32 GiB.
static cudaError_t ff_tables(dm_plan *p) {
  if (p->ptab) return cudaSuccess;
  const double full = 6.0 * sizeof(float) * (double)p->nalm * p->npairs;
  if (full <= (double)p->ffs_cap || (p->ff_legendre && !p->ffs_cap_set && full <= 32.0 * (1u << 30)))
    return ensure_ptab(p);
  return cudaSuccess;
}

cudaError_t legendre_synthesis_ff(dm_plan *p, const double2 *alm, cudaStream_t st) {
  const SolveState *stp = p->state_active ? p->state : nullptr;
  if (cudaError_t e = ff_tables(p)) return e;
  if (p->ptab) {
    dim3 g((p->batch + FF_NB - 1) / FF_NB, (p->npairs + FF_SYN_THREADS - 1) / FF_SYN_THREADS, p->mmax + 1);
    k_leg_syn_ff<FF_NB><<<g, FF_SYN_THREADS, 0, st>>>(p->ptab, p->ptab_lo, alm, p->rc, p->lmax, p->mmax, p->npairs,
                                                      p->nalm, p->batch, stp, 0, 0, p->nalm * (int64_t)p->npairs);
    return cudaGetLastError();
  }
  if (cudaError_t e = ff_slabs(p)) return e;
  for (size_t k = 0; k + 1 < p->ffs_m.size(); ++k) {
    const int m0 = p->ffs_m[k], m1 = p->ffs_m[k + 1];
    if (cudaError_t e = gen_tables32_slab(p, p->ffs, p->ffs_lo, m0, m1, st)) return e;
    const int64_t b0 = alm_start_h(p->lmax, m0), b1 = alm_start_h(p->lmax, m1);
    dim3 g((p->batch + FF_NB - 1) / FF_NB, (p->npairs + FF_SYN_THREADS - 1) / FF_SYN_THREADS, m1 - m0);
    k_leg_syn_ff<FF_NB><<<g, FF_SYN_THREADS, 0, st>>>(p->ffs, p->ffs_lo, alm, p->rc, p->lmax, p->mmax, p->npairs,
                                                      p->nalm, p->batch, stp, m0, b0,
                                                      (b1 - b0) * (int64_t)p->npairs);
  }
  return cudaGetLastError();
}

// partial sums per chunk of 64 ring pairs into p->apart (the FP64 reduction
// follows), in chunk waves when the plan holds fewer slots than chunks
// (chunk_waves); *used = the slots holding the sums
cudaError_t legendre_analysis_ff_parts(dm_plan *p, cudaStream_t st, int *used) {
  const SolveState *stp = p->state_active ? p->state : nullptr;
  if (cudaError_t e = ff_tables(p)) return e;
  if (p->ptab) {
    return chunk_waves(p, 0, p->mmax + 1, st, [&](int c0, int slot0, int n, int m0, int m1) {
      dim3 g((p->batch + FF_NB - 1) / FF_NB, n, m1 - m0);
      k_leg_ana_ff<FF_NB><<<g, FF_ANA_P, 0, st>>>(p->ptab, p->ptab_lo, p->rc, p->apart, p->lmax, p->mmax,
                                                  p->npairs, p->nalm, c0, slot0, p->nslot, p->batch, stp, m0, 0,
                                                  p->nalm * (int64_t)p->npairs);
      return cudaGetLastError();
    }, used);
  }
  if (cudaError_t e = ff_slabs(p)) return e;
  for (size_t k = 0; k + 1 < p->ffs_m.size(); ++k) {
    const int s0 = p->ffs_m[k], s1 = p->ffs_m[k + 1];
    if (cudaError_t e = gen_tables32_slab(p, p->ffs, p->ffs_lo, s0, s1, st)) return e;
    const int64_t b0 = alm_start_h(p->lmax, s0), b1 = alm_start_h(p->lmax, s1);
    cudaError_t e = chunk_waves(p, s0, s1, st, [&](int c0, int slot0, int n, int m0, int m1) {
      dim3 g((p->batch + FF_NB - 1) / FF_NB, n, m1 - m0);
      k_leg_ana_ff<FF_NB><<<g, FF_ANA_P, 0, st>>>(p->ffs, p->ffs_lo, p->rc, p->apart, p->lmax, p->mmax, p->npairs,
                                                  p->nalm, c0, slot0, p->nslot, p->batch, stp, m0, b0,
                                                  (b1 - b0) * (int64_t)p->npairs);
      return cudaGetLastError();
    }, used);
    if (e) return e;
  }
  return cudaGetLastError();
}

}  // namespace dmwf
