// dm_legendre.cu -- FP64 Legendre/Wigner-d stages of the spherical harmonic
// transforms: the harmonic-space half of a dual messenger iteration.
//
// Synthesis (F in Algorithm 1), per order m and ring pair (theta, pi - theta):
//   F^T = sum_l aT lambda,  F^Q = -sum_l (aE lam+ + i aB lam-),
//   F^U = -sum_l (aB lam+ - i aE lam-),  lam+- = (2lambda +- -2lambda)/2.
// Analysis (sigma^{-1} F^dagger), the Omega-scaled adjoint:
//   aT = Omega sum_r lambda G^T,  aE = -Omega sum_r (lam+ G^Q + i lam- G^U),
//   aB = -Omega sum_r (lam+ G^U - i lam- G^Q).
// The recurrences (spin 0 and the lam+- pair of the k = -+2 Wigner-d
// recurrence) run on the fly in FP64 from per-(m, pair) seeds, one ring pair
// per thread; the mirror ring comes from the parities
//   lambda(pi - theta) = (-1)^{l+m} lambda,  lam+(pi - theta) = (-1)^{l+m} lam+,
//   lam-(pi - theta) = -(-1)^{l+m} lam-.
// Seeds below 2^-600 are carried as v 2^-S (S >= 600) and advanced without
// accumulation until they become representable (negligible region).
#include "dm_fft.cuh"
#include "dm_internal.h"
#include "dm_rec.cuh"

namespace dmwf {

__device__ __forceinline__ int64_t alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }
__device__ __forceinline__ int64_t rc_index2(int b, int f, int m, int mmax, int pair, int npairs) {
  return ((((int64_t)b * 3 + f) * (mmax + 1) + m) * npairs + pair) * 2;
}

// ------------------------------------------------------------- synthesis
constexpr int SYN_THREADS = 128;
constexpr int SYN_CH = 64;

__global__ void __launch_bounds__(SYN_THREADS) k_leg_syn64(const PairDev *__restrict__ pairs,
                                                           const RecCoef *__restrict__ rec,
                                                           const double *__restrict__ seed,
                                                           const int *__restrict__ seed_exp,
                                                           const double2 *__restrict__ alm, double2 *__restrict__ rc,
                                                           int lmax, int mmax, int npairs, int64_t nalm,
                                                           const SolveState *__restrict__ state) {
  __shared__ double2 sT[SYN_CH], sE[SYN_CH], sB[SYN_CH];
  __shared__ RecCoef sc[SYN_CH];
  const int m = blockIdx.y, b = blockIdx.z;
  if (state != nullptr && state[b].done) return;
  const int p = blockIdx.x * SYN_THREADS + threadIdx.x;
  const bool act = p < npairs;
  const int pp = act ? p : npairs - 1;
  const double x = pairs[pp].x;
  Rec s;
  rec_init(s, seed, seed_exp, m, pp, npairs);
  // accumulators: index 0 = parity of (l + m) even, 1 = odd
  double2 T0 = {0, 0}, T1 = {0, 0}, Q0 = {0, 0}, Q1 = {0, 0}, U0 = {0, 0}, U1 = {0, 0};
  const int64_t base = alm_base(lmax, m);
  const double2 *aT = alm + ((int64_t)b * 3 + 0) * nalm + base;
  const double2 *aE = alm + ((int64_t)b * 3 + 1) * nalm + base;
  const double2 *aB = alm + ((int64_t)b * 3 + 2) * nalm + base;
  for (int lc = m; lc <= lmax; lc += SYN_CH) {
    const int cnt = min(SYN_CH, lmax + 1 - lc);
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += SYN_THREADS) {
      const int l = lc + j;
      sT[j] = aT[l];
      double2 e = aE[l], bb = aB[l];
      sE[j] = make_double2(-e.x, -e.y);   // -aE
      sB[j] = make_double2(-bb.x, -bb.y); // -aB
      sc[j] = rec[base + l + 1];          // coefficients of target l + 1
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const int l = lc + j;
      if (s.S == 0) {
        const double2 t = sT[j], ne = sE[j], nb = sB[j];
        const double lam = s.l0, lp = 0.5 * (s.p0 + s.q0), lq = 0.5 * (s.p0 - s.q0);
        if (((l - m) & 1) == 0) {
          T0.x = fma(t.x, lam, T0.x); T0.y = fma(t.y, lam, T0.y);
          Q0.x = fma(ne.x, lp, Q0.x); Q0.y = fma(ne.y, lp, Q0.y);   // -aE lam+
          U0.x = fma(nb.x, lp, U0.x); U0.y = fma(nb.y, lp, U0.y);   // -aB lam+
          Q1.x = fma(-nb.y, lq, Q1.x); Q1.y = fma(nb.x, lq, Q1.y);  // -i aB lam-
          U1.x = fma(ne.y, lq, U1.x); U1.y = fma(-ne.x, lq, U1.y);  // +i aE lam-
        } else {
          T1.x = fma(t.x, lam, T1.x); T1.y = fma(t.y, lam, T1.y);
          Q1.x = fma(ne.x, lp, Q1.x); Q1.y = fma(ne.y, lp, Q1.y);
          U1.x = fma(nb.x, lp, U1.x); U1.y = fma(nb.y, lp, U1.y);
          Q0.x = fma(-nb.y, lq, Q0.x); Q0.y = fma(nb.x, lq, Q0.y);
          U0.x = fma(ne.y, lq, U0.x); U0.y = fma(-ne.x, lq, U0.y);
        }
      }
      if (l < lmax) rec_advance(s, sc[j], x, m, l, seed, pp, npairs);
    }
  }
  if (!act) return;
  const bool equator = (p == npairs - 1);
  double2 *o0 = rc + rc_index2(b, 0, m, mmax, p, npairs);
  double2 *o1 = rc + rc_index2(b, 1, m, mmax, p, npairs);
  double2 *o2 = rc + rc_index2(b, 2, m, mmax, p, npairs);
  o0[0] = cadd(T0, T1);
  o1[0] = cadd(Q0, Q1);
  o2[0] = cadd(U0, U1);
  if (!equator) {
    o0[1] = csub(T0, T1);
    o1[1] = csub(Q0, Q1);
    o2[1] = csub(U0, U1);
  }
}

cudaError_t legendre_synthesis32(dm_plan *p, const double2 *alm, cudaStream_t st);
cudaError_t legendre_analysis32(dm_plan *p, int epilogue, double2 *out, cudaStream_t st, cudaEvent_t mid);

cudaError_t legendre_synthesis(dm_plan *p, const double2 *alm, cudaStream_t st) {
  if (p->flat) return flat_synthesis(p, alm, st);  // flat sky: column transforms (dm_flat.cu)
  if (p->prec != DM_FP64) return legendre_synthesis32(p, alm, st);
  if (p->ff_legendre || p->ff_now) return legendre_synthesis_ff(p, alm, st);
  dim3 grid((p->npairs + SYN_THREADS - 1) / SYN_THREADS, p->mmax + 1, p->batch);
  k_leg_syn64<<<grid, SYN_THREADS, 0, st>>>(p->pairs, p->rec, p->seed, p->seed_exp, alm, p->rc, p->lmax, p->mmax,
                                           p->npairs, p->nalm, p->state_active ? p->state : nullptr);
  return cudaGetLastError();
}

// -------------------------------------------------------------- analysis
// Block = ANA_P ring pairs x one m.  For each chunk of ANA_L multipoles:
//  phase A: thread = pair, runs the recurrence, writes lambda, lam+, lam- to smem;
//  phase B: thread = (l, half of the pairs), contracts over pairs in FP64.
// Partial sums per pair chunk go to apart[b][chunk][f][alm]; k_ana_reduce
// sums the chunks in a fixed order (deterministic).
constexpr int ANA_P = 64;
constexpr int ANA_L = 16;
constexpr int ANA_PARTS = ANA_P / ANA_L;

__global__ void __launch_bounds__(ANA_P) k_leg_ana64(const PairDev *__restrict__ pairs,
                                                     const RecCoef *__restrict__ rec,
                                                     const double *__restrict__ seed,
                                                     const int *__restrict__ seed_exp,
                                                     const double2 *__restrict__ rc, double2 *__restrict__ apart,
                                                     int lmax, int mmax, int npairs, int64_t nalm, int c0,
                                                     int slot0, int nslot, const SolveState *__restrict__ state) {
  __shared__ double P0[ANA_P][ANA_L + 1], Pp[ANA_P][ANA_L + 1], Pq[ANA_P][ANA_L + 1];
  // per pair: GT even, GT odd, GQ even, GQ odd, GU even, GU odd (complex)
  __shared__ double2 G[ANA_P][6];
  __shared__ double red[ANA_PARTS][ANA_L][6];
  __shared__ RecCoef sc[ANA_L];
  const int m = blockIdx.y, b = blockIdx.z, chunk = c0 + blockIdx.x, slot = slot0 + blockIdx.x;
  if (state != nullptr && state[b].done) return;
  const int t = threadIdx.x;
  const int p = chunk * ANA_P + t;
  const bool act = p < npairs;
  const int pp = act ? p : npairs - 1;
  const double x = pairs[pp].x;
  {
    double2 gn[3], gs[3];
    for (int f = 0; f < 3; ++f) {
      const double2 *g = rc + rc_index2(b, f, m, mmax, pp, npairs);
      gn[f] = act ? g[0] : make_double2(0, 0);
      gs[f] = (act && p != npairs - 1) ? g[1] : make_double2(0, 0);  // equator: no mirror ring
    }
    for (int f = 0; f < 3; ++f) {
      G[t][2 * f] = cadd(gn[f], gs[f]);
      G[t][2 * f + 1] = csub(gn[f], gs[f]);
    }
  }
  Rec s;
  rec_init(s, seed, seed_exp, m, pp, npairs);
  const int64_t base = alm_base(lmax, m);
  const int lj = t % ANA_L, part = t / ANA_L;
  for (int lc = m; lc <= lmax; lc += ANA_L) {
    const int cnt = min(ANA_L, lmax + 1 - lc);
    __syncthreads();
    if (t < cnt) sc[t] = rec[base + lc + t + 1];
    __syncthreads();
    // phase A
    for (int j = 0; j < cnt; ++j) {
      const int l = lc + j;
      const bool live = (s.S == 0) && act;
      P0[t][j] = live ? s.l0 : 0.0;
      Pp[t][j] = live ? 0.5 * (s.p0 + s.q0) : 0.0;
      Pq[t][j] = live ? 0.5 * (s.p0 - s.q0) : 0.0;
      if (l < lmax) rec_advance(s, sc[j], x, m, l, seed, pp, npairs);
    }
    __syncthreads();
    // phase B: thread (lj, part) sums pairs [part*ANA_L, part*ANA_L + ANA_L)
    double aTr = 0, aTi = 0, aEr = 0, aEi = 0, aBr = 0, aBi = 0;
    if (lj < cnt) {
      const int l = lc + lj;
      const int par = (l - m) & 1, opp = par ^ 1;
      for (int q = part * ANA_L; q < (part + 1) * ANA_L; ++q) {
        const double lam = P0[q][lj], lp = Pp[q][lj], lq = Pq[q][lj];
        const double2 gt = G[q][par], gqp = G[q][2 + par], gup = G[q][4 + par];
        const double2 gqo = G[q][2 + opp], guo = G[q][4 + opp];
        aTr = fma(lam, gt.x, aTr);
        aTi = fma(lam, gt.y, aTi);
        // aE = -(lam+ GQ_par + i lam- GU_opp)
        aEr = fma(-lp, gqp.x, fma(lq, guo.y, aEr));
        aEi = fma(-lp, gqp.y, fma(-lq, guo.x, aEi));
        // aB = -(lam+ GU_par - i lam- GQ_opp)
        aBr = fma(-lp, gup.x, fma(-lq, gqo.y, aBr));
        aBi = fma(-lp, gup.y, fma(lq, gqo.x, aBi));
      }
    }
    red[part][lj][0] = aTr; red[part][lj][1] = aTi; red[part][lj][2] = aEr;
    red[part][lj][3] = aEi; red[part][lj][4] = aBr; red[part][lj][5] = aBi;
    __syncthreads();
    if (part == 0 && lj < cnt) {
      const int l = lc + lj;
      double v[6];
      for (int k = 0; k < 6; ++k) {
        double a = red[0][lj][k];
        for (int q = 1; q < ANA_PARTS; ++q) a += red[q][lj][k];
        v[k] = a;
      }
      double2 *o = apart + ((int64_t)b * nslot + slot) * 3 * nalm + base + l;
      o[0] = make_double2(v[0], v[1]);
      o[nalm] = make_double2(v[2], v[3]);
      o[2 * nalm] = make_double2(v[4], v[5]);
    }
  }
}

// Sum the pair chunks, scale by Omega; epilogue:
//  ANA_PLAIN   : out = Omega sum
//  ANA_DM_STEP : out = F_level (out + Omega sum)   (a <- F [a + A (t - s)])
// grid: (l blocks, batch, m)
__global__ void k_ana_reduce(const double2 *__restrict__ apart, double2 *out, int lmax, int64_t nalm, int nchunk,
                             int nslot, double omega, int epilogue, const double *__restrict__ filt, int nlev,
                             const SolveState *__restrict__ state, const double2 *__restrict__ src) {
  const int b = blockIdx.y, m = blockIdx.z;
  if (state != nullptr && state[b].done) return;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const int64_t i = alm_base(lmax, m) + l;
  double2 acc[3];
  for (int f = 0; f < 3; ++f) {
    double2 a = make_double2(0, 0);
    for (int c = 0; c < nchunk; ++c) a = cadd(a, apart[(((int64_t)b * nslot + c) * 3 + f) * nalm + i]);
    acc[f] = make_double2(omega * a.x, omega * a.y);
  }
  double2 *o = out + (int64_t)b * 3 * nalm + i;
  if (epilogue == ANA_PLAIN) {
    o[0] = acc[0];
    o[nalm] = acc[1];
    o[2 * nalm] = acc[2];
    return;
  }
  const double *c = filt + (((int64_t)b * nlev + state[b].level) * (lmax + 1) + l) * 4;
  if (src != nullptr) {  // a harmonic source (the Jacobi refinement's W~ runs): a <- F [a + g + A (t - s)]
    const double2 *g = src + (int64_t)b * 3 * nalm + i;
    acc[0] = cadd(acc[0], g[0]);
    acc[1] = cadd(acc[1], g[nalm]);
    acc[2] = cadd(acc[2], g[2 * nalm]);
  }
  double2 t = cadd(o[0], acc[0]), e = cadd(o[nalm], acc[1]), bb = cadd(o[2 * nalm], acc[2]);
  o[0] = make_double2(c[0] * t.x + c[1] * e.x, c[0] * t.y + c[1] * e.y);
  o[nalm] = make_double2(c[1] * t.x + c[2] * e.x, c[1] * t.y + c[2] * e.y);
  o[2 * nalm] = make_double2(c[3] * bb.x, c[3] * bb.y);
}

// Slot 0 += slots 1 .. nused - 1 for the orders [m0, m0 + gridDim.z)
// (grid: l blocks, batch, orders)
__global__ void k_fold_slots(double2 *apart, int nslot, int nused, int lmax, int64_t nalm, int m0,
                             const SolveState *__restrict__ state) {
  const int b = blockIdx.y, m = m0 + blockIdx.z;
  if (state != nullptr && state[b].done) return;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const int64_t i = alm_base(lmax, m) + l;
  for (int f = 0; f < 3; ++f) {
    double2 a = apart[(((int64_t)b * nslot) * 3 + f) * nalm + i];
    for (int c = 1; c < nused; ++c) a = cadd(a, apart[(((int64_t)b * nslot + c) * 3 + f) * nalm + i]);
    apart[(((int64_t)b * nslot) * 3 + f) * nalm + i] = a;
  }
}

cudaError_t fold_slots(dm_plan *p, int nused, int m0, int m1, cudaStream_t st) {
  if (nused <= 1 || m1 <= m0) return cudaSuccess;
  dim3 g((unsigned)((p->lmax + 1 + 127) / 128), p->batch, m1 - m0);
  k_fold_slots<<<g, 128, 0, st>>>(p->apart, p->nslot, nused, p->lmax, p->nalm, m0,
                                  p->state_active ? p->state : nullptr);
  return cudaGetLastError();
}

cudaError_t analysis64_parts(dm_plan *p, cudaStream_t st, int *used) {
  const SolveState *stp = p->state_active ? p->state : nullptr;
  return chunk_waves(p, 0, p->mmax + 1, st, [&](int c0, int slot0, int n, int m0, int m1) {
    dim3 grid(n, m1 - m0, p->batch);
    k_leg_ana64<<<grid, ANA_P, 0, st>>>(p->pairs, p->rec, p->seed, p->seed_exp, p->rc, p->apart, p->lmax, p->mmax,
                                        p->npairs, p->nalm, c0, slot0, p->nslot, stp);
    return cudaGetLastError();
  }, used);
}

cudaError_t legendre_analysis(dm_plan *p, int epilogue, double2 *out, cudaStream_t st, cudaEvent_t mid) {
  if (p->flat) return flat_analysis(p, epilogue, out, st, mid);
  if (p->prec != DM_FP64) return legendre_analysis32(p, epilogue, out, st, mid);
  const SolveState *stp = p->state_active ? p->state : nullptr;
  int used = p->nchunk;
  cudaError_t e = (p->ff_legendre || p->ff_now) ? legendre_analysis_ff_parts(p, st, &used)
                                                : analysis64_parts(p, st, &used);
  if (e) return e;
  if (mid) cudaEventRecord(mid, st);
  double omega = 4.0 * M_PI / (double)p->npix;
  dim3 g2((unsigned)((p->lmax + 1 + 127) / 128), p->batch, p->mmax + 1);
  k_ana_reduce<<<g2, 128, 0, st>>>(p->apart, out, p->lmax, p->nalm, used, p->nslot, omega, epilogue, p->filt,
                                   p->filt_levels,
                                   epilogue == ANA_DM_STEP ? p->state : stp,
                                   (epilogue == ANA_DM_STEP && p->src_active) ? p->jsrc : nullptr);
  return cudaGetLastError();
}

// standalone filter (for testing the a3 step): out = F in, coefficients given
__global__ void k_apply_filter(const double *__restrict__ coef, const double2 *in, double2 *out, int lmax,
                               int64_t nalm) {
  const int b = blockIdx.y;
  const int m = blockIdx.z;
  const int64_t base = alm_base(lmax, m);
  for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
    const double *c = coef + 4 * l;
    const double2 *ip = in + (int64_t)b * 3 * nalm + base + l;
    double2 *op = out + (int64_t)b * 3 * nalm + base + l;
    double2 t = ip[0], e = ip[nalm], bb = ip[2 * nalm];
    op[0] = make_double2(c[0] * t.x + c[1] * e.x, c[0] * t.y + c[1] * e.y);
    op[nalm] = make_double2(c[1] * t.x + c[2] * e.x, c[1] * t.y + c[2] * e.y);
    op[2 * nalm] = make_double2(c[3] * bb.x, c[3] * bb.y);
  }
}

cudaError_t apply_filter_level(dm_plan *p, const double *coef, const double2 *in, double2 *out, cudaStream_t st) {
  k_apply_filter<<<dim3(1, p->batch, p->mmax + 1), 128, 0, st>>>(coef, in, out, p->lmax, p->nalm);
  return cudaGetLastError();
}

// ======================================================================
// DM_MIXED_FP32: Legendre values from the FP64 recurrence, stored once in
// FP32 tables ptab[f][idx(l, m)][pair] (f = lambda, lam+, lam-); FP32
// contraction; FP32 ring coefficients; FP64 harmonic state and filter.
// ======================================================================

// Tables of the orders m0 + blockIdx.y: entry (idx(l, m) - base0) * npairs +
// pair of each function plane (plane entries apart), base0 = idx(m0, m0).
__global__ void __launch_bounds__(128) k_gen_tables(const PairDev *__restrict__ pairs, const RecCoef *__restrict__ rec,
                                                    const double *__restrict__ seed, const int *__restrict__ seed_exp,
                                                    float *__restrict__ ptab, float *__restrict__ ptab_lo, int lmax,
                                                    int npairs, int m0, int64_t base0, int64_t plane) {
  __shared__ RecCoef sc[SYN_CH];
  const int m = m0 + blockIdx.y;
  const int p = blockIdx.x * 128 + threadIdx.x;
  const bool act = p < npairs;
  const int pp = act ? p : npairs - 1;
  const double x = pairs[pp].x;
  Rec s;
  rec_init(s, seed, seed_exp, m, pp, npairs);
  const int64_t base = alm_base(lmax, m);
  for (int lc = m; lc <= lmax; lc += SYN_CH) {
    const int cnt = min(SYN_CH, lmax + 1 - lc);
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += 128) sc[j] = rec[base + lc + j + 1];
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const int l = lc + j;
      if (act) {
        const int64_t o = (base + l - base0) * (int64_t)npairs + p;
        const bool live = (s.S == 0);
        const double v0 = live ? s.l0 : 0.0, v1 = live ? 0.5 * (s.p0 + s.q0) : 0.0,
                     v2 = live ? 0.5 * (s.p0 - s.q0) : 0.0;
        const float h0 = (float)v0, h1 = (float)v1, h2 = (float)v2;
        ptab[o] = h0;
        ptab[plane + o] = h1;
        ptab[2 * plane + o] = h2;
        ptab_lo[o] = (float)(v0 - (double)h0);
        ptab_lo[plane + o] = (float)(v1 - (double)h1);
        ptab_lo[2 * plane + o] = (float)(v2 - (double)h2);
      }
      if (l < lmax) rec_advance(s, sc[j], x, m, l, seed, pp, npairs);
    }
  }
}

// Tables of the orders [m0, m1) into hi / lo, laid out as the full tables
// restricted to those orders (planes of (idx(m1, m1) - idx(m0, m0)) x npairs).
cudaError_t gen_tables32_slab(dm_plan *p, float *hi, float *lo, int m0, int m1, cudaStream_t st) {
  if (m1 <= m0) return cudaSuccess;
  const int64_t b0 = alm_start_h(p->lmax, m0), b1 = alm_start_h(p->lmax, m1);
  dim3 g((p->npairs + 127) / 128, m1 - m0);
  k_gen_tables<<<g, 128, 0, st>>>(p->pairs, p->rec, p->seed, p->seed_exp, hi, lo, p->lmax, p->npairs, m0, b0,
                                  (b1 - b0) * (int64_t)p->npairs);
  return cudaGetLastError();
}

// Synthesis, FP32 contraction over l; NB right-hand sides per thread.
// grid: (batch / NB, pair blocks, m); consecutive blocks share the table tile in L2.
template <int NB>
__global__ void __launch_bounds__(SYN_THREADS) k_leg_syn32(const float *__restrict__ ptab,
                                                           const double2 *__restrict__ alm,
                                                           const double2 *__restrict__ a_sub,
                                                           const float2 *__restrict__ e32,
                                                           float2 *__restrict__ rc, int lmax, int mmax, int npairs,
                                                           int64_t nalm, const SolveState *__restrict__ state) {
  __shared__ float2 sT[NB][SYN_CH], sE[NB][SYN_CH], sB[NB][SYN_CH];
  const int b0 = blockIdx.x * NB, m = blockIdx.z;
  bool any = false;
  for (int k = 0; k < NB; ++k) any = any || state == nullptr || !state[b0 + k].done;
  if (!any) return;
  const int p = blockIdx.y * SYN_THREADS + threadIdx.x;
  const bool act = p < npairs;
  const int pp = act ? p : npairs - 1;
  float2 T0[NB], T1[NB], Q0[NB], Q1[NB], U0[NB], U1[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    T0[k] = T1[k] = Q0[k] = Q1[k] = U0[k] = U1[k] = make_float2(0.f, 0.f);
  }
  const int64_t base = alm_base(lmax, m);
  const int64_t plane = nalm * (int64_t)npairs;
  const float *P0 = ptab + base * npairs + pp, *Pp = P0 + plane, *Pq = P0 + 2 * plane;
  for (int lc = m; lc <= lmax; lc += SYN_CH) {
    const int cnt = min(SYN_CH, lmax + 1 - lc);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * NB; i += SYN_THREADS) {
      const int k = i / cnt, j = i % cnt;
      const int64_t ob = (int64_t)(b0 + k) * 3 * nalm + base + lc + j;
      if (e32 != nullptr) {  // FP32 iteration state e = a - a_hi
        const float2 t = e32[ob], e = e32[ob + nalm], bb = e32[ob + 2 * nalm];
        sT[k][j] = t;
        sE[k][j] = make_float2(-e.x, -e.y);
        sB[k][j] = make_float2(-bb.x, -bb.y);
        continue;
      }
      double2 t = alm[ob], e = alm[ob + nalm], bb = alm[ob + 2 * nalm];
      if (a_sub != nullptr) {  // correction e = a - a_hi (FP64 difference, then FP32)
        t = csub(t, a_sub[ob]);
        e = csub(e, a_sub[ob + nalm]);
        bb = csub(bb, a_sub[ob + 2 * nalm]);
      }
      sT[k][j] = make_float2((float)t.x, (float)t.y);
      sE[k][j] = make_float2((float)-e.x, (float)-e.y);
      sB[k][j] = make_float2((float)-bb.x, (float)-bb.y);
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const int l = lc + j;
      const int64_t o = (int64_t)l * npairs;  // table entry idx(l, m) = base + l
      const float lam = P0[o], lp = Pp[o], lq = Pq[o];
      if (((l - m) & 1) == 0) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          const float2 t = sT[k][j], ne = sE[k][j], nb = sB[k][j];
          T0[k].x = fmaf(t.x, lam, T0[k].x); T0[k].y = fmaf(t.y, lam, T0[k].y);
          Q0[k].x = fmaf(ne.x, lp, Q0[k].x); Q0[k].y = fmaf(ne.y, lp, Q0[k].y);
          U0[k].x = fmaf(nb.x, lp, U0[k].x); U0[k].y = fmaf(nb.y, lp, U0[k].y);
          Q1[k].x = fmaf(-nb.y, lq, Q1[k].x); Q1[k].y = fmaf(nb.x, lq, Q1[k].y);
          U1[k].x = fmaf(ne.y, lq, U1[k].x); U1[k].y = fmaf(-ne.x, lq, U1[k].y);
        }
      } else {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          const float2 t = sT[k][j], ne = sE[k][j], nb = sB[k][j];
          T1[k].x = fmaf(t.x, lam, T1[k].x); T1[k].y = fmaf(t.y, lam, T1[k].y);
          Q1[k].x = fmaf(ne.x, lp, Q1[k].x); Q1[k].y = fmaf(ne.y, lp, Q1[k].y);
          U1[k].x = fmaf(nb.x, lp, U1[k].x); U1[k].y = fmaf(nb.y, lp, U1[k].y);
          Q0[k].x = fmaf(-nb.y, lq, Q0[k].x); Q0[k].y = fmaf(nb.x, lq, Q0[k].y);
          U0[k].x = fmaf(ne.y, lq, U0[k].x); U0[k].y = fmaf(-ne.x, lq, U0[k].y);
        }
      }
    }
  }
  if (!act) return;
  const bool equator = (p == npairs - 1);
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = b0 + k;
    if (state != nullptr && state[b].done) continue;
    float2 *o0 = rc + rc_index2(b, 0, m, mmax, p, npairs);
    float2 *o1 = rc + rc_index2(b, 1, m, mmax, p, npairs);
    float2 *o2 = rc + rc_index2(b, 2, m, mmax, p, npairs);
    o0[0] = cadd(T0[k], T1[k]);
    o1[0] = cadd(Q0[k], Q1[k]);
    o2[0] = cadd(U0[k], U1[k]);
    if (!equator) {
      o0[1] = csub(T0[k], T1[k]);
      o1[1] = csub(Q0[k], Q1[k]);
      o2[1] = csub(U0[k], U1[k]);
    }
  }
}

// Analysis, FP32: P tile from the table into smem, then the per-l contraction
// over the pairs of the chunk (same structure as k_leg_ana64), NB RHS per block.
template <int NB>
__global__ void __launch_bounds__(ANA_P) k_leg_ana32(const float *__restrict__ ptab, const float2 *__restrict__ rc,
                                                     float2 *__restrict__ apart, int lmax, int mmax, int npairs,
                                                     int64_t nalm, int nchunk, const SolveState *__restrict__ state) {
  __shared__ float P0[ANA_P][ANA_L + 1], Pp[ANA_P][ANA_L + 1], Pq[ANA_P][ANA_L + 1];
  __shared__ float4 G[ANA_P][NB][3];  // (GT_e, GT_o), (GQ_e, GQ_o), (GU_e, GU_o)
  __shared__ float red[ANA_PARTS][ANA_L][NB][6];
  const int b0 = blockIdx.x * NB, chunk = blockIdx.y, m = blockIdx.z;
  bool any = false;
  for (int k = 0; k < NB; ++k) any = any || state == nullptr || !state[b0 + k].done;
  if (!any) return;
  const int t = threadIdx.x;
  const int p = chunk * ANA_P + t;
  const bool act = p < npairs;
  const int pp = act ? p : npairs - 1;
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    float2 gn[3], gs[3];
    for (int f = 0; f < 3; ++f) {
      const float2 *g = rc + rc_index2(b0 + k, f, m, mmax, pp, npairs);
      gn[f] = act ? g[0] : make_float2(0.f, 0.f);
      gs[f] = (act && p != npairs - 1) ? g[1] : make_float2(0.f, 0.f);
    }
    for (int f = 0; f < 3; ++f) {
      float2 e = cadd(gn[f], gs[f]), o = csub(gn[f], gs[f]);
      G[t][k][f] = make_float4(e.x, e.y, o.x, o.y);
    }
  }
  const int64_t base = alm_base(lmax, m);
  const int64_t plane = nalm * (int64_t)npairs;
  const int lj = t % ANA_L, part = t / ANA_L;
  for (int lc = m; lc <= lmax; lc += ANA_L) {
    const int cnt = min(ANA_L, lmax + 1 - lc);
    __syncthreads();
    // phase A: tile of the tables, coalesced over pairs
    for (int j = 0; j < cnt; ++j) {
      const int64_t o = (base + lc + j) * (int64_t)npairs + pp;
      P0[t][j] = act ? ptab[o] : 0.f;
      Pp[t][j] = act ? ptab[plane + o] : 0.f;
      Pq[t][j] = act ? ptab[2 * plane + o] : 0.f;
    }
    __syncthreads();
    float acc[NB][6];
#pragma unroll
    for (int k = 0; k < NB; ++k)
#pragma unroll
      for (int i = 0; i < 6; ++i) acc[k][i] = 0.f;
    if (lj < cnt) {
      const int l = lc + lj;
      const bool odd = ((l - m) & 1) != 0;
      for (int q = part * ANA_L; q < (part + 1) * ANA_L; ++q) {
        const float lam = P0[q][lj], lp = Pp[q][lj], lq = Pq[q][lj];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          const float4 gt4 = G[q][k][0], gq4 = G[q][k][1], gu4 = G[q][k][2];
          const float2 gt = odd ? make_float2(gt4.z, gt4.w) : make_float2(gt4.x, gt4.y);
          const float2 gqp = odd ? make_float2(gq4.z, gq4.w) : make_float2(gq4.x, gq4.y);
          const float2 gup = odd ? make_float2(gu4.z, gu4.w) : make_float2(gu4.x, gu4.y);
          const float2 gqo = odd ? make_float2(gq4.x, gq4.y) : make_float2(gq4.z, gq4.w);
          const float2 guo = odd ? make_float2(gu4.x, gu4.y) : make_float2(gu4.z, gu4.w);
          acc[k][0] = fmaf(lam, gt.x, acc[k][0]);
          acc[k][1] = fmaf(lam, gt.y, acc[k][1]);
          acc[k][2] = fmaf(-lp, gqp.x, fmaf(lq, guo.y, acc[k][2]));
          acc[k][3] = fmaf(-lp, gqp.y, fmaf(-lq, guo.x, acc[k][3]));
          acc[k][4] = fmaf(-lp, gup.x, fmaf(-lq, gqo.y, acc[k][4]));
          acc[k][5] = fmaf(-lp, gup.y, fmaf(lq, gqo.x, acc[k][5]));
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
        float v[6];
        for (int i = 0; i < 6; ++i) {
          float a = red[0][lj][k][i];
          for (int q = 1; q < ANA_PARTS; ++q) a += red[q][lj][k][i];
          v[i] = a;
        }
        float2 *o = apart + ((int64_t)(b0 + k) * nchunk + chunk) * 3 * nalm + base + l;
        o[0] = make_float2(v[0], v[1]);
        o[nalm] = make_float2(v[2], v[3]);
        o[2 * nalm] = make_float2(v[4], v[5]);
      }
    }
  }
}

__global__ void k_ana_reduce32(const float2 *__restrict__ apart, double2 *out, int lmax, int64_t nalm, int nchunk,
                               double omega, int epilogue, const double *__restrict__ filt, int nlev,
                               const SolveState *__restrict__ state, const double2 *__restrict__ g_add) {
  const int b = blockIdx.y, m = blockIdx.z;
  if (state != nullptr && state[b].done) return;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const int64_t i = alm_base(lmax, m) + l;
  // chunk sum in FP32 (it carries the analysis of the FP32 correction only),
  // harmonic step and filter in FP64
  double2 acc[3];
  for (int f = 0; f < 3; ++f) {
    float ax = 0.f, ay = 0.f;
    for (int c = 0; c < nchunk; ++c) {
      const float2 v = apart[(((int64_t)b * nchunk + c) * 3 + f) * nalm + i];
      ax += v.x;
      ay += v.y;
    }
    acc[f] = make_double2(omega * (double)ax, omega * (double)ay);
  }
  double2 *o = out + (int64_t)b * 3 * nalm + i;
  if (epilogue == ANA_PLAIN) {
    o[0] = acc[0];
    o[nalm] = acc[1];
    o[2 * nalm] = acc[2];
    return;
  }
  if (g_add != nullptr) {  // anchor term A W (d - Y a_hi), FP64
    const double2 *g = g_add + (int64_t)b * 3 * nalm + i;
    acc[0] = cadd(acc[0], g[0]);
    acc[1] = cadd(acc[1], g[nalm]);
    acc[2] = cadd(acc[2], g[2 * nalm]);
  }
  const double *c = filt + (((int64_t)b * nlev + state[b].level) * (lmax + 1) + l) * 4;
  double2 t = cadd(o[0], acc[0]), e = cadd(o[nalm], acc[1]), bb = cadd(o[2 * nalm], acc[2]);
  o[0] = make_double2(c[0] * t.x + c[1] * e.x, c[0] * t.y + c[1] * e.y);
  o[nalm] = make_double2(c[1] * t.x + c[2] * e.x, c[1] * t.y + c[2] * e.y);
  o[2 * nalm] = make_double2(c[3] * bb.x, c[3] * bb.y);
}

cudaError_t legendre_synthesis32(dm_plan *p, const double2 *alm, cudaStream_t st) {
  if (p->use_tc && tc_batch_ok(p->batch)) return legendre_synthesis_tc(p, alm, st);
  if (cudaError_t e = ensure_ptab(p)) return e;
  const SolveState *stp = p->state_active ? p->state : nullptr;
  const int pb = (p->npairs + SYN_THREADS - 1) / SYN_THREADS;
  if (p->batch % 4 == 0) {
    dim3 g(p->batch / 4, pb, p->mmax + 1);
    k_leg_syn32<4><<<g, SYN_THREADS, 0, st>>>(p->ptab, alm, p->anchor_active ? p->a_hi : nullptr,
                                              p->anchor_active ? p->e32 : nullptr, p->rc32, p->lmax, p->mmax,
                                              p->npairs, p->nalm, stp);
  } else {
    dim3 g(p->batch, pb, p->mmax + 1);
    k_leg_syn32<1><<<g, SYN_THREADS, 0, st>>>(p->ptab, alm, p->anchor_active ? p->a_hi : nullptr,
                                              p->anchor_active ? p->e32 : nullptr, p->rc32, p->lmax, p->mmax,
                                              p->npairs, p->nalm, stp);
  }
  return cudaGetLastError();
}

// Filtered harmonic step of an anchored mixed iteration, on the FP32 state
// e = a - a_hi (a_hi the FP64 anchor, g_hi = A W (d - Y a_hi) its FP64 term):
//   a_new = F (a + Omega A r + g_hi)  <=>  e_new = c + F (e + Omega A r),
//   c = F (a_hi + g_hi) - a_hi.
// c depends on the level's filter F; it is formed in FP64 (and e_new with it)
// whenever the level differs from the one c was formed at (clev, advanced by
// the level control after this kernel), otherwise the step is all FP32.
__global__ void k_ana_step_e32(const float2 *__restrict__ apart, int nchunk, float omega, int lmax, int64_t nalm,
                               const double *__restrict__ filt, const float *__restrict__ filt32, int nlev,
                               const SolveState *__restrict__ state, const int *__restrict__ clev,
                               const double2 *__restrict__ a_hi, const double2 *__restrict__ g_hi,
                               float2 *__restrict__ e32, float2 *__restrict__ c32) {
  const int b = blockIdx.y, m = blockIdx.z;
  if (state[b].done) return;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const int64_t i = alm_base(lmax, m) + l, ib = (int64_t)b * 3 * nalm + i;
  float2 acc[3];
  for (int f = 0; f < 3; ++f) {
    float ax = 0.f, ay = 0.f;
    for (int c = 0; c < nchunk; ++c) {
      const float2 v = apart[(((int64_t)b * nchunk + c) * 3 + f) * nalm + i];
      ax += v.x;
      ay += v.y;
    }
    acc[f] = make_float2(omega * ax, omega * ay);
  }
  const int lev = state[b].level;
  const int64_t co = (((int64_t)b * nlev + lev) * (lmax + 1) + l) * 4;
  if (lev != clev[b]) {
    const double *cf = filt + co;
    double2 h[3], x[3], y[3];
    for (int f = 0; f < 3; ++f) {
      h[f] = a_hi[ib + f * nalm];
      const double2 g = g_hi[ib + f * nalm];
      const float2 e = e32[ib + f * nalm];
      x[f] = make_double2(h[f].x + g.x, h[f].y + g.y);
      y[f] = make_double2(x[f].x + (double)e.x + (double)acc[f].x, x[f].y + (double)e.y + (double)acc[f].y);
    }
    const double2 cT = make_double2(cf[0] * x[0].x + cf[1] * x[1].x - h[0].x, cf[0] * x[0].y + cf[1] * x[1].y - h[0].y);
    const double2 cE = make_double2(cf[1] * x[0].x + cf[2] * x[1].x - h[1].x, cf[1] * x[0].y + cf[2] * x[1].y - h[1].y);
    const double2 cB = make_double2(cf[3] * x[2].x - h[2].x, cf[3] * x[2].y - h[2].y);
    const double2 eT = make_double2(cf[0] * y[0].x + cf[1] * y[1].x - h[0].x, cf[0] * y[0].y + cf[1] * y[1].y - h[0].y);
    const double2 eE = make_double2(cf[1] * y[0].x + cf[2] * y[1].x - h[1].x, cf[1] * y[0].y + cf[2] * y[1].y - h[1].y);
    const double2 eB = make_double2(cf[3] * y[2].x - h[2].x, cf[3] * y[2].y - h[2].y);
    c32[ib] = make_float2((float)cT.x, (float)cT.y);
    c32[ib + nalm] = make_float2((float)cE.x, (float)cE.y);
    c32[ib + 2 * nalm] = make_float2((float)cB.x, (float)cB.y);
    e32[ib] = make_float2((float)eT.x, (float)eT.y);
    e32[ib + nalm] = make_float2((float)eE.x, (float)eE.y);
    e32[ib + 2 * nalm] = make_float2((float)eB.x, (float)eB.y);
    return;
  }
  const float4 cf = *reinterpret_cast<const float4 *>(filt32 + co);
  float2 y[3], c[3];
  for (int f = 0; f < 3; ++f) {
    const float2 e = e32[ib + f * nalm];
    c[f] = c32[ib + f * nalm];
    y[f] = make_float2(e.x + acc[f].x, e.y + acc[f].y);
  }
  e32[ib] = make_float2(c[0].x + cf.x * y[0].x + cf.y * y[1].x, c[0].y + cf.x * y[0].y + cf.y * y[1].y);
  e32[ib + nalm] = make_float2(c[1].x + cf.y * y[0].x + cf.z * y[1].x, c[1].y + cf.y * y[0].y + cf.z * y[1].y);
  e32[ib + 2 * nalm] = make_float2(c[2].x + cf.w * y[2].x, c[2].y + cf.w * y[2].y);
}

// At an anchor: c = F (a_hi + g_hi) - a_hi at each RHS's current level, e = 0.
__global__ void k_anchor_c32(const double *__restrict__ filt, int nlev, const SolveState *__restrict__ state,
                             int *__restrict__ clev, const double2 *__restrict__ a_hi,
                             const double2 *__restrict__ g_hi, float2 *__restrict__ e32, float2 *__restrict__ c32,
                             int lmax, int64_t nalm) {
  const int b = blockIdx.y, m = blockIdx.z;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  const int lev = state[b].level;
  if (blockIdx.x == 0 && m == 0 && threadIdx.x == 0) clev[b] = lev;
  if (l > lmax) return;
  const int64_t i = alm_base(lmax, m) + l, ib = (int64_t)b * 3 * nalm + i;
  const double *cf = filt + (((int64_t)b * nlev + lev) * (lmax + 1) + l) * 4;
  double2 h[3], x[3];
  for (int f = 0; f < 3; ++f) {
    h[f] = a_hi[ib + f * nalm];
    const double2 g = g_hi[ib + f * nalm];
    x[f] = make_double2(h[f].x + g.x, h[f].y + g.y);
    e32[ib + f * nalm] = make_float2(0.f, 0.f);
  }
  c32[ib] = make_float2((float)(cf[0] * x[0].x + cf[1] * x[1].x - h[0].x), (float)(cf[0] * x[0].y + cf[1] * x[1].y - h[0].y));
  c32[ib + nalm] = make_float2((float)(cf[1] * x[0].x + cf[2] * x[1].x - h[1].x),
                               (float)(cf[1] * x[0].y + cf[2] * x[1].y - h[1].y));
  c32[ib + 2 * nalm] = make_float2((float)(cf[3] * x[2].x - h[2].x), (float)(cf[3] * x[2].y - h[2].y));
}

// a = a_hi + e (FP64), before an anchor consumes the iterate
__global__ void k_materialize(const double2 *__restrict__ a_hi, const float2 *__restrict__ e32,
                              double2 *__restrict__ a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 h = a_hi[i];
    const float2 e = e32[i];
    a[i] = make_double2(h.x + (double)e.x, h.y + (double)e.y);
  }
}

cudaError_t anchor_c32(dm_plan *p, cudaStream_t st) {
  dim3 g((unsigned)((p->lmax + 1 + 127) / 128), p->batch, p->mmax + 1);
  k_anchor_c32<<<g, 128, 0, st>>>(p->filt, p->filt_levels, p->state, p->clev, p->a_hi, p->g_hi, p->e32, p->c32,
                                  p->lmax, p->nalm);
  return cudaGetLastError();
}

cudaError_t materialize_a(dm_plan *p, cudaStream_t st) {
  k_materialize<<<1024, 256, 0, st>>>(p->a_hi, p->e32, p->a, (int64_t)p->batch * 3 * p->nalm);
  return cudaGetLastError();
}

cudaError_t legendre_analysis32(dm_plan *p, int epilogue, double2 *out, cudaStream_t st, cudaEvent_t mid) {
  const SolveState *stp = p->state_active ? p->state : nullptr;
  int nchunk = p->nchunk;
  if (p->use_tc && tc_batch_ok(p->batch)) {
    cudaError_t e = legendre_analysis_tc(p, st);
    if (e) return e;
    nchunk = 1;
  } else if (p->nchunk32 < p->nchunk) {
    return cudaErrorInvalidValue;  // the CUDA-core FP32 analysis needs every chunk (see setup_fp32)
  } else if (cudaError_t e = ensure_ptab(p)) {
    return e;
  } else if (p->batch % 4 == 0) {
    dim3 g(p->batch / 4, p->nchunk, p->mmax + 1);
    k_leg_ana32<4><<<g, ANA_P, 0, st>>>(p->ptab, p->rc32, p->apart32, p->lmax, p->mmax, p->npairs, p->nalm,
                                        p->nchunk, stp);
  } else {
    dim3 g(p->batch, p->nchunk, p->mmax + 1);
    k_leg_ana32<1><<<g, ANA_P, 0, st>>>(p->ptab, p->rc32, p->apart32, p->lmax, p->mmax, p->npairs, p->nalm,
                                        p->nchunk, stp);
  }
  if (mid) cudaEventRecord(mid, st);
  double omega = 4.0 * M_PI / (double)p->npix;
  dim3 g2((unsigned)((p->lmax + 1 + 127) / 128), p->batch, p->mmax + 1);
  if (epilogue == ANA_DM_STEP && p->anchor_active) {  // FP32 state e between anchors
    k_ana_step_e32<<<g2, 128, 0, st>>>(p->apart32, nchunk, (float)omega, p->lmax, p->nalm, p->filt, p->filt32,
                                       p->filt_levels, p->state, p->clev, p->a_hi, p->g_hi, p->e32, p->c32);
    return cudaGetLastError();
  }
  k_ana_reduce32<<<g2, 128, 0, st>>>(p->apart32, out, p->lmax, p->nalm, nchunk, omega, epilogue, p->filt,
                                     p->filt_levels,
                                     epilogue == ANA_DM_STEP ? p->state : stp,
                                     (p->anchor_active && epilogue == ANA_DM_STEP) ? p->g_hi : nullptr);
  return cudaGetLastError();
}

}  // namespace dmwf
