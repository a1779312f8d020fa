// dm_prog.cu -- progressive working resolution (the speed-up the paper
// proposes in Section 4, with l_iter of Section 2): each cooling level of a
// Wiener-filter solve runs at the smallest HEALPix resolution whose band
// limit stays a margin above that level's l_iter, so the early levels cost a
// fraction of the full transforms.
//
//  - l_iter(mu): the largest l whose (TT, TE, EE) block or BB has an
//    eigenvalue above mu (the l beyond which S-bar = Theta(S - U) vanishes);
//  - level k, mu_k = (lambda_k - 1) T_h of the full resolution: band limit
//    L_k = min(lmax, max(l_min, ceil((1 + margin) l_iter(mu_k)))), nside_k the
//    smallest power of two with 2 nside_k >= L_k (at most nside); the last
//    level (mu = 0) always runs at full resolution;
//  - a coarse level sees, per Stokes component, the inverse-noise weighted
//    mean of the observed children of each coarse pixel (HEALPix nested
//    hierarchy) with noise variance 1 / sum N_c^-1, and its own alpha, w and
//    T_h; its filter uses mu_k: lambda' = 1 + mu_k / T_h,k in that plan;
//  - the harmonic iterate carries over between levels (l <= L_k kept, zero
//    above) and the next level continues the usual iteration from it,
//    a <- F_k [a + A(w (d - Y a))]; the first level starts as Algorithm 1
//    does (s_0 = 0, t_0 = d).
// Each resolution has its own plan (made on first use and kept), running the
// same kernels as any plan of that size and precision.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dm_internal.h"

namespace dmwf {

namespace {

// ---------------------------------------------------------------- geometry
// RING index of a NESTED pixel of a power-of-two nside (Gorski et al. 2005):
// base face f and in-face (x, y) from the even and odd bits, then the ring
// number counted from the north pole and the position along the ring.
int64_t nested_to_ring(int nside, int64_t pn) {
  static const int jrll[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
  static const int jpll[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};
  const int64_t npface = (int64_t)nside * nside, npix = 12 * npface, ncap = 2LL * nside * (nside - 1);
  const int f = (int)(pn / npface);
  const int64_t ipf = pn % npface;
  int64_t x = 0, y = 0;
  for (int b = 0; b < 31; ++b) {
    x |= ((ipf >> (2 * b)) & 1) << b;
    y |= ((ipf >> (2 * b + 1)) & 1) << b;
  }
  const int64_t jr = (int64_t)jrll[f] * nside - x - y - 1;
  int64_t nr, before, kshift = 0;
  if (jr < nside) {
    nr = jr;
    before = 2 * nr * (nr - 1);
  } else if (jr > 3 * (int64_t)nside) {
    nr = 4 * (int64_t)nside - jr;
    before = npix - 2 * nr * (nr + 1);
  } else {
    nr = nside;
    before = ncap + (jr - nside) * 4 * nside;
    kshift = (jr - nside) & 1;
  }
  int64_t jp = (jpll[f] * nr + x - y + 1 + kshift) / 2;
  if (jp > 4 * nr) jp -= 4 * nr;
  if (jp < 1) jp += 4 * nr;
  return before + jp - 1;
}

// children of every coarse pixel (RING order at nside_k) as fine RING
// indices at nside, 4^j per parent, parent-major
std::vector<int> children_table(int nside, int nk) {
  const int64_t npk = 12LL * nk * nk, per = (int64_t)(nside / nk) * (nside / nk);
  std::vector<int> out(npk * per);
  for (int64_t pn = 0; pn < npk; ++pn) {
    const int64_t pr = nested_to_ring(nk, pn);
    for (int64_t c = 0; c < per; ++c) out[pr * per + c] = (int)nested_to_ring(nside, pn * per + c);
  }
  return out;
}

int ell_iter(const std::vector<double> &cl, int lmax, double mu) {
  const int L = lmax + 1;
  int best = 0;
  for (int l = 0; l <= lmax; ++l) {
    const double tt = cl[l], ee = cl[L + l], bb = cl[2 * L + l], te = cl[3 * L + l];
    const double tr = tt + ee, det = tt * ee - te * te;
    const double emax = 0.5 * tr + sqrt(std::max(0.25 * tr * tr - det, 0.0));
    if (std::max(emax, bb) > mu) best = l;
  }
  return best;
}

// ------------------------------------------------------------------ kernels
// d_k[b][f][P] = sum over the children c of P of v[f][c] d[b][f][child(c)],
// v the normalised inverse-noise weights (0 on masked children)
__global__ void k_degrade(const double *__restrict__ d, const int *__restrict__ child,
                          const double *__restrict__ v, double *__restrict__ dk, int64_t npix, int64_t npk, int per,
                          int batch) {
  const int64_t total = (int64_t)batch * 3 * npk;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t P = i % npk, bf = i / npk, f = bf % 3;
    const double *db = d + bf * npix;
    const int *ch = child + P * per;
    const double *vv = v + f * npk * per + P * per;
    double acc = 0.0;
    for (int c = 0; c < per; ++c) acc += vv[c] * db[ch[c]];
    dk[i] = acc;
  }
}

__device__ __forceinline__ int64_t pg_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// harmonic iterate from band limit lf to lt: l <= min(lf, lt) kept, zero above
__global__ void k_change_band(const double2 *__restrict__ in, double2 *__restrict__ out, int lf, int lt,
                              int64_t nf, int64_t nt) {
  const int m = blockIdx.x, bf = blockIdx.y;
  for (int l = m + threadIdx.x; l <= lt; l += blockDim.x) {
    const double2 v = (l <= lf && m <= lf) ? in[bf * nf + pg_base(lf, m) + l] : make_double2(0.0, 0.0);
    out[bf * nt + pg_base(lt, m) + l] = v;
  }
}

}  // namespace

// The usual level loop from the iterate the plan holds in p->a (instead of
// a = 0, t_0 = d): the first step is a <- F [a + A(w (d - Y a))].
dm_status solve_begin_warm(dm_plan *p, const double *d, cudaStream_t st) {
  if (p->tc_err && cudaMemsetAsync(p->tc_err, 0, sizeof(int), st)) return DM_ECUDA;
  if (prepare_wd(p, d, st) || control_init(p, st)) return DM_ECUDA;
  p->launches += 2;
  if (p->prec == DM_FP64) {
    p->state_active = false;
    if (legendre_synthesis(p, p->a, st)) return DM_ECUDA;               // Y a
    if (ring_stage(p, RING_INV_MAP, nullptr, p->s64, st)) return DM_ECUDA;  // s_prev = Y a
    p->state_active = true;
    if (ring_stage(p, RING_ITER, nullptr, p->s64, st)) return DM_ECUDA;  // t - s = w (d - Y a)
    p->launches += 3;
  } else {
    p->anchor_active = false;  // a itself is the anchor: a_hi = a, e = 0
    dm_status r = anchor(p, st, false, d, true);
    if (r != DM_OK) return r;
    p->anchor_active = true;
  }
  p->state_active = true;
  p->session = true;
  p->iters_launched = 0;
  return DM_OK;
}

namespace {

struct ProgLevelPlan {
  int nside, L;
  dm_plan *q;             // nullptr: the main plan itself
  int *child = nullptr;   // device [npk][per]
  double *v = nullptr;    // device [3][npk][per]
  int per = 1;
};

// plan of one working resolution: spectra to L, the degraded noise, same
// precision and batch; the degrade tables
dm_status make_level_plan(dm_plan *p, int nk, int L, ProgLevelPlan &lp, std::string &err) {
  lp.nside = nk;
  lp.L = L;
  lp.q = nullptr;
  dm_status r = dm_plan_create(nk, L, p->batch, &lp.q);
  if (r != DM_OK) {
    err = "level plan";
    return r;
  }
  dm_plan *q = lp.q;
  std::vector<double> cl(4 * (size_t)(L + 1));
  for (int c = 0; c < 4; ++c)
    for (int l = 0; l <= L; ++l) cl[c * (L + 1) + l] = p->cl_h[c * (p->lmax + 1) + l];
  if ((r = dm_set_spectra(q, cl.data())) != DM_OK) {
    err = q->err;
    return r;
  }
  const int nside = p->nside;
  const int64_t npix = p->npix, npk = 12LL * nk * nk;
  lp.per = (nside / nk) * (nside / nk);
  const std::vector<int> ch = children_table(nside, nk);
  std::vector<double> v(3 * (size_t)npk * lp.per, 0.0), sk(3 * (size_t)npk, 1.0);
  std::vector<uint8_t> mk(npk, 0);
  for (int64_t P = 0; P < npk; ++P)
    for (int f = 0; f < 3; ++f) {
      double W = 0.0;
      for (int c = 0; c < lp.per; ++c) {
        const int i = ch[P * lp.per + c];
        if (p->mask_h[i]) W += 1.0 / (p->sigma_h[f * npix + i] * p->sigma_h[f * npix + i]);
      }
      if (W > 0.0) {
        for (int c = 0; c < lp.per; ++c) {
          const int i = ch[P * lp.per + c];
          const double s = p->sigma_h[f * npix + i];
          v[(f * npk + P) * lp.per + c] = p->mask_h[i] ? 1.0 / (s * s) / W : 0.0;
        }
        sk[f * npk + P] = 1.0 / sqrt(W);
        if (f == 0) mk[P] = 1;
      }
    }
  if ((r = dm_set_noise_mask(q, sk.data(), mk.data())) != DM_OK) {
    err = q->err;
    return r;
  }
  const dm_precision prec = p->ff_legendre ? DM_FLOAT_FLOAT : p->prec;
  if ((r = dm_set_precision(q, prec)) != DM_OK) {
    err = q->err;
    return r;
  }
  q->use_tc = p->use_tc;
  q->anchor_every = p->anchor_every;
  q->anchor_ff = p->anchor_ff;
  q->ring_lr = p->ring_lr;
  if (cudaMalloc(&lp.child, sizeof(int) * ch.size()) || cudaMalloc(&lp.v, sizeof(double) * v.size()) ||
      cudaMemcpy(lp.child, ch.data(), sizeof(int) * ch.size(), cudaMemcpyHostToDevice) ||
      cudaMemcpy(lp.v, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice)) {
    err = "degrade tables";
    return DM_ENOMEM;
  }
  q->bytes += (int64_t)(sizeof(int) * ch.size() + sizeof(double) * v.size());
  return DM_OK;
}

}  // namespace

// Drop the plans of the working resolutions (after the spectra, the noise or
// the arithmetic of the main plan changed).
void prog_release(dm_plan *p) {
  for (auto &lv : p->prog_levels) {
    ProgLevelPlan *lp = static_cast<ProgLevelPlan *>(lv);
    if (lp->child) cudaFree(lp->child);
    if (lp->v) cudaFree(lp->v);
    if (lp->q) dm_plan_destroy(lp->q);
    delete lp;
  }
  p->prog_levels.clear();
}

// The whole progressive solve of d (device [B][3][npix]); on return the main
// plan holds the final iterate (p->a, p->s64 = Y a) and per-level counts.
dm_status run_progressive(dm_plan *p, const double *d, cudaStream_t st) {
  const dm_schedule S = p->sched;
  const std::vector<int> forced = p->forced;
  const int nl = S.n_levels;
  const double th = p->t_h[0];
  p->prog_counts.assign((size_t)p->batch * nl, 0);
  p->prog_res.assign(2 * (size_t)nl, 0);
  long remaining = S.max_iter;
  const double2 *a_prev = nullptr;
  int L_prev = 0;
  dm_status r = DM_OK;
  std::string err;
  for (int k = 0; k < nl && r == DM_OK; ++k) {
    const double mu = (p->lambdas[k] - 1.0) * th;
    int nk = p->nside, L = p->lmax;
    if (k < nl - 1 && mu > 0.0) {
      L = std::min(p->lmax, std::max(p->prog_lmin, (int)ceil((1.0 + p->prog_margin) * ell_iter(p->cl_h, p->lmax, mu))));
      nk = 1;
      while (2 * nk < L && nk < p->nside) nk *= 2;
    }
    p->prog_res[2 * k] = nk;
    p->prog_res[2 * k + 1] = L;
    // the plan of this resolution
    dm_plan *q = p;
    ProgLevelPlan *lp = nullptr;
    if (nk != p->nside || L != p->lmax) {
      for (auto &lv : p->prog_levels) {
        ProgLevelPlan *c = static_cast<ProgLevelPlan *>(lv);
        if (c->nside == nk && c->L == L) lp = c;
      }
      if (!lp) {
        lp = new ProgLevelPlan();
        p->prog_levels.push_back(lp);
        r = make_level_plan(p, nk, L, *lp, err);
        if (r != DM_OK) break;
      }
      q = lp->q;
    }
    // one level: lambda' = 1 + mu / T_h of that resolution, this level's count or threshold
    dm_schedule s1 = S;
    s1.n_levels = 1;
    s1.max_iter = (int)std::max(1L, remaining);
    const bool fixed = !forced.empty() || S.iters_per_level > 0;
    const int count = !forced.empty() ? forced[k] : S.iters_per_level;
    s1.iters_per_level = fixed ? std::max(count, 0) : 0;
    double ek;
    if (S.eta > 0.0)
      ek = std::max(S.eps_final, S.eps0 * pow(S.eta, -(double)k));
    else
      ek = (nl == 1) ? S.eps_final : S.eps0 * pow(S.eps_final / S.eps0, (double)k / (double)(nl - 1));
    if (k == nl - 1) ek = S.eps_final;
    s1.eps0 = s1.eps_final = ek;
    q->sched = s1;
    q->forced.clear();
    q->lambda_single = 1.0 + mu / q->t_h[0];
    q->eps_final_rhs.assign(q->batch, ek);
    if (fixed && count <= 0) {  // an empty level: the iterate carries over unchanged
      q->lambda_single = 0.0;
      continue;
    }
    if ((r = upload_levels(q)) != DM_OK) break;
    for (int b = 0; b < q->batch && r == DM_OK; ++b)
      if (build_filters(q, b, st)) r = DM_ECUDA;
    if (r != DM_OK) break;
    // data at this resolution
    const double *dq = d;
    if (q != p) {
      const int64_t npk = q->npix;
      k_degrade<<<2048, 256, 0, st>>>(d, lp->child, lp->v, q->tmpmap2, p->npix, npk, lp->per, p->batch);
      if (cudaGetLastError()) {
        r = DM_ECUDA;
        break;
      }
      dq = q->tmpmap2;
    }
    if (a_prev == nullptr) {
      r = solve_begin(q, dq, st);
    } else {
      k_change_band<<<dim3(L + 1, 3 * p->batch), 128, 0, st>>>(a_prev, q->a, L_prev, L,
                                                              (int64_t)(L_prev + 1) * (L_prev + 2) / 2, q->nalm);
      r = cudaGetLastError() ? DM_ECUDA : solve_begin_warm(q, dq, st);
    }
    int all = 0;
    if (r == DM_OK) r = solve_iterate(q, s1.max_iter + 4, &all, st);
    if (r == DM_OK) r = solve_end(q, nullptr, nullptr, st, false);
    if (r != DM_OK) {
      q->session = q->state_active = q->anchor_active = false;
      break;
    }
    std::vector<SolveState> hs(p->batch);
    if (cudaMemcpyAsync(hs.data(), q->state, sizeof(SolveState) * p->batch, cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st)) {
      r = DM_ECUDA;
      break;
    }
    long most = 0;
    for (int b = 0; b < p->batch; ++b) {
      p->prog_counts[(size_t)b * nl + k] = hs[b].iters_total;
      most = std::max<long>(most, hs[b].iters_total);
      if (hs[b].notconv) p->prog_notconv = true;
    }
    remaining -= most;
    a_prev = q->a;
    L_prev = L;
  }
  // the main plan gets its own schedule back
  p->sched = S;
  p->forced = forced;
  p->lambda_single = 0.0;
  p->eps_final_rhs.assign(p->batch, S.eps_final);
  dm_status r2 = upload_levels(p);
  if (r == DM_OK && r2 != DM_OK) r = r2;
  for (int b = 0; b < p->batch && r == DM_OK; ++b)
    if (build_filters(p, b, st)) r = DM_ECUDA;
  if (r == DM_OK && cudaStreamSynchronize(st)) r = DM_ECUDA;
  if (r != DM_OK && !err.empty()) p->err = "progressive solve: " + err;
  return r;
}

}  // namespace dmwf
