// dm_api.cu -- the extern "C" entry points of include/dmwf.h: plan lifecycle,
// argument validation, and the host driver of Algorithm 1 that enqueues the
// device stages and polls the device-side convergence state.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "dm_internal.h"

using namespace dmwf;

namespace {

dm_status fail(dm_plan *p, dm_status s, const std::string &msg) {
  if (p) p->err = msg;
  return s;
}

dm_status cuda_fail(dm_plan *p, cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (p) p->err = m;
  return e == cudaErrorMemoryAllocation ? DM_ENOMEM : DM_ECUDA;
}

#define DM_CU(call, where)                          \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(p, e_, where); \
  } while (0)

template <typename T>
cudaError_t dalloc(dm_plan *p, T **ptr, size_t count) {
  size_t bytes = sizeof(T) * (count > 0 ? count : 1);
  cudaError_t e = cudaMalloc((void **)ptr, bytes);
  if (e == cudaSuccess) p->bytes += (int64_t)bytes;
  return e;
}

void free_all(dm_plan *p) {
  prog_release(p);
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  p->ev.clear();
  void *ptrs[] = {p->rings, p->pairs, p->phase, p->bhat, p->twid, p->rec, p->seed, p->seed_exp, p->cl,
                  p->filt, p->w, p->mask, p->sigma, p->rc, p->a, p->apart, p->wd, p->norms, p->state,
                  p->lev, p->tmpmap, p->tmpmap2, p->tmpalm, p->seeds_dev, p->coef_tmp,
                  p->ptab, p->rc32, p->apart32, p->s32, p->w32, p->wd32, p->phase32, p->bhat32, p->twid32,
                  p->a_hi, p->g_hi, p->shi32, p->s64, p->rhi, p->tc_err, p->ring_order, p->pair_order,
                  p->tc_synA[0], p->tc_synA[1], p->tc_anaA[0], p->tc_anaA[1], p->tc_soff, p->tc_aoff,
                  p->tc_synB[0], p->tc_synB[1], p->ptab_lo, p->e32, p->c32, p->clev, p->filt32,
                  p->twr, p->twr32, p->chirp, p->chirp32, p->wcov, p->diag_tab, p->diag_alm, p->diag_part,
                  p->diag_ao, p->covdraw, p->jsrc, p->jacc, p->bhatT[0], p->bhatT[1], p->bhatT32[0],
                  p->bhatT32[1], p->ck0, p->ck2, p->cko, p->rq0, p->rq2, p->rq2d, p->ffs, p->ffs_lo};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  if (p->ev_begin) cudaEventDestroy(p->ev_begin);
  if (p->ev_end) cudaEventDestroy(p->ev_end);
}

void default_schedule(dm_schedule *s) {
  s->lambda0 = 1000.0;
  s->n_levels = 10;
  s->iters_per_level = 10;
  s->eps0 = 1e-4;
  s->eps_final = 1e-6;
  s->eta = 0.0;
  s->max_iter = 100000;
  s->check_every = 8;
}

}  // namespace

namespace dmwf {
// Host copy of the level tables (one per RHS); the device copies drive
// k_control_step.
dm_status upload_levels(dm_plan *p) {
  const dm_schedule &s = p->sched;
  p->lambdas.assign(s.n_levels, 1.0);
  for (int k = 0; k < s.n_levels; ++k)
    p->lambdas[k] = (s.n_levels == 1) ? 1.0 : pow(s.lambda0, 1.0 - (double)k / (double)(s.n_levels - 1));
  p->lambdas[s.n_levels - 1] = 1.0;
  if (s.n_levels == 1 && p->lambda_single > 0.0) p->lambdas[0] = p->lambda_single;
  if ((int)p->eps_final_rhs.size() != p->batch) p->eps_final_rhs.assign(p->batch, s.eps_final);
  std::vector<LevelDev> Ls(p->batch);
  for (int b = 0; b < p->batch; ++b) {
    LevelDev &L = Ls[b];
    L = LevelDev{};
    L.n_levels = s.n_levels;
    L.max_iter = s.max_iter;
    const double ef = p->eps_final_rhs[b];
    for (int k = 0; k < s.n_levels; ++k) {
      double e;
      if (s.eta > 0.0)
        e = std::max(ef, s.eps0 * pow(s.eta, -(double)k));
      else
        e = (s.n_levels == 1) ? ef : s.eps0 * pow(ef / s.eps0, (double)k / (double)(s.n_levels - 1));
      L.eps[k] = e;
    }
    L.eps[s.n_levels - 1] = ef;
    if (!p->forced.empty()) {
      L.forced = 1;
      for (int k = 0; k < s.n_levels; ++k) L.fixed_iters[k] = p->forced[k];
    } else if (s.iters_per_level > 0) {
      L.forced = 1;
      for (int k = 0; k < s.n_levels; ++k) L.fixed_iters[k] = s.iters_per_level;
    }
  }
  DM_CU(cudaMemcpy(p->lev, Ls.data(), sizeof(LevelDev) * p->batch, cudaMemcpyHostToDevice), "upload levels");
  return DM_OK;
}

// The schedule's levels with a forced count per RHS and level (counts[B][n_levels]).
dm_status upload_levels_counts(dm_plan *p, const std::vector<int> &counts) {
  dm_status r = upload_levels(p);
  if (r != DM_OK) return r;
  const int nl = p->sched.n_levels;
  std::vector<LevelDev> Ls(p->batch);
  DM_CU(cudaMemcpy(Ls.data(), p->lev, sizeof(LevelDev) * p->batch, cudaMemcpyDeviceToHost), "levels");
  for (int b = 0; b < p->batch; ++b) {
    Ls[b].forced = 1;
    for (int k = 0; k < nl; ++k) Ls[b].fixed_iters[k] = counts[(size_t)b * nl + k];
  }
  DM_CU(cudaMemcpy(p->lev, Ls.data(), sizeof(LevelDev) * p->batch, cudaMemcpyHostToDevice), "upload levels");
  return DM_OK;
}

}  // namespace dmwf

namespace {

dm_status refresh_filters(dm_plan *p) {
  if (!p->have_cl || !p->have_noise) return DM_OK;
  for (int b = 0; b < p->batch; ++b) DM_CU(build_filters(p, b, 0), "build filters");
  DM_CU(cudaDeviceSynchronize(), "build filters");
  return DM_OK;
}

// A failed solve leaves the plan usable: no session, no stage state.
void end_session(dm_plan *p) {
  p->state_active = false;
  p->anchor_active = false;
  p->session = false;
}

dm_status check_ready(dm_plan *p) {
  if (!p) return DM_EINVAL;
  if (!p->have_cl) return fail(p, DM_EINVAL, "spectra not set (dm_set_spectra)");
  if (!p->have_noise) return fail(p, DM_EINVAL, "noise not set (dm_set_noise_mask)");
  return DM_OK;
}

}  // namespace

namespace dmwf {

// The iteration driver.  Device stages per iteration:
//   analysis + harmonic step  a <- F_k [a + A (t - s)]      (k_leg_ana + k_ana_reduce)
//   synthesis                 F_m(theta) from a             (k_leg_syn)
//   ring stage                s, Cauchy partials, t - s, G_m (k_ring<RING_ITER>)
//   control                   Cauchy ratio, level, stop     (k_control_step)
// Mixed precision adds FP64 anchors (iterative refinement): a = a_hi + e, the
// FP32 stages transform e only, and g_hi = A W (d - Y a_hi) is recomputed in
// FP64 every anchor_every iterations, so the fixed point is the FP64 one.
cudaError_t enqueue_iteration(dm_plan *p, cudaStream_t st, cudaEvent_t *E) {
  cudaError_t e;
  if (E) cudaEventRecord(E[0], st);
  if ((e = legendre_analysis(p, ANA_DM_STEP, p->a, st, E ? E[1] : nullptr))) return e;
  if (E) cudaEventRecord(E[2], st);
  if ((e = legendre_synthesis(p, p->a, st))) return e;
  if (E) cudaEventRecord(E[3], st);
  if ((e = p->cov ? (p->prec == DM_FP64 ? cov_ring_stage(p, st) : cov_ring_stage32(p, st))
                  : ring_stage(p, RING_ITER, nullptr, p->s64, st)))
    return e;
  if (E) cudaEventRecord(E[4], st);
  if ((e = control_step(p, st))) return e;
  if (E) cudaEventRecord(E[5], st);
  p->launches += 5;
  return cudaSuccess;
}

// FP64 anchor at the current iterate (all RHS): a_hi = a, s64 = Y a_hi,
// rhi = w (d - s64), g_hi = A rhi; the FP32 correction restarts from e = 0.
// initial: a_hi = 0 and rhi = d on observed pixels (Algorithm 1's t_0 = d).
dm_status anchor(dm_plan *p, cudaStream_t st, bool initial, const double *d, bool need_g) {
  const bool sa = p->state_active;
  const size_t an = sizeof(double2) * 3 * p->nalm * p->batch;
  const size_t mn = sizeof(double) * 3 * p->npix * p->batch;
  p->state_active = false;
  p->prec = DM_FP64;
  p->ff_now = p->anchor_ff;
  cudaError_t e = cudaSuccess;
  cudaEvent_t ta = nullptr, tb = nullptr;
  if (p->prof_on) {
    cudaEventCreate(&ta);
    cudaEventCreate(&tb);
    cudaEventRecord(ta, st);
  }
  if (initial) {
    if (!e) e = cudaMemsetAsync(p->a_hi, 0, an, st);
    if (!e) e = cudaMemsetAsync(p->s64, 0, mn, st);
    if (!e) e = anchor_residual(p, d, nullptr, st);
    p->launches += 1;
  } else {
    if (!e && p->anchor_active) e = materialize_a(p, st);  // the iterate lives in e between anchors
    if (!e) e = cudaMemcpyAsync(p->a_hi, p->a, an, cudaMemcpyDeviceToDevice, st);
    if (!e) e = legendre_synthesis(p, p->a_hi, st);
    if (!e) e = ring_stage(p, RING_INV_MAP, nullptr, p->s64, st);
    if (!e) e = p->cov ? anchor_residual_wd_cov(p, p->s64, st) : anchor_residual_wd(p, p->s64, st);
    p->launches += 3;
  }
  if (need_g) {
    if (!e) e = ring_stage(p, RING_FWD_MAP, p->rhi, nullptr, st);
    if (!e) e = legendre_analysis(p, ANA_PLAIN, p->g_hi, st);
    if (!e && p->src_active)  // harmonic source of a W~ run: g_hi = g + A W (d - Y a_hi)
      e = axpy_maps(6 * p->nalm * p->batch, (const double *)p->jsrc, 1.0, (double *)p->g_hi, st);
    if (!e) e = anchor_c32(p, st);
    p->launches += 4;
  }
  p->prec = DM_MIXED_FP32;
  p->ff_now = false;
  if (!e) e = cudaMemsetAsync(p->s32, 0, sizeof(float) * 3 * p->npix * p->batch, st);
  if (!e)
    e = cudaMemsetAsync(p->rc32, 0, sizeof(float2) * (size_t)p->batch * 3 * (p->mmax + 1) * p->npairs * 2, st);
  p->state_active = sa;
  p->since_anchor = 0;
  if (p->prof_on) {
    cudaEventRecord(tb, st);
    cudaEventSynchronize(tb);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ta, tb);
    p->prof.ms_anchor += ms;
    p->prof.anchors += 1;
    cudaEventDestroy(ta);
    cudaEventDestroy(tb);
  }
  if (e) return cuda_fail(p, e, "anchor");
  return DM_OK;
}

dm_status solve_begin(dm_plan *p, const double *d, cudaStream_t st) {
  // a tensor-core wait that gave up in an earlier solve does not count against this one
  if (p->tc_err) DM_CU(cudaMemsetAsync(p->tc_err, 0, sizeof(int), st), "clear wait flag");
  DM_CU(cudaMemsetAsync(p->a, 0, sizeof(double2) * 3 * p->nalm * p->batch, st), "zero a");
  DM_CU(p->cov ? cov_prepare_wd(p, d, st) : prepare_wd(p, d, st), "w d");
  DM_CU(control_init(p, st), "control init");
  p->launches += 2;
  if (p->prec == DM_FP64) {
    DM_CU(cudaMemsetAsync(p->s64, 0, sizeof(double) * 3 * p->npix * p->batch, st), "zero s");
    p->state_active = true;
    DM_CU(ring_stage(p, RING_INIT, d, nullptr, st), "ring init");
    p->launches += 1;
  } else {
    p->anchor_active = true;
    dm_status r = anchor(p, st, true, d, true);
    if (r != DM_OK) return r;
  }
  p->state_active = true;
  p->session = true;
  p->iters_launched = 0;
  return DM_OK;
}

// Up to max_iters iterations; *all_done = 1 once every RHS has stopped.
dm_status solve_iterate(dm_plan *p, long max_iters, int *all_done, cudaStream_t st) {
  if (!p->session) return fail(p, DM_EINVAL, "no solve in progress (dm_solve_begin)");
  const int every = std::max(1, p->sched.check_every);
  if (p->prof_on && (int)p->ev.size() < 6 * every) {
    int have = (int)p->ev.size();
    p->ev.resize(6 * every);
    for (int i = have; i < 6 * every; ++i) cudaEventCreate(&p->ev[i]);
  }
  std::vector<SolveState> hs(p->batch);
  const bool mixed = p->prec != DM_FP64;
  long done_iters = 0;
  *all_done = 0;
  while (done_iters < max_iters) {
    long window = std::min<long>(every, max_iters - done_iters);
    if (mixed && p->iters_launched == 0) window = 1;  // re-anchor after the t_0 = d step
    for (long k = 0; k < window; ++k) {
      cudaError_t e = enqueue_iteration(p, st, p->prof_on ? &p->ev[6 * k] : nullptr);
      if (e) return cuda_fail(p, e, "iteration");
    }
    done_iters += window;
    p->iters_launched += window;
    p->since_anchor += (int)window;
    cudaError_t e = cudaMemcpyAsync(hs.data(), p->state, sizeof(SolveState) * p->batch, cudaMemcpyDeviceToHost, st);
    int tcerr = 0;
    if (!e && p->tc_err) e = cudaMemcpyAsync(&tcerr, p->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return cuda_fail(p, e, "poll state");
    if (tcerr) return fail(p, DM_ETIMEOUT, "a tensor-core pipeline wait gave up");
    if (p->prof_on) {
      for (long k = 0; k < window; ++k) {
        float t[5];
        for (int j = 0; j < 5; ++j) cudaEventElapsedTime(&t[j], p->ev[6 * k + j], p->ev[6 * k + j + 1]);
        p->prof.ms_analysis += t[0];
        p->prof.ms_reduce += t[1];
        p->prof.ms_synthesis += t[2];
        p->prof.ms_ring += t[3];
        p->prof.ms_control += t[4];
        p->prof.iterations += 1;
      }
    }
    bool all = true;
    for (auto &s : hs) all = all && s.done;
    if (all) {
      *all_done = 1;
      break;
    }
    if (mixed && (p->iters_launched == 1 || p->since_anchor >= p->anchor_every)) {
      dm_status r = anchor(p, st, false, nullptr, true);
      if (r != DM_OK) return r;
    }
  }
  return DM_OK;
}

// Final iterate into s_out (mixed: one last FP64 synthesis of a).  After a
// progressive solve (which ended its sessions itself) only the copies remain.
dm_status solve_end(dm_plan *p, double *s_out, double *alm_out, cudaStream_t st, bool to_host) {
  if (!p->session && p->prog_margin > 0.0 && !p->prog_res.empty()) {
    const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (s_out) DM_CU(cudaMemcpyAsync(s_out, p->s64, sizeof(double) * 3 * p->npix * p->batch, kind, st), "copy s");
    if (alm_out)
      DM_CU(cudaMemcpyAsync(alm_out, p->a, sizeof(double2) * 3 * p->nalm * p->batch, kind, st), "copy alm");
    return DM_OK;
  }
  if (!p->session) return fail(p, DM_EINVAL, "no solve in progress (dm_solve_begin)");
  if (p->prec != DM_FP64) {
    dm_status r = anchor(p, st, false, nullptr, false);
    if (r != DM_OK) {
      end_session(p);
      return r;
    }
  }
  end_session(p);
  const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (s_out) DM_CU(cudaMemcpyAsync(s_out, p->s64, sizeof(double) * 3 * p->npix * p->batch, kind, st), "copy s");
  if (alm_out) DM_CU(cudaMemcpyAsync(alm_out, p->a, sizeof(double2) * 3 * p->nalm * p->batch, kind, st), "copy alm");
  return DM_OK;
}

dm_status run_dm(dm_plan *p, const double *d, cudaStream_t st) {
  if (p->prog_margin > 0.0) {
    if (!p->noise_shared || p->cov || p->flat || (p->nside & (p->nside - 1)) != 0)
      return fail(p, DM_EINVAL,
                  "progressive resolution needs a sphere plan of power-of-two nside with plan-wide diagonal noise");
    p->prog_notconv = false;
    dm_status r = run_progressive(p, d, st);
    if (r != DM_OK) return r;
    return p->prog_notconv ? fail(p, DM_ENOTCONV, "iteration cap reached") : DM_OK;
  }
  dm_status r = solve_begin(p, d, st);
  if (r != DM_OK) {
    end_session(p);
    return r;
  }
  const dm_schedule &S = p->sched;
  long cap = (long)S.max_iter + 4;
  if (S.iters_per_level > 0 || !p->forced.empty()) {
    long tot = 0;
    for (int k = 0; k < S.n_levels; ++k) tot += p->forced.empty() ? S.iters_per_level : p->forced[k];
    cap = tot + 4;
  }
  int all = 0;
  r = solve_iterate(p, cap, &all, st);
  if (r != DM_OK) {
    end_session(p);
    return r;
  }
  if (!all) return fail(p, DM_ENOTCONV, "iteration cap reached");
  return DM_OK;
}

}  // namespace dmwf

namespace {

// Stats of every RHS after a solve (the stream is synchronised): counts,
// Cauchy value, the FP64 diagnostics when enabled and ms_total from the
// solve's begin and end events.
void fill_stats(dm_plan *p, dm_stats *stats, dm_status *rs, cudaStream_t st) {
  std::vector<SolveState> hs(p->batch);
  cudaMemcpy(hs.data(), p->state, sizeof(SolveState) * p->batch, cudaMemcpyDeviceToHost);
  std::vector<double> resid(p->batch, NAN), chi2(p->batch, NAN);
  float ms = NAN;
  if (stats) {
    if (cudaEventSynchronize(p->ev_end) == cudaSuccess) cudaEventElapsedTime(&ms, p->ev_begin, p->ev_end);
    if (p->diag_on) {
      cudaError_t e = diagnostics(p, st, resid, chi2);
      if (e != cudaSuccess && *rs == DM_OK) *rs = cuda_fail(p, e, "diagnostics");
    }
  }
  bool notconv = false;
  for (int b = 0; b < p->batch; ++b) {
    notconv = notconv || hs[b].notconv;
    if (!stats) continue;
    dm_stats &o = stats[b];
    memset(&o, 0, sizeof(o));
    o.iters_total = hs[b].iters_total;
    o.levels_done = hs[b].done ? p->sched.n_levels : hs[b].level;
    for (int k = 0; k < DM_MAX_LEVELS; ++k) o.iters_per_level[k] = hs[b].iters_per_level[k];
    o.cauchy_final = hs[b].cauchy;
    o.true_resid = resid[b];
    o.chi2 = chi2[b];
    o.ms_total = ms;
    if (p->prog_margin > 0.0 && !p->prog_res.empty()) {  // a progressive solve: counts of every level's plan
      const int nl = (int)p->prog_res.size() / 2;
      o.iters_total = 0;
      for (int k = 0; k < nl && k < DM_MAX_LEVELS; ++k) {
        o.iters_per_level[k] = p->prog_counts[(size_t)b * nl + k];
        o.iters_total += o.iters_per_level[k];
      }
      o.levels_done = nl;
    }
  }
  if (notconv && *rs == DM_OK) *rs = fail(p, DM_ENOTCONV, "max_iter reached before the last level converged");
}

}  // namespace

namespace dmwf {

// The workspace of a plan whose geometry tables are built (sizes from
// npix, nalm, nrings, npairs, mmax and batch): allocates, initialises the
// schedule and hands the plan out; frees it on failure.
dm_status plan_workspace(dm_plan *p, dm_plan **out) {
  for (int i = 0; i < DM_TUNE_MAX_CLASSES; ++i) p->tune_ring_lr[i] = p->tune_ring_fuse[i] = -1;
  default_schedule(&p->sched);
  cudaError_t e = cudaSuccess;
  auto bad = [&](cudaError_t err, const char *w) {
    dm_status s = cuda_fail(p, err, w);
    fprintf(stderr, "dm_plan_create: %s\n", p->err.c_str());
    free_all(p);
    delete p;
    return s;
  };
  const int64_t B = p->batch, n3 = 3 * p->npix;
  const int L = p->flat ? (int)p->nmodes : p->lmax + 1;  // spectra entries per field
  if ((e = dalloc(p, &p->cl, 4 * (size_t)L))) return bad(e, "alloc");
  if ((e = dalloc(p, &p->w, (size_t)B * n3))) return bad(e, "alloc");
  if ((e = dalloc(p, &p->mask, (size_t)B * p->npix))) return bad(e, "alloc");
  if ((e = dalloc(p, &p->sigma, (size_t)B * n3))) return bad(e, "alloc");
  p->alpha.assign(B, 0.0);
  p->t_h.assign(B, 0.0);
  if ((e = dalloc(p, &p->rc, (size_t)B * 3 * (p->mmax + 1) * p->npairs * 2))) return bad(e, "alloc rc");
  if ((e = dalloc(p, &p->a, (size_t)B * 3 * p->nalm))) return bad(e, "alloc a");
  // FP64 analysis partials: every pair chunk at once while that takes at most
  // 24 GiB, else a few slots and the chunks in waves (legendre_analysis)
  {
    const double per_slot = (double)B * 3 * p->nalm * sizeof(double2);
    const int fit = (int)std::max(2.0, std::floor(24.0 * (1u << 30) / per_slot));
    p->nslot = std::min(p->nchunk, fit);
  }
  if (!p->flat && (e = dalloc(p, &p->apart, (size_t)B * p->nslot * 3 * p->nalm))) return bad(e, "alloc apart");
  if ((e = dalloc(p, &p->wd, (size_t)B * n3))) return bad(e, "alloc wd");
  if ((e = dalloc(p, &p->norms, (size_t)B * 3 * p->nrings * 2))) return bad(e, "alloc norms");
  if ((e = dalloc(p, &p->state, (size_t)B))) return bad(e, "alloc state");
  if ((e = dalloc(p, &p->lev, (size_t)B))) return bad(e, "alloc lev");
  if ((e = dalloc(p, &p->tmpmap, (size_t)B * n3))) return bad(e, "alloc tmp");
  if ((e = dalloc(p, &p->tmpmap2, (size_t)B * n3))) return bad(e, "alloc tmp");
  if ((e = dalloc(p, &p->tmpalm, (size_t)B * 3 * p->nalm))) return bad(e, "alloc tmp");
  if ((e = dalloc(p, &p->seeds_dev, (size_t)B))) return bad(e, "alloc seeds");
  if ((e = dalloc(p, &p->coef_tmp, 4 * (size_t)L))) return bad(e, "alloc coef");
  if ((e = dalloc(p, &p->s64, (size_t)B * n3))) return bad(e, "alloc s");
  if ((e = dalloc(p, &p->rhi, (size_t)B * n3))) return bad(e, "alloc rhi");
  if ((e = cudaEventCreate(&p->ev_begin)) || (e = cudaEventCreate(&p->ev_end))) return bad(e, "events");
  cudaMemset(p->rc, 0, sizeof(double2) * (size_t)B * 3 * (p->mmax + 1) * p->npairs * 2);
  cudaMemset(p->mask, 1, (size_t)B * p->npix);
  dm_status s = upload_levels(p);
  if (s != DM_OK) {
    free_all(p);
    delete p;
    return s;
  }
  if ((e = cudaDeviceSynchronize())) return bad(e, "create");
  *out = p;
  return DM_OK;
}

}  // namespace dmwf

extern "C" {

dm_status dm_plan_create(int nside, int lmax, int batch, dm_plan **out) {
  if (!out) return DM_EINVAL;
  *out = nullptr;
  if (nside < 1 || nside > 2048 || lmax < 2 || lmax > 4 * nside || batch < 1 || batch > 4096) return DM_EINVAL;
  // above nside 1024, keep the pixel-components of a plan within 31 bits
  if (nside > 1024 && (int64_t)batch * 3 * 12 * nside * nside > INT32_MAX) return DM_EINVAL;
  dm_plan *p = new dm_plan();
  cudaGetDevice(&p->device);
  p->nside = nside;
  p->lmax = lmax;
  p->mmax = lmax;
  p->batch = batch;
  p->npix = 12LL * nside * nside;
  p->nalm = (int64_t)(lmax + 1) * (lmax + 2) / 2;
  p->nrings = 4 * nside - 1;
  p->npairs = 2 * nside;
  p->nchunk = (p->npairs + 63) / 64;
  cudaError_t e = build_tables(p);
  if (e) {
    dm_status s = cuda_fail(p, e, "build tables");
    fprintf(stderr, "dm_plan_create: %s\n", p->err.c_str());
    free_all(p);
    delete p;
    return s;
  }
  return plan_workspace(p, out);
}

void dm_plan_destroy(dm_plan *p) {
  if (!p) return;
  cudaDeviceSynchronize();
  free_all(p);
  delete p;
}

const char *dm_last_error(const dm_plan *p) { return p ? p->err.c_str() : "null plan"; }

dm_status dm_plan_info(const dm_plan *p, int64_t *npix, int64_t *nalm, int *nrings, int64_t *ws) {
  if (!p) return DM_EINVAL;
  if (npix) *npix = p->npix;
  if (nalm) *nalm = p->nalm;
  if (nrings) *nrings = p->nrings;
  if (ws) *ws = p->bytes;
  return DM_OK;
}

dm_status dm_set_precision(dm_plan *p, dm_precision prec) {
  if (!p) return DM_EINVAL;
  if (prec != DM_FP64 && prec != DM_MIXED_FP32 && prec != DM_FLOAT_FLOAT)
    return fail(p, DM_EINVAL, "unknown precision mode");
  if (p->flat && prec != DM_FP64) return fail(p, DM_EINVAL, "flat-sky plans run in DM_FP64");
  if (p->session) return fail(p, DM_EBUSY, "a solve is in progress");
  prog_release(p);
  if (prec != DM_FP64) DM_CU(setup_fp32(p), "float tables");
  // DM_FLOAT_FLOAT runs the FP64 path with float-float Legendre stages
  p->prec = prec == DM_MIXED_FP32 ? DM_MIXED_FP32 : DM_FP64;
  p->ff_legendre = prec == DM_FLOAT_FLOAT;
  return DM_OK;
}

dm_status dm_set_anchor_precision(dm_plan *p, dm_precision prec) {
  if (!p) return DM_EINVAL;
  if (prec != DM_FP64 && prec != DM_FLOAT_FLOAT) return fail(p, DM_EINVAL, "anchors run in DM_FP64 or DM_FLOAT_FLOAT");
  p->anchor_ff = prec == DM_FLOAT_FLOAT;
  return DM_OK;
}

dm_status dm_set_spectra(dm_plan *p, const double *cl) {
  if (p && p->flat) return fail(p, DM_EINVAL, "flat-sky plans take dm_set_spectra_flat");
  if (!p || !cl) return DM_EINVAL;
  if (p->session) return fail(p, DM_EBUSY, "a solve is in progress on this plan");
  const int L = p->lmax + 1;
  for (int l = 0; l < L; ++l) {
    double tt = cl[l], ee = cl[L + l], bb = cl[2 * L + l], te = cl[3 * L + l];
    if (!std::isfinite(tt) || !std::isfinite(ee) || !std::isfinite(bb) || !std::isfinite(te))
      return fail(p, DM_EINVAL, "non-finite spectrum");
    if (tt < 0 || ee < 0 || bb < 0 || te * te > tt * ee * (1.0 + 1e-12))
      return fail(p, DM_EINVAL, "spectrum block not positive semi-definite at l = " + std::to_string(l));
  }
  p->cl_h.assign(cl, cl + 4 * L);
  prog_release(p);
  DM_CU(cudaMemcpy(p->cl, cl, sizeof(double) * 4 * L, cudaMemcpyHostToDevice), "upload cl");
  DM_CU(diag_tables(p), "diagnostic tables");
  p->have_cl = true;
  return refresh_filters(p);
}

namespace {
dm_status check_noise(dm_plan *p, const double *sigma, const uint8_t *mask) {
  const int64_t np = p->npix;
  int64_t nobs = 0;
  for (int64_t i = 0; i < np; ++i) {
    bool obs = !mask || mask[i];
    if (!obs) continue;
    ++nobs;
    for (int f = 0; f < 3; ++f) {
      double s = sigma[f * np + i];
      if (!(s > 0.0) || !std::isfinite(s))
        return fail(p, DM_EINVAL, "sigma must be finite and > 0 on observed pixels");
    }
  }
  if (nobs == 0) return fail(p, DM_EINVAL, "mask leaves no observed pixel");
  return DM_OK;
}

dm_status upload_noise(dm_plan *p, int b, const double *sigma, const uint8_t *mask) {
  const int64_t np = p->npix;
  DM_CU(cudaMemcpy(p->sigma + (size_t)b * 3 * np, sigma, sizeof(double) * 3 * np, cudaMemcpyHostToDevice), "sigma");
  if (mask)
    DM_CU(cudaMemcpy(p->mask + (size_t)b * np, mask, np, cudaMemcpyHostToDevice), "mask");
  else
    DM_CU(cudaMemset(p->mask + (size_t)b * np, 1, np), "mask");
  DM_CU(build_noise(p, b, 0), "noise");
  return DM_OK;
}
}  // namespace

dm_status dm_set_noise_mask(dm_plan *p, const double *sigma, const uint8_t *mask) {
  if (p && p->flat) return fail(p, DM_EINVAL, "flat-sky plans take dm_set_noise_flat");
  if (!p || !sigma) return DM_EINVAL;
  if (p->session) return fail(p, DM_EBUSY, "a solve is in progress on this plan");
  dm_status r = check_noise(p, sigma, mask);
  if (r != DM_OK) return r;
  p->have_noise = false;  // until every RHS has the new model (a failed upload leaves none)
  r = upload_noise(p, 0, sigma, mask);
  if (r != DM_OK) return r;
  const int64_t np = p->npix;
  for (int b = 1; b < p->batch; ++b) {  // every RHS gets the same noise model
    DM_CU(cudaMemcpy(p->sigma + (size_t)b * 3 * np, p->sigma, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice), "sigma");
    DM_CU(cudaMemcpy(p->mask + (size_t)b * np, p->mask, np, cudaMemcpyDeviceToDevice), "mask");
    DM_CU(cudaMemcpy(p->w + (size_t)b * 3 * np, p->w, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice), "w");
    p->alpha[b] = p->alpha[0];
    p->t_h[b] = p->t_h[0];
  }
  p->have_noise = true;
  p->cov = false;
  p->noise_shared = true;
  p->sigma_h.assign(sigma, sigma + 3 * np);
  if (mask)
    p->mask_h.assign(mask, mask + np);
  else
    p->mask_h.assign(np, 1);
  prog_release(p);
  return refresh_filters(p);
}

dm_status dm_set_noise_mask_rhs(dm_plan *p, int b, const double *sigma, const uint8_t *mask) {
  if (p && p->flat) return fail(p, DM_EINVAL, "flat-sky plans share one noise model (dm_set_noise_flat)");
  if (!p || !sigma || b < 0 || b >= p->batch) return DM_EINVAL;
  if (!p->have_noise) return fail(p, DM_EINVAL, "set the plan-wide noise first (dm_set_noise_mask)");
  if (p->cov) return fail(p, DM_EINVAL, "per-RHS diagonal noise cannot be mixed with dm_set_noise_cov");
  if (p->session) return fail(p, DM_EBUSY, "a solve is in progress on this plan");
  dm_status r = check_noise(p, sigma, mask);
  if (r != DM_OK) return r;
  p->have_noise = false;  // a failed upload leaves RHS b half-set: the plan then needs its noise again
  p->noise_shared = false;
  r = upload_noise(p, b, sigma, mask);
  if (r != DM_OK) return r;
  if (p->have_cl) {
    DM_CU(build_filters(p, b, 0), "filters");
    DM_CU(cudaDeviceSynchronize(), "filters");
  }
  p->have_noise = true;
  return DM_OK;
}

dm_status dm_set_schedule(dm_plan *p, const dm_schedule *s) {
  if (!p || !s) return DM_EINVAL;
  if (p->session) return fail(p, DM_EBUSY, "a solve is in progress on this plan");
  if (s->n_levels < 1 || s->n_levels > DM_MAX_LEVELS || !(s->lambda0 >= 1.0) || s->max_iter < 1 ||
      s->iters_per_level < 0)
    return fail(p, DM_EINVAL, "bad schedule");
  if (s->iters_per_level == 0 && (!(s->eps0 > 0) || !(s->eps_final > 0) || s->eta < 0))
    return fail(p, DM_EINVAL, "bad Cauchy thresholds");
  p->sched = *s;
  if (p->sched.check_every < 1) p->sched.check_every = 1;
  // every RHS takes the schedule's final tolerance (the server then sets its
  // slots' own tolerances through their views)
  p->eps_final_rhs.assign(p->batch, s->eps_final);
  if (!p->forced.empty() && (int)p->forced.size() != s->n_levels) p->forced.clear();
  dm_status r = upload_levels(p);
  if (r != DM_OK) return r;
  return refresh_filters(p);
}

dm_status dm_set_forced_iters(dm_plan *p, const int *iters) {
  if (!p) return DM_EINVAL;
  if (p->session) return fail(p, DM_EBUSY, "a solve is in progress on this plan");
  if (!iters) {
    p->forced.clear();
  } else {
    for (int k = 0; k < p->sched.n_levels; ++k)
      if (iters[k] < 0) return fail(p, DM_EINVAL, "negative iteration count");
    p->forced.assign(iters, iters + p->sched.n_levels);
  }
  return upload_levels(p);
}

dm_status dm_wiener_filter(dm_plan *p, const double *d, double *s_out, double *alm_out, dm_stats *stats,
                           void *stream) {
  dm_status r = check_ready(p);
  if (r != DM_OK) return r;
  if (!d || !s_out) return fail(p, DM_EINVAL, "null buffer");
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(cudaEventRecord(p->ev_begin, st), "event");
  r = run_dm(p, d, st);
  if (r != DM_OK && r != DM_ENOTCONV) return r;
  dm_status r2 = solve_end(p, s_out, alm_out, st, false);
  if (r2 != DM_OK) return r2;
  DM_CU(cudaEventRecord(p->ev_end, st), "event");
  DM_CU(cudaStreamSynchronize(st), "sync");
  fill_stats(p, stats, &r, st);
  return r;
}

dm_status dm_wiener_filter_host(dm_plan *p, const double *d_host, double *s_host, double *alm_host,
                                dm_stats *stats, void *stream) {
  dm_status r = check_ready(p);
  if (r != DM_OK) return r;
  if (!d_host || !s_host) return fail(p, DM_EINVAL, "null buffer");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t mb = sizeof(double) * 3 * p->npix * p->batch;
  DM_CU(cudaEventRecord(p->ev_begin, st), "event");
  // tmpmap2 holds d
  DM_CU(cudaMemcpyAsync(p->tmpmap2, d_host, mb, cudaMemcpyHostToDevice, st), "h2d");
  r = run_dm(p, p->tmpmap2, st);
  if (r != DM_OK && r != DM_ENOTCONV) return r;
  dm_status r2 = solve_end(p, s_host, alm_host, st, true);
  if (r2 != DM_OK) return r2;
  DM_CU(cudaEventRecord(p->ev_end, st), "event");
  DM_CU(cudaStreamSynchronize(st), "sync");
  fill_stats(p, stats, &r, st);
  return r;
}

dm_status dm_draw_cr_inputs(dm_plan *p, const uint64_t *seeds, double *ahat, double *shat, double *dhat,
                            void *stream) {
  if (!p || !seeds) return DM_EINVAL;
  if (!p->have_cl || !p->have_noise) return fail(p, DM_EINVAL, "spectra and noise must be set");
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(cudaMemcpyAsync(p->seeds_dev, seeds, sizeof(uint64_t) * p->batch, cudaMemcpyHostToDevice, st), "seeds");
  DM_CU(p->flat ? flat_draw_signal(p, p->seeds_dev, p->tmpalm, st) : draw_signal(p, p->seeds_dev, p->tmpalm, st),
        "draw signal");
  DM_CU(legendre_synthesis(p, p->tmpalm, st), "synthesis");
  DM_CU(ring_stage(p, RING_INV_MAP, nullptr, p->tmpmap, st), "ring inverse");
  if (dhat) DM_CU(draw_noise_add(p, p->seeds_dev, p->tmpmap, dhat, st), "draw noise");
  const size_t mb = sizeof(double) * 3 * p->npix * p->batch;
  if (shat) DM_CU(cudaMemcpyAsync(shat, p->tmpmap, mb, cudaMemcpyDeviceToDevice, st), "copy shat");
  if (ahat)
    DM_CU(cudaMemcpyAsync(ahat, p->tmpalm, sizeof(double2) * 3 * p->nalm * p->batch, cudaMemcpyDeviceToDevice, st),
          "copy ahat");
  DM_CU(cudaStreamSynchronize(st), "sync");
  return DM_OK;
}

dm_status dm_constrained_realization(dm_plan *p, const double *d, const uint64_t *seeds, double *s_cr_out,
                                     double *alm_cr_out, dm_stats *stats, void *stream) {
  dm_status r = check_ready(p);
  if (r != DM_OK) return r;
  if (!d || !seeds || !s_cr_out) return fail(p, DM_EINVAL, "null buffer");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = 3 * p->npix * p->batch;
  // shat -> tmpmap, ahat -> tmpalm, dhat -> tmpmap2, then tmpmap2 = d - dhat
  DM_CU(cudaEventRecord(p->ev_begin, st), "event");
  DM_CU(cudaMemcpyAsync(p->seeds_dev, seeds, sizeof(uint64_t) * p->batch, cudaMemcpyHostToDevice, st), "seeds");
  DM_CU(p->flat ? flat_draw_signal(p, p->seeds_dev, p->tmpalm, st) : draw_signal(p, p->seeds_dev, p->tmpalm, st),
        "draw signal");
  DM_CU(legendre_synthesis(p, p->tmpalm, st), "synthesis");
  DM_CU(ring_stage(p, RING_INV_MAP, nullptr, p->tmpmap, st), "ring inverse");
  DM_CU(draw_noise_add(p, p->seeds_dev, p->tmpmap, p->tmpmap2, st), "draw noise");
  DM_CU(axpy_maps(n, p->tmpmap2, -2.0, p->tmpmap2, st), "negate");   // -dhat
  DM_CU(axpy_maps(n, d, 1.0, p->tmpmap2, st), "d - dhat");
  r = run_dm(p, p->tmpmap2, st);
  if (r != DM_OK && r != DM_ENOTCONV) return r;
  dm_status r2 = solve_end(p, s_cr_out, alm_cr_out, st, false);
  if (r2 != DM_OK) return r2;
  DM_CU(axpy_maps(n, p->tmpmap, 1.0, s_cr_out, st), "+ shat");
  if (alm_cr_out) DM_CU(axpy_maps(6 * p->nalm * p->batch, (const double *)p->tmpalm, 1.0, alm_cr_out, st), "+ ahat");
  DM_CU(cudaEventRecord(p->ev_end, st), "event");
  DM_CU(cudaStreamSynchronize(st), "sync");
  fill_stats(p, stats, &r, st);
  return r;
}

dm_status dm_alm2map(dm_plan *p, const double *alm, double *map, void *stream) {
  if (!p || !alm || !map) return DM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(legendre_synthesis(p, (const double2 *)alm, st), "synthesis");
  DM_CU(ring_stage(p, RING_INV_MAP, nullptr, map, st), "ring inverse");
  return DM_OK;
}

dm_status dm_map2alm(dm_plan *p, const double *map, double *alm, void *stream) {
  if (!p || !alm || !map) return DM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(ring_stage(p, RING_FWD_MAP, map, nullptr, st), "ring forward");
  DM_CU(legendre_analysis(p, ANA_PLAIN, (double2 *)alm, st), "analysis");
  return DM_OK;
}

dm_status dm_ring_fft_forward(dm_plan *p, const double *map, double *rc, void *stream) {
  if (!p || !map || !rc) return DM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(ring_stage(p, RING_FWD_MAP, map, nullptr, st), "ring forward");
  DM_CU(rc_to_public(p, (double2 *)rc, st), "layout");
  return DM_OK;
}

dm_status dm_ring_fft_inverse(dm_plan *p, const double *rc, double *map, void *stream) {
  if (!p || !map || !rc) return DM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(rc_from_public(p, (const double2 *)rc, st), "layout");
  DM_CU(ring_stage(p, RING_INV_MAP, nullptr, map, st), "ring inverse");
  return DM_OK;
}

dm_status dm_legendre_synthesis(dm_plan *p, const double *alm, double *rc, void *stream) {
  if (!p || !alm || !rc) return DM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(legendre_synthesis(p, (const double2 *)alm, st), "synthesis");
  DM_CU(rc_to_public(p, (double2 *)rc, st), "layout");
  return DM_OK;
}

dm_status dm_legendre_analysis(dm_plan *p, const double *rc, double *alm, void *stream) {
  if (!p || !alm || !rc) return DM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(rc_from_public(p, (const double2 *)rc, st), "layout");
  DM_CU(legendre_analysis(p, ANA_PLAIN, (double2 *)alm, st), "analysis");
  return DM_OK;
}

dm_status dm_apply_filter(dm_plan *p, double lambda, const double *alm_in, double *alm_out, void *stream) {
  if (p && p->flat) return fail(p, DM_EINVAL, "dm_apply_filter takes per-l spectra (sphere plans)");
  if (!p || !alm_in || !alm_out) return DM_EINVAL;
  if (!p->have_cl || !p->have_noise) return fail(p, DM_EINVAL, "spectra and noise must be set");
  if (!(lambda >= 1.0)) return fail(p, DM_EINVAL, "lambda must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(build_filter_one(p, lambda, p->t_h[0], p->coef_tmp, st), "filter");
  DM_CU(apply_filter_level(p, p->coef_tmp, (const double2 *)alm_in, (double2 *)alm_out, st), "apply filter");
  return DM_OK;
}

dm_status dm_solve_begin(dm_plan *p, const double *d, void *stream) {
  dm_status r = check_ready(p);
  if (r != DM_OK) return r;
  if (!d) return fail(p, DM_EINVAL, "null buffer");
  if (p->session) return fail(p, DM_EBUSY, "a solve is already in progress on this plan");
  DM_CU(cudaEventRecord(p->ev_begin, (cudaStream_t)stream), "event");
  r = solve_begin(p, d, (cudaStream_t)stream);
  if (r != DM_OK) end_session(p);
  return r;
}

dm_status dm_solve_iterate(dm_plan *p, int max_iters, int *all_done, void *stream) {
  if (!p || max_iters < 0) return DM_EINVAL;
  int dummy = 0;
  return solve_iterate(p, max_iters, all_done ? all_done : &dummy, (cudaStream_t)stream);
}

dm_status dm_solve_end(dm_plan *p, double *s_out, double *alm_out, dm_stats *stats, void *stream) {
  if (!p) return DM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  dm_status r = solve_end(p, s_out, alm_out, st, false);
  if (r != DM_OK) return r;
  DM_CU(cudaEventRecord(p->ev_end, st), "event");
  DM_CU(cudaStreamSynchronize(st), "sync");
  fill_stats(p, stats, &r, st);
  return r;
}

dm_status dm_jacobi_refine(dm_plan *p, const double *d, int n_refine, double *s_out, double *alm_out,
                           dm_stats *stats, void *stream) {
  dm_status r = check_ready(p);
  if (r != DM_OK) return r;
  if (!d || !s_out || n_refine < 0) return fail(p, DM_EINVAL, "null buffer or negative refinement count");
  if (p->cov) return fail(p, DM_EINVAL, "the Jacobi refinement takes the diagonal noise model");
  if (p->session) return fail(p, DM_EBUSY, "a solve is in progress on this plan");
  cudaStream_t st = (cudaStream_t)stream;
  DM_CU(cudaEventRecord(p->ev_begin, st), "event");
  // the usual solve, whose per-level counts W~ then repeats
  r = run_dm(p, d, st);
  if (r != DM_OK && r != DM_ENOTCONV) return r;
  const dm_status r_solve = r;
  dm_status r2 = solve_end(p, nullptr, nullptr, st, false);
  if (r2 != DM_OK) return r2;
  const int nl = p->sched.n_levels, B = p->batch;
  std::vector<SolveState> hs(B);
  DM_CU(cudaMemcpyAsync(hs.data(), p->state, sizeof(SolveState) * B, cudaMemcpyDeviceToHost, st), "state");
  DM_CU(cudaStreamSynchronize(st), "sync");
  std::vector<int> counts((size_t)B * nl);
  long cap = 4;
  for (int b = 0; b < B; ++b) {
    long tot = 0;
    for (int k = 0; k < nl; ++k) tot += counts[(size_t)b * nl + k] = hs[b].iters_per_level[k];
    cap = std::max(cap, tot + 4);
  }
  DM_CU(jacobi_alloc(p), "refinement buffers");
  const size_t an = sizeof(double2) * 3 * (size_t)p->nalm * B;
  DM_CU(cudaMemcpyAsync(p->jacc, p->a, an, cudaMemcpyDeviceToDevice, st), "copy a");
  const size_t mb = sizeof(double) * 3 * (size_t)p->npix * B;
  for (int it = 0; it < n_refine; ++it) {
    DM_CU(jacobi_source(p, d, st), "refinement source");
    r = upload_levels_counts(p, counts);
    if (r != DM_OK) return r;
    // W~(g): the iteration from a = 0 with w d = 0 and g added before the filter
    DM_CU(cudaMemsetAsync(p->tmpmap2, 0, mb, st), "zero data");
    p->src_active = true;
    r = solve_begin(p, p->tmpmap2, st);
    int all = 0;
    if (r == DM_OK) r = solve_iterate(p, cap, &all, st);
    if (r == DM_OK) r = solve_end(p, nullptr, nullptr, st, false);
    p->src_active = false;
    if (r != DM_OK) {
      end_session(p);
      upload_levels(p);
      return r;
    }
    DM_CU(axpy_maps(6 * p->nalm * B, (const double *)p->a, 1.0, (double *)p->jacc, st), "a += W~ g");
  }
  r = upload_levels(p);
  if (r != DM_OK) return r;
  DM_CU(cudaMemcpyAsync(p->a, p->jacc, an, cudaMemcpyDeviceToDevice, st), "copy a");
  DM_CU(jacobi_final(p, d, st), "final map");
  DM_CU(cudaMemcpyAsync(s_out, p->s64, mb, cudaMemcpyDeviceToDevice, st), "copy s");
  if (alm_out) DM_CU(cudaMemcpyAsync(alm_out, p->a, an, cudaMemcpyDeviceToDevice, st), "copy alm");
  DM_CU(cudaEventRecord(p->ev_end, st), "event");
  DM_CU(cudaStreamSynchronize(st), "sync");
  r = r_solve;
  fill_stats(p, stats, &r, st);
  if (stats)
    for (int b = 0; b < B; ++b) stats[b].iters_total = hs[b].iters_total * (1 + n_refine);
  return r;
}

dm_status dm_set_ff_slab_bytes(dm_plan *p, int64_t bytes) {
  if (!p || bytes < 1) return DM_EINVAL;
  if (p->session) return DM_EBUSY;
  p->ffs_cap = bytes;
  p->ffs_cap_set = true;
  if (p->ffs) cudaFree(p->ffs);
  if (p->ffs_lo) cudaFree(p->ffs_lo);
  p->ffs = p->ffs_lo = nullptr;
  p->ffs_m.clear();
  return DM_OK;
}

dm_status dm_set_analysis_slots(dm_plan *p, int slots) {
  if (!p || slots < 2) return DM_EINVAL;
  if (p->session) return DM_EBUSY;
  if (p->flat) return DM_OK;
  const int ns = std::min(slots, p->nchunk);
  if (ns == p->nslot) return DM_OK;
  prog_release(p);
  const size_t n = (size_t)p->batch * ns * 3 * p->nalm;
  double2 *a = nullptr;
  if (cudaMalloc(&a, sizeof(double2) * n) != cudaSuccess) return fail(p, DM_ENOMEM, "analysis slots");
  cudaFree(p->apart);
  p->bytes += (int64_t)sizeof(double2) * ((int64_t)n - (int64_t)p->batch * p->nslot * 3 * p->nalm);
  p->apart = a;
  p->nslot = ns;
  return DM_OK;
}

dm_status dm_test_tc_withhold(dm_plan *p, int on) {
  if (!p) return DM_EINVAL;
  p->tc_withhold = on != 0;
  return DM_OK;
}

dm_status dm_set_progressive(dm_plan *p, double margin, int lmin) {
  if (!p || !(margin >= 0.0) || !std::isfinite(margin) || lmin < 2) return DM_EINVAL;
  if (p->session) return fail(p, DM_EBUSY, "a solve is in progress on this plan");
  if (margin > 0.0 && (p->flat || (p->nside & (p->nside - 1)) != 0))
    return fail(p, DM_EINVAL, "progressive resolution needs a sphere plan of power-of-two nside");
  p->prog_margin = margin;
  p->prog_lmin = lmin;
  p->prog_res.clear();
  return DM_OK;
}

dm_status dm_get_progressive_levels(const dm_plan *p, int *nside_k, int *lmax_k) {
  if (!p || p->prog_res.empty()) return DM_EINVAL;
  const int nl = (int)p->prog_res.size() / 2;
  for (int k = 0; k < nl; ++k) {
    if (nside_k) nside_k[k] = p->prog_res[2 * k];
    if (lmax_k) lmax_k[k] = p->prog_res[2 * k + 1];
  }
  return DM_OK;
}

dm_status dm_set_diagnostics(dm_plan *p, int on) {
  if (!p) return DM_EINVAL;
  p->diag_on = on != 0;
  return DM_OK;
}

dm_status dm_set_tensor_cores(dm_plan *p, int on) {
  if (!p) return DM_EINVAL;
  prog_release(p);
  p->use_tc = on != 0;
  return DM_OK;
}

dm_status dm_set_tc_tiles(dm_plan *p, int generate) {
  if (!p) return DM_EINVAL;
  if (p->session) return DM_EBUSY;
  prog_release(p);
  p->tc_gen = generate < 0 ? -1 : (generate != 0 ? 1 : 0);
  p->tc_gen_used = -1;
  return DM_OK;
}

dm_status dm_set_ring_radix(dm_plan *p, int lr) {
  if (!p || (lr != 0 && lr != 3 && lr != 4)) return DM_EINVAL;
  p->ring_lr = lr;
  for (int i = 0; i < DM_TUNE_MAX_CLASSES; ++i) p->tune_ring_lr[i] = -1;  // an explicit radix overrides a tuned one
  return DM_OK;
}

dm_status dm_set_refinement(dm_plan *p, int anchor_every) {
  if (!p || anchor_every < 1) return DM_EINVAL;
  prog_release(p);
  p->anchor_every = anchor_every;
  return DM_OK;
}

dm_status dm_profile_enable(dm_plan *p, int on) {
  if (!p) return DM_EINVAL;
  p->prof_on = on != 0;
  memset(&p->prof, 0, sizeof(p->prof));
  p->launches = 0;
  return DM_OK;
}

dm_status dm_profile_read(const dm_plan *p, dm_profile *out) {
  if (!p || !out) return DM_EINVAL;
  *out = p->prof;
  out->launches = p->launches;
  return DM_OK;
}

dm_status dm_noise_info(const dm_plan *p, double *alpha, double *t_h) {
  if (!p || !p->have_noise) return DM_EINVAL;
  if (alpha) *alpha = p->alpha[0];
  if (t_h) *t_h = p->t_h[0];
  return DM_OK;
}

}  // extern "C"
