// dm_serve.cu -- continuous-batching server for Wiener-filter and
// constrained-realisation requests of different geometries.
//
// A pool is one dm_plan per (nside, lmax, spectra, precision) whose RHS are
// slots; a request tighter than the strict tolerance goes to an FP64-class
// pool (DM_FP64 or DM_FLOAT_FLOAT), any other to the default mode.  One
// worker thread owns the device work:
//   admission : queued requests go to free slots of their pool, or into a new
//               pool while the device-memory budget allows; a slot is set up
//               alone through a one-RHS view of the plan (its own noise, mask,
//               alpha, filters, tolerance, data, and for a constrained
//               realisation its Philox draws), including its first iteration;
//   rounds    : every pool with busy slots and no round in flight enqueues
//               iters_per_round dual messenger iterations on its own stream
//               and a copy of its solver states behind them; the worker polls
//               the rounds' events, so pools of different sizes run
//               concurrently and a small pool is not held to a large one's
//               pace; free or finished slots are skipped by the kernels;
//   retirement: a slot whose last level met its stopping rule writes its map
//               to the caller's buffer and frees the slot for the queue.
// The messenger state of a request stays on the device from admission to
// retirement.  Results do not depend on what else shares the pool: every
// kernel acts per RHS (tested: result alone == result in the mix).
#include <math.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "dm_internal.h"

using namespace dmwf;

namespace {

using clk = std::chrono::steady_clock;

double ms_since(clk::time_point t0) {
  return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
}

struct Request {
  uint64_t ticket = 0;
  int nside = 0, lmax = 0, kind = 0;
  double tol = 1e-6;
  uint64_t seed = 0;
  std::vector<double> cl, sigma, d;
  std::vector<uint8_t> mask;
  bool has_mask = false;
  double *s_out = nullptr;
  clk::time_point t_submit;
  double queue_ms = 0.0;
};

struct Slot {
  bool busy = false;
  std::unique_ptr<Request> req;
  int since_anchor = 0;
};

struct Pool {
  int nside = 0, lmax = 0;
  uint64_t cl_hash = 0;
  dm_precision prec = DM_FP64;  // mode the plan was set to (DM_FLOAT_FLOAT kept as such)
  dm_plan *plan = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<Slot> slots;
  // a round in flight: its iterations and the copy of the solver states into
  // hs (pinned) are enqueued, done_ev is recorded after them
  bool inflight = false;
  cudaEvent_t done_ev = nullptr;
  SolveState *hs = nullptr;
  int busy() const {
    int n = 0;
    for (auto &s : slots) n += s.busy ? 1 : 0;
    return n;
  }
};

uint64_t hash_bytes(const void *p, size_t n) {  // FNV-1a
  const unsigned char *c = (const unsigned char *)p;
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

// One-RHS view of a plan: same tables, every per-RHS buffer offset to slot b.
dm_plan make_view(const dm_plan *p, int b) {
  dm_plan v = *p;
  v.batch = 1;
  v.prof_on = false;
  v.ev.clear();
  const size_t n3 = 3 * (size_t)p->npix, na = 3 * (size_t)p->nalm;
  const size_t nrc = 3 * (size_t)(p->mmax + 1) * p->npairs * 2;
  v.rc += b * nrc;
  v.a += b * na;
  v.apart += (size_t)b * p->nslot * na;
  v.wd += b * n3;
  v.norms += (size_t)b * 3 * p->nrings * 2;
  v.state += b;
  v.lev += b;
  v.tmpmap += b * n3;
  v.tmpmap2 += b * n3;
  v.tmpalm += b * na;
  v.seeds_dev += b;
  v.s64 += b * n3;
  v.rhi += b * n3;
  v.w += b * n3;
  v.sigma += b * n3;
  v.mask += (size_t)b * p->npix;
  v.filt += (size_t)b * p->filt_levels * 4 * (p->lmax + 1);
  if (p->fp32_ready) {
    v.rc32 += b * nrc;
    v.apart32 += (size_t)b * p->nchunk32 * na;
    v.s32 += b * n3;
    v.w32 += b * n3;
    v.wd32 += b * n3;
    v.a_hi += b * na;
    v.g_hi += b * na;
    v.shi32 += b * n3;
    v.e32 += b * na;
    v.c32 += b * na;
    v.clev += b;
  }
  if (p->filt32) v.filt32 += (size_t)b * p->filt_levels * 4 * (p->lmax + 1);
  v.alpha.assign(1, p->alpha[b]);
  v.t_h.assign(1, p->t_h[b]);
  v.eps_final_rhs.assign(1, p->eps_final_rhs.empty() ? p->sched.eps_final : p->eps_final_rhs[b]);
  return v;
}

__global__ void k_mark_done(SolveState *st, int n) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) st[b].done = 1;
}

__global__ void k_sub_maps(const double *__restrict__ x, double *__restrict__ y, int64_t n) {  // y = x - y
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] - y[i];
}

// rough device footprint of a pool, from the plan's own allocation list
size_t estimate_bytes(int nside, int lmax, int S, dm_precision prec) {
  const double npix = 12.0 * nside * nside, nalm = (lmax + 1.0) * (lmax + 2.0) / 2.0, npairs = 2.0 * nside;
  const double nchunk = ceil(npairs / 64.0);
  double b = 0;
  b += S * 3 * (lmax + 1.0) * npairs * 2 * 16;   // rc
  b += S * nchunk * 3 * nalm * 16;               // apart
  b += S * 3 * nalm * 16 * 2;                    // a, tmpalm
  b += S * 3 * npix * 8 * 7;                     // wd, tmpmap(2), s64, rhi, w, sigma
  b += nalm * 48 + (lmax + 1.0) * npairs * 28;   // coefficients, seeds
  const bool tc = prec == DM_MIXED_FP32 && dmwf::tc_batch_ok(S);
  const bool stored = tc && dmwf::tc_tables_fit(lmax, lmax, (int)npairs, S);
  if (prec != DM_FP64) {                         // DM_MIXED_FP32 and DM_FLOAT_FLOAT
    const double full = 3 * nalm * npairs * 4 * 2;  // FP32 tables, hi and lo
    if (stored || (prec == DM_MIXED_FP32 && !tc) || (prec == DM_FLOAT_FLOAT && full <= 32.0 * (1u << 30)) ||
        full <= (double)(1u << 30))
      b += full;
    else
      b += (double)(1u << 30);                   // per-slab tables of the float-float stages
    b += S * 3 * (lmax + 1.0) * npairs * 2 * 8;  // rc32
    b += S * nchunk * 3 * nalm * 8;              // apart32
    b += S * 3 * npix * 4 * 4;                   // s32, w32, wd32, shi32
    b += S * 3 * nalm * 16 * 2;                  // a_hi, g_hi
    b += S * 3 * nalm * 8 * 2;                   // e32, c32
  }
  if (stored)
    b += (double)dmwf::tc_table_bytes(lmax, lmax, (int)npairs, S);  // tiled BF16 tables
  else if (tc)
    b += (double)dmwf::gen_bytes(lmax, lmax, (int)npairs) + S * (lmax + 1.0) * (lmax + 2.0) * 12 * 32;  // checkpoints, B scratch
  return (size_t)(b * 1.05) + (64u << 20);
}

}  // namespace

struct dm_server {
  dm_server_config cfg{};
  int device = 0;
  size_t used = 0;
  std::vector<std::unique_ptr<Pool>> pools;
  std::deque<std::unique_ptr<Request>> pending;
  std::map<uint64_t, dm_result> done;
  std::map<uint64_t, bool> known;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::thread worker;
  std::string err;
  std::atomic<int64_t> rounds{0}, admitted{0}, retired{0};  // written by the worker, read by dm_server_info
};

namespace {

void finish(dm_server *S, Request &r, dm_status st, int iters, double cauchy) {
  dm_result res{};
  res.status = st;
  res.iters = iters;
  res.cauchy_final = cauchy;
  res.latency_ms = ms_since(r.t_submit);
  res.queue_ms = r.queue_ms;
  std::lock_guard<std::mutex> lk(S->mu);
  S->done[r.ticket] = res;
}

// Requests tighter than strict_tol go to pools of strict_prec, the rest to
// pools of prec.
dm_precision request_prec(const dm_server *S, const Request &r) {
  return (S->cfg.strict_tol > 0.0 && r.tol < S->cfg.strict_tol) ? S->cfg.strict_prec : S->cfg.prec;
}

void release_pool(Pool *q) {
  if (q->done_ev) cudaEventDestroy(q->done_ev);
  if (q->hs) cudaFreeHost(q->hs);
  cudaStreamDestroy(q->stream);
  dm_plan_destroy(q->plan);
}

// A new pool for r, or nullptr with *why = DM_ENOMEM when the budget (or the
// device) has no room for it, else the status of the call that rejected r.
Pool *make_pool(dm_server *S, const Request &r, dm_status *why) {
  *why = DM_ENOMEM;
  const int slots = S->cfg.slots_per_plan;
  const dm_precision prec = request_prec(S, r);
  size_t need = estimate_bytes(r.nside, r.lmax, slots, prec);
  if (S->used + need > S->cfg.hbm_budget_bytes) {
    // free idle pools (no busy slot) to make room
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t i = 0; i < S->pools.size();) {
      Pool *q = S->pools[i].get();
      if (q->busy() == 0) {
        S->used -= estimate_bytes(q->nside, q->lmax, slots, q->prec);
        release_pool(q);
        S->pools.erase(S->pools.begin() + i);
      } else {
        ++i;
      }
    }
    if (S->used + need > S->cfg.hbm_budget_bytes) return nullptr;
  }
  auto pool = std::make_unique<Pool>();
  pool->nside = r.nside;
  pool->lmax = r.lmax;
  pool->cl_hash = hash_bytes(r.cl.data(), r.cl.size() * sizeof(double));
  pool->prec = prec;
  dm_status rs = dm_plan_create(r.nside, r.lmax, slots, &pool->plan);
  if (rs != DM_OK) {
    *why = rs == DM_EINVAL ? DM_EINVAL : DM_ENOMEM;
    return nullptr;
  }
  dm_plan *p = pool->plan;
  dm_schedule sc = S->cfg.sched;
  sc.iters_per_level = 0;
  if ((rs = dm_set_schedule(p, &sc)) != DM_OK || (rs = dm_set_spectra(p, r.cl.data())) != DM_OK ||
      (rs = dm_set_noise_mask(p, r.sigma.data(), r.has_mask ? r.mask.data() : nullptr)) != DM_OK ||
      (rs = dm_set_precision(p, prec)) != DM_OK) {
    dm_plan_destroy(p);
    *why = rs;
    return nullptr;
  }
  p->anchor_every = S->cfg.anchor_every > 0 ? S->cfg.anchor_every : 256;
  // Pools run their rounds concurrently; the strict-precision pools, whose
  // requests are the long ones, take the higher stream priority so that the
  // short rounds of the default pools fill the gaps instead of delaying them.
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  const int prio = (prec == S->cfg.strict_prec && S->cfg.strict_prec != S->cfg.prec) ? prio_hi : prio_lo;
  if (cudaStreamCreateWithPriority(&pool->stream, cudaStreamNonBlocking, prio) != cudaSuccess) {
    dm_plan_destroy(p);
    *why = DM_ECUDA;
    return nullptr;
  }
  if (cudaEventCreateWithFlags(&pool->done_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&pool->hs, sizeof(SolveState) * slots) != cudaSuccess) {
    if (pool->done_ev) cudaEventDestroy(pool->done_ev);
    cudaStreamDestroy(pool->stream);
    dm_plan_destroy(p);
    *why = DM_ECUDA;
    return nullptr;
  }
  pool->slots.resize(slots);
  k_mark_done<<<(slots + 127) / 128, 128, 0, pool->stream>>>(p->state, slots);
  p->session = true;
  p->state_active = true;
  if (prec == DM_MIXED_FP32) p->anchor_active = true;
  cudaStreamSynchronize(pool->stream);
  std::lock_guard<std::mutex> lk(S->mu);
  S->used += need;
  S->pools.push_back(std::move(pool));
  return S->pools.back().get();
}

Pool *find_pool(dm_server *S, const Request &r, bool *full) {
  const uint64_t h = hash_bytes(r.cl.data(), r.cl.size() * sizeof(double));
  const dm_precision prec = request_prec(S, r);
  *full = false;
  for (auto &q : S->pools)
    if (q->nside == r.nside && q->lmax == r.lmax && q->cl_hash == h && q->prec == prec) {
      // a pool with a round in flight takes new requests when the round ends
      // (setting a slot up waits on the pool's stream)
      if (!q->inflight && q->busy() < (int)q->slots.size()) return q.get();
      *full = true;
    }
  return nullptr;
}

// Set slot b up alone and run its first iteration (t_0 = d), then anchor.
dm_status slot_begin(Pool *pool, int b, Request &r) {
  dm_plan *p = pool->plan;
  cudaStream_t st = pool->stream;
  const int64_t n3 = 3 * p->npix;
  dm_plan v = make_view(p, b);
  // noise and mask of this request, its alpha, T_h, weights and filters
  cudaMemcpyAsync(v.sigma, r.sigma.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, st);
  if (r.has_mask)
    cudaMemcpyAsync(v.mask, r.mask.data(), p->npix, cudaMemcpyHostToDevice, st);
  else
    cudaMemsetAsync(v.mask, 1, p->npix, st);
  if (build_noise(&v, 0, st) != cudaSuccess) return DM_ECUDA;
  p->alpha[b] = v.alpha[0];
  p->t_h[b] = v.t_h[0];
  v.filt_levels = p->filt_levels;
  v.filt = p->filt + (size_t)b * p->filt_levels * 4 * (p->lmax + 1);
  if (p->filt32) v.filt32 = p->filt32 + (size_t)b * p->filt_levels * 4 * (p->lmax + 1);
  {
    const int nl = (int)p->lambdas.size();
    for (int k = 0; k < nl; ++k)
      build_filter_one(p, p->lambdas[k], p->t_h[b], v.filt + (size_t)k * 4 * (p->lmax + 1), st);
  }
  // tolerance of this request
  p->eps_final_rhs[b] = r.tol;
  v.eps_final_rhs.assign(1, r.tol);
  if (upload_levels(&v) != DM_OK) return DM_ECUDA;
  // data (constrained realisation: d - dhat, shat kept in tmpmap)
  cudaMemcpyAsync(v.tmpmap2, r.d.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, st);
  if (r.kind == DM_REQ_CR) {
    cudaMemcpyAsync(v.seeds_dev, &r.seed, sizeof(uint64_t), cudaMemcpyHostToDevice, st);
    const dm_precision pr = v.prec;
    v.prec = DM_FP64;  // draws and their synthesis in FP64
    v.state_active = false;
    draw_signal(&v, v.seeds_dev, v.tmpalm, st);
    legendre_synthesis(&v, v.tmpalm, st);
    ring_stage(&v, RING_INV_MAP, nullptr, v.tmpmap, st);
    draw_noise_add(&v, v.seeds_dev, v.tmpmap, v.rhi, st);   // dhat into rhi (free until the first anchor)
    k_sub_maps<<<512, 256, 0, st>>>(v.tmpmap2, v.rhi, n3);  // rhi := d - dhat
    cudaMemcpyAsync(v.tmpmap2, v.rhi, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st);
    v.prec = pr;
  }
  dm_status rs = solve_begin(&v, v.tmpmap2, st);
  if (rs != DM_OK) return rs;
  if (enqueue_iteration(&v, st, nullptr) != cudaSuccess) return DM_ECUDA;
  if (v.prec != DM_FP64) {
    rs = anchor(&v, st, false, nullptr, true);
    if (rs != DM_OK) return rs;
  }
  pool->slots[b].since_anchor = 0;
  return cudaStreamSynchronize(st) == cudaSuccess ? DM_OK : DM_ECUDA;
}

void slot_end(dm_server *S, Pool *pool, int b, const SolveState &ss) {
  dm_plan *p = pool->plan;
  cudaStream_t st = pool->stream;
  Request &r = *pool->slots[b].req;
  dm_plan v = make_view(p, b);
  dm_status rs = DM_OK;
  if (v.prec != DM_FP64) rs = anchor(&v, st, false, nullptr, false);  // s = Y a in FP64
  const int64_t n3 = 3 * p->npix;
  if (rs == DM_OK && r.kind == DM_REQ_CR) axpy_maps(n3, v.tmpmap, 1.0, v.s64, st);
  if (rs == DM_OK) cudaMemcpyAsync(r.s_out, v.s64, sizeof(double) * n3, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) rs = DM_ECUDA;
  finish(S, r, rs != DM_OK ? rs : (ss.notconv ? DM_ENOTCONV : DM_OK), ss.iters_total, ss.cauchy);
  std::lock_guard<std::mutex> lk(S->mu);
  pool->slots[b].busy = false;
  pool->slots[b].req.reset();
  S->retired++;
}

void worker_main(dm_server *S) {
  cudaSetDevice(S->device);
  const int N = std::max(1, S->cfg.iters_per_round);
  for (;;) {
    // ---- admission
    std::vector<std::pair<Pool *, int>> fresh;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      bool any_busy = false;
      for (auto &q : S->pools) any_busy = any_busy || q->busy() > 0;
      if (S->pending.empty() && !any_busy) {
        if (S->stop) return;
        S->cv.wait_for(lk, std::chrono::milliseconds(50));
        continue;
      }
      // no iterator survives an unlock: requests are moved out of the queue
      // before a pool is created without the lock held
      for (size_t idx = 0; idx < S->pending.size();) {
        bool full = false;
        Pool *pool = find_pool(S, *S->pending[idx], &full);
        if (!pool && !full) {
          std::unique_ptr<Request> req = std::move(S->pending[idx]);
          S->pending.erase(S->pending.begin() + idx);
          lk.unlock();
          dm_status why = DM_OK;
          pool = make_pool(S, *req, &why);
          lk.lock();
          if (!pool) {
            bool busy_elsewhere = false;
            for (auto &q : S->pools) busy_elsewhere = busy_elsewhere || q->busy() > 0;
            if (why != DM_ENOMEM || !busy_elsewhere) {  // rejected, or can never fit: fail the request
              dm_result res{};
              res.status = why;
              res.latency_ms = ms_since(req->t_submit);
              S->done[req->ticket] = res;
            } else {                // retry once memory frees up
              S->pending.insert(S->pending.begin() + std::min(idx, S->pending.size()), std::move(req));
              ++idx;
            }
            continue;
          }
          req->queue_ms = ms_since(req->t_submit);
          pool->slots[0].busy = true;
          pool->slots[0].req = std::move(req);
          fresh.emplace_back(pool, 0);
          continue;
        }
        if (!pool) {
          ++idx;
          continue;
        }
        int b = -1;
        for (int i = 0; i < (int)pool->slots.size(); ++i)
          if (!pool->slots[i].busy) {
            b = i;
            break;
          }
        if (b < 0) {
          ++idx;
          continue;
        }
        std::unique_ptr<Request> req = std::move(S->pending[idx]);
        S->pending.erase(S->pending.begin() + idx);
        req->queue_ms = ms_since(req->t_submit);
        pool->slots[b].busy = true;
        pool->slots[b].req = std::move(req);
        fresh.emplace_back(pool, b);
      }
    }
    for (auto &pb : fresh) {
      Pool *pool = pb.first;
      const int b = pb.second;
      dm_status rs = slot_begin(pool, b, *pool->slots[b].req);
      S->admitted++;
      if (rs != DM_OK) {
        finish(S, *pool->slots[b].req, rs, 0, 0.0);
        k_mark_done<<<1, 1, 0, pool->stream>>>(pool->plan->state + b, 1);
        std::lock_guard<std::mutex> lk(S->mu);
        pool->slots[b].busy = false;
        pool->slots[b].req.reset();
      }
    }
    // ---- rounds: every pool with busy slots and no round in flight starts
    // one of N iterations; pools of different sizes run concurrently, each
    // on its own stream, and each is retired as soon as its own round ends
    bool progressed = !fresh.empty();
    for (auto &qq : S->pools) {
      Pool *q = qq.get();
      if (q->inflight || q->busy() == 0) continue;
      for (int k = 0; k < N; ++k) enqueue_iteration(q->plan, q->stream, nullptr);
      cudaMemcpyAsync(q->hs, q->plan->state, sizeof(SolveState) * q->slots.size(), cudaMemcpyDeviceToHost,
                      q->stream);
      cudaEventRecord(q->done_ev, q->stream);
      q->inflight = true;
    }
    // ---- retirement and anchors of the pools whose round has ended
    for (auto &qq : S->pools) {
      Pool *q = qq.get();
      if (!q->inflight || cudaEventQuery(q->done_ev) != cudaSuccess) continue;
      q->inflight = false;
      progressed = true;
      S->rounds++;
      for (int b = 0; b < (int)q->slots.size(); ++b) {
        Slot &sl = q->slots[b];
        if (!sl.busy) continue;
        if (q->hs[b].done) {
          slot_end(S, q, b, q->hs[b]);
          continue;
        }
        sl.since_anchor += N;
        if (q->plan->prec != DM_FP64 && sl.since_anchor >= q->plan->anchor_every) {
          dm_plan v = make_view(q->plan, b);
          anchor(&v, q->stream, false, nullptr, true);
          sl.since_anchor = 0;
        }
      }
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" {

dm_status dm_server_create(const dm_server_config *cfg, dm_server **out) {
  if (!cfg || !out) return DM_EINVAL;
  *out = nullptr;
  if (cfg->slots_per_plan < 1 || cfg->slots_per_plan > 1024 || cfg->hbm_budget_bytes == 0 ||
      (cfg->prec != DM_FP64 && cfg->prec != DM_MIXED_FP32) || !(cfg->strict_tol >= 0.0) ||
      (cfg->strict_tol > 0.0 && cfg->strict_prec != DM_FP64 && cfg->strict_prec != DM_FLOAT_FLOAT))
    return DM_EINVAL;
  dm_server *S = new dm_server();
  S->cfg = *cfg;
  if (S->cfg.max_pending <= 0) S->cfg.max_pending = 100000;
  cudaGetDevice(&S->device);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return DM_OK;
}

dm_status dm_serve_submit(dm_server *S, const dm_request *q, uint64_t *ticket) {
  if (!S || !q || !ticket) return DM_EINVAL;
  if (q->nside < 1 || q->nside > 1024 || q->lmax < 2 || q->lmax > 4 * q->nside || !q->cl || !q->sigma || !q->d ||
      !q->s_out || (q->kind != DM_REQ_WF && q->kind != DM_REQ_CR) || !(q->tol > 0.0))
    return DM_EINVAL;
  const int64_t npix = 12LL * q->nside * q->nside;
  int64_t observed = 0;
  for (int64_t i = 0; i < npix; ++i) {
    if (q->mask && !q->mask[i]) continue;
    ++observed;
    for (int f = 0; f < 3; ++f) {
      const double s = q->sigma[f * npix + i];
      if (!(s > 0.0) || !std::isfinite(s)) return DM_EINVAL;
    }
  }
  if (observed == 0) return DM_EINVAL;  // the mask leaves nothing to filter
  auto r = std::make_unique<Request>();
  r->nside = q->nside;
  r->lmax = q->lmax;
  r->kind = q->kind;
  r->tol = q->tol;
  r->seed = q->seed;
  r->cl.assign(q->cl, q->cl + 4 * (size_t)(q->lmax + 1));
  r->sigma.assign(q->sigma, q->sigma + 3 * npix);
  r->d.assign(q->d, q->d + 3 * npix);
  r->has_mask = q->mask != nullptr;
  if (q->mask) r->mask.assign(q->mask, q->mask + npix);
  r->s_out = q->s_out;
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int64_t)S->pending.size() >= S->cfg.max_pending) return DM_EBUSY;  // admission overflow
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    S->known[r->ticket] = true;
    S->pending.push_back(std::move(r));
  }
  S->cv.notify_all();
  return DM_OK;
}

dm_status dm_serve_poll(dm_server *S, uint64_t ticket, dm_result *out) {
  if (!S || !out) return DM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->done.find(ticket);
  if (it == S->done.end()) return S->known.count(ticket) ? DM_EAGAIN : DM_EINVAL;
  *out = it->second;
  S->done.erase(it);
  S->known.erase(ticket);
  return DM_OK;
}

dm_status dm_serve_cancel(dm_server *S, uint64_t ticket) {
  if (!S) return DM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto it = S->pending.begin(); it != S->pending.end(); ++it)
    if ((*it)->ticket == ticket) {
      dm_result res{};
      res.status = DM_EAGAIN;
      res.latency_ms = ms_since((*it)->t_submit);
      S->done[ticket] = res;
      S->pending.erase(it);
      return DM_OK;
    }
  return DM_EBUSY;  // already admitted (runs to completion) or unknown
}

dm_status dm_server_info(dm_server *S, dm_server_info_t *out) {
  if (!S || !out) return DM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  out->pending = (int64_t)S->pending.size();
  int64_t busy = 0;
  for (auto &q : S->pools) busy += q->busy();
  out->busy_slots = busy;
  out->pools = (int64_t)S->pools.size();
  out->bytes_reserved = (int64_t)S->used;
  out->rounds = S->rounds.load();
  out->admitted = S->admitted.load();
  out->retired = S->retired.load();
  return DM_OK;
}

void dm_server_destroy(dm_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto &q : S->pools) {
    if (q->inflight) cudaEventSynchronize(q->done_ev);
    release_pool(q.get());
  }
  delete S;
}

}  // extern "C"
