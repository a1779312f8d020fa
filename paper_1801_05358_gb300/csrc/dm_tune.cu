// dm_tune.cu -- the launch autotuner of the batched iteration: for each
// launch of the ring stage (one per FFT-size class) the radix of the
// fixed-size transforms and the (RHS, field) lanes per block, and for the
// tensor-core Legendre kernels their pipeline depth and l tiles per CTA, each
// picked by timing the candidates with CUDA events on the plan's own buffers.
// Picks are cached per process for (device, nside, lmax, batch, precision,
// tensor cores).  The paper has no counterpart: this is how the batched form
// chooses its tile sizes on the GPU at hand.
#include <math.h>
#include <string.h>

#include <array>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "dm_internal.h"

namespace dmwf {

namespace {

std::mutex g_tune_mu;
std::map<std::string, dm_tuning> g_tune_cache;

std::string tune_key(const dm_plan *p) {
  cudaDeviceProp prop;
  std::string dev = "?";
  if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess)
    dev = std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount);
  return dev + "|" + std::to_string(p->nside) + "|" + std::to_string(p->lmax) + "|" + std::to_string(p->batch) +
         "|" + std::to_string((int)p->prec) + "|" + std::to_string((int)p->ff_legendre) + "|" +
         std::to_string((int)(p->use_tc && tc_batch_ok(p->batch))) + "|" + std::to_string(p->tc_gen);
}

void apply(dm_plan *p, const dm_tuning &t) {
  for (int i = 0; i < DM_TUNE_MAX_CLASSES; ++i) {
    const bool in = i < t.n_ring_classes;
    const int lr = in ? t.ring_radix_lr[i] : -1;
    p->tune_ring_lr[i] = (lr == 0 || lr == 3 || lr == 4) ? lr : -1;
    const int g = in ? t.ring_lanes[i] : 0;
    p->tune_ring_G[i] = (g >= 1 && g <= 16) ? g : 0;
    const int fu = in ? t.ring_fused[i] : -1;
    p->tune_ring_fuse[i] = (fu >= 0 && fu <= 2) ? fu : -1;
  }
  for (int k = 0; k < 2; ++k) {
    p->tune_syn_ns[k] = (t.syn_stages[k] >= 2 && t.syn_stages[k] <= 8) ? t.syn_stages[k] : 0;
    p->tune_ana_lt[k] = (t.ana_ltiles[k] >= 1 && t.ana_ltiles[k] <= 4) ? t.ana_ltiles[k] : 0;
    p->tune_ana_S[k] = (t.ana_stages[k] >= 1 && t.ana_stages[k] <= 5) ? t.ana_stages[k] : 0;
  }
}

// mean device time of `reps` calls of f after one untimed call; < 0 when a
// call failed or a tensor-core wait gave up (the candidate is then skipped)
template <typename F>
float time_it(dm_plan *p, cudaStream_t st, F f, int reps, cudaEvent_t e0, cudaEvent_t e1) {
  if (f() != cudaSuccess) return -1.f;
  cudaEventRecord(e0, st);
  for (int i = 0; i < reps; ++i)
    if (f() != cudaSuccess) return -1.f;
  cudaEventRecord(e1, st);
  if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  if (p->tc_err) {
    int bad = 0;
    cudaMemcpy(&bad, p->tc_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (bad) {
      cudaMemset(p->tc_err, 0, sizeof(int));
      return -1.f;
    }
  }
  return ms / reps;
}

}  // namespace

// Tune the plan's launches in place; on return p->tuning holds the picks.
dm_status autotune(dm_plan *p, cudaStream_t st, std::string &err) {
  const int ncls = std::min((int)p->ring_classes.size(), DM_TUNE_MAX_CLASSES);
  const bool tc = p->prec == DM_MIXED_FP32 && p->use_tc && tc_batch_ok(p->batch);
  const int reps = 3;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    err = "event creation failed";
    return DM_ECUDA;
  }
  const bool sa = p->state_active, aa = p->anchor_active;
  p->state_active = false;
  p->anchor_active = false;
  dm_tuning t{};
  t.n_ring_classes = ncls;
  dm_status rs = DM_OK;
  // ---- ring stage: per class, every (radix, lanes per block) the launch allows
  for (int ci = 0; ci < ncls && rs == DM_OK; ++ci) {
    p->tune_only_class = ci;
    auto run = [&]() { return ring_stage(p, RING_ITER, nullptr, p->s64, st); };
    p->tune_ring_lr[ci] = -1;
    p->tune_ring_G[ci] = 0;
    p->tune_ring_fuse[ci] = -1;
    const float t_def = time_it(p, st, run, reps, e0, e1);
    if (t_def < 0.f) {
      err = "ring stage failed with the default configuration";
      rs = DM_ECUDA;
      break;
    }
    // a candidate is (radix, lanes per block, pass variant: 1 fused update
    // pass, 0 separate passes, 2 separate passes with the register-capped
    // radix-16 kernels); the generic kernels have no variants
    auto used_now = [&]() {
      const int lr = p->ring_lr_used[ci];
      return std::array<int, 3>{lr, p->ring_G_used[ci], lr > 0 ? p->ring_fuse_used[ci] : 0};
    };
    float best = t_def;
    std::array<int, 3> bestc = used_now();
    std::vector<std::array<int, 3>> seen{bestc};
    const int lrs[3] = {3, 4, 0};
    for (int li = 0; li < 3; ++li)
      for (int fu : {1, 0, 2}) {
        if (lrs[li] == 0 && fu != 1) continue;
        if (fu == 2 && (lrs[li] != 4 || p->prec == DM_FP64)) continue;
        for (int g = 1; g <= 16; ++g) {
          p->tune_ring_lr[ci] = lrs[li];
          p->tune_ring_G[ci] = g;
          p->tune_ring_fuse[ci] = fu;
          if (run() != cudaSuccess) break;  // the untimed probe call sets the *_used fields
          const std::array<int, 3> used = used_now();
          bool dup = false;
          for (auto &s : seen) dup = dup || s == used;
          if (dup) continue;
          seen.push_back(used);
          const float ms = time_it(p, st, run, reps, e0, e1);
          if (ms > 0.f && ms < best) {
            best = ms;
            bestc = used;
          }
        }
      }
    t.ring_radix_lr[ci] = bestc[0];
    t.ring_lanes[ci] = bestc[1];
    t.ring_fused[ci] = bestc[0] > 0 ? bestc[2] : -1;
    p->tune_ring_lr[ci] = bestc[0];
    p->tune_ring_G[ci] = bestc[1];
    p->tune_ring_fuse[ci] = t.ring_fused[ci];
    t.ms_ring += best;
    t.ms_ring_default += t_def;
  }
  p->tune_only_class = -1;
  // ---- tensor-core Legendre stages
  if (tc && rs == DM_OK) {
    for (int part = 0; part < 2 && rs == DM_OK; ++part) {
      p->tune_only_part = part;
      auto syn = [&]() { return legendre_synthesis_tc(p, p->a, st); };
      p->tune_syn_ns[part] = 0;
      const float s_def = time_it(p, st, syn, reps, e0, e1);
      if (s_def < 0.f) {
        err = "tensor-core synthesis failed with the default configuration";
        rs = DM_ECUDA;
        break;
      }
      float best = s_def;
      int best_ns = p->syn_ns_used[part];
      std::vector<int> seen{best_ns};
      for (int ns = 2; ns <= 8; ++ns) {
        p->tune_syn_ns[part] = ns;
        if (syn() != cudaSuccess) break;
        const int used = p->syn_ns_used[part];
        bool dup = false;
        for (int v : seen) dup = dup || v == used;
        if (dup) continue;
        seen.push_back(used);
        const float ms = time_it(p, st, syn, reps, e0, e1);
        if (ms > 0.f && ms < best) {
          best = ms;
          best_ns = used;
        }
      }
      t.syn_stages[part] = best_ns;
      p->tune_syn_ns[part] = best_ns;
      t.ms_synthesis += best;
      t.ms_synthesis_default += s_def;

      auto ana = [&]() { return legendre_analysis_tc(p, st); };
      p->tune_ana_lt[part] = 0;
      p->tune_ana_S[part] = 0;
      const float a_def = time_it(p, st, ana, reps, e0, e1);
      if (a_def < 0.f) {
        err = "tensor-core analysis failed with the default configuration";
        rs = DM_ECUDA;
        break;
      }
      best = a_def;
      int best_lt = p->ana_lt_used[part], best_S = p->ana_S_used[part];
      std::vector<std::pair<int, int>> aseen{{best_lt, best_S}};
      for (int lt = 1; lt <= 4; ++lt)
        for (int S = 2; S <= (p->tc_gen ? 5 : 4); ++S) {
          p->tune_ana_lt[part] = lt;
          p->tune_ana_S[part] = S;
          if (ana() != cudaSuccess) break;
          const std::pair<int, int> used{p->ana_lt_used[part], p->ana_S_used[part]};
          bool dup = false;
          for (auto &v : aseen) dup = dup || v == used;
          if (dup) continue;
          aseen.push_back(used);
          const float ms = time_it(p, st, ana, reps, e0, e1);
          if (ms > 0.f && ms < best) {
            best = ms;
            best_lt = used.first;
            best_S = used.second;
          }
        }
      t.ana_ltiles[part] = best_lt;
      t.ana_stages[part] = best_S;
      p->tune_ana_lt[part] = best_lt;
      p->tune_ana_S[part] = best_S;
      t.ms_analysis += best;
      t.ms_analysis_default += a_def;
    }
    p->tune_only_part = -1;
  }
  p->tune_only_class = -1;
  p->tune_only_part = -1;
  p->state_active = sa;
  p->anchor_active = aa;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (p->tc_err) cudaMemset(p->tc_err, 0, sizeof(int));
  if (rs != DM_OK) return rs;
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    err = "a tuning launch failed";
    return DM_ECUDA;
  }
  apply(p, t);
  p->tuning = t;
  p->tuned = true;
  return DM_OK;
}

}  // namespace dmwf

using namespace dmwf;

extern "C" {

dm_status dm_autotune(dm_plan *p, int force, void *stream) {
  if (!p) return DM_EINVAL;
  if (p->session) {
    p->err = "dm_autotune: a solve is in progress on this plan";
    return DM_EBUSY;
  }
  const std::string key = tune_key(p);
  if (!force) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      apply(p, it->second);
      p->tuning = it->second;
      p->tuning.from_cache = 1;
      p->tuned = true;
      return DM_OK;
    }
  }
  std::string err;
  dm_status r = autotune(p, (cudaStream_t)stream, err);
  if (r != DM_OK) {
    p->err = "dm_autotune: " + err;
    return r;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = p->tuning;
  return DM_OK;
}

dm_status dm_get_tuning(const dm_plan *p, dm_tuning *out) {
  if (!p || !out) return DM_EINVAL;
  if (p->tuned) {
    *out = p->tuning;
    return DM_OK;
  }
  memset(out, 0, sizeof(*out));
  out->n_ring_classes = std::min((int)p->ring_classes.size(), DM_TUNE_MAX_CLASSES);
  for (int i = 0; i < DM_TUNE_MAX_CLASSES; ++i) {
    out->ring_radix_lr[i] = p->tune_ring_lr[i];
    out->ring_lanes[i] = p->tune_ring_G[i];
    out->ring_fused[i] = p->tune_ring_fuse[i];
  }
  for (int k = 0; k < 2; ++k) {
    out->syn_stages[k] = p->tune_syn_ns[k];
    out->ana_ltiles[k] = p->tune_ana_lt[k];
    out->ana_stages[k] = p->tune_ana_S[k];
  }
  return DM_OK;
}

dm_status dm_set_tuning(dm_plan *p, const dm_tuning *t) {
  if (!p || !t) return DM_EINVAL;
  if (p->session) {
    p->err = "dm_set_tuning: a solve is in progress on this plan";
    return DM_EBUSY;
  }
  apply(p, *t);
  p->tuning = *t;
  p->tuning.from_cache = 0;
  p->tuned = true;
  return DM_OK;
}

}  // extern "C"
