// dm_internal.h -- plan layout and kernel launchers shared by the CUDA
// translation units of libdmwf.  Not part of the public ABI (include/dmwf.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <algorithm>
#include <vector>

#include "../../include/dmwf.h"

namespace dmwf {

constexpr int DIAG_TAB_W = 12;  // doubles per l of the diagnostic tables

// Per-ring geometry and FFT plan (device array, one entry per ring).
struct RingDev {
  int64_t start;     // first pixel of the ring (RING order)
  int n;             // pixels in the ring (4i or 4 nside)
  int h;             // n / 2: length of the complex FFT of the packed real ring
  int M;             // FFT size: h when h is a power of two, else the Bluestein size
  int bluestein;     // 1 when h is not a power of two
  int shift;         // 1 when the first pixel sits half a pixel east of phi = 0
  int pair;          // ring-pair index (north ring index - 1)
  int side;          // 0 = northern (or equatorial) member, 1 = southern member
  int64_t ph_off;    // offset of e^{-i pi q / n}, q in [0, 2n), in the phase table
  int64_t bh_off;    // offset of the Bluestein kernel spectrum (M entries), -1 if none
  int64_t ch_off;    // offset of the Bluestein chirp e^{-i pi j^2 / h} (h entries), -1 if none
};

// Per-ring-pair data for the Legendre stages.
struct PairDev {
  double x;          // cos(theta) of the northern ring
  double omz, opz;   // 1 - x and 1 + x without cancellation
};

// Per-(m, l) recurrence coefficients (m-major like the alm index).
//  spin 0 : lam_l = al * x * lam_{l-1} - bl * lam_{l-2}
//  spin 2 : lp_l = a x lp_{l-1} + ac lm_{l-1} - b lp_{l-2}
//           lm_l = a x lm_{l-1} + ac lp_{l-1} - b lm_{l-2}
// with lp/lm = (2lambda +- -2lambda)/2 and a, ac, b taken at the source l-1;
// the kernels run the equivalent separate recurrences of 2lambda = lp + lm
// (coefficient a x + ac) and -2lambda = lp - lm (a x - ac).
struct RecCoef {
  double al, bl, a, ac, b, pad;
};

// Device-side solver state of one RHS.
struct SolveState {
  int level;          // current cooling level
  int iter_in_level;  // iterations done at this level
  int iters_total;
  int done;           // 1 once the last level met its stopping rule
  int first;          // 1 before the first iteration (t_0 = d)
  int notconv;        // 1 when max_iter was hit
  double cauchy;      // last Cauchy ratio
  int iters_per_level[DM_MAX_LEVELS];
};

// Rings of one launch of the ring kernel: ring_order[off .. off + count) with
// FFT sizes up to M and ring lengths up to n.
struct RingClass {
  int off, count;
  int M, n;
  int poff, pcount;  // pair_order[poff .. poff + pcount): the northern (or equatorial) rings of the class
};

struct LevelDev {
  int n_levels;
  int max_iter;
  int forced;                         // 1: fixed counts per level
  int fixed_iters[DM_MAX_LEVELS];     // counts when forced
  double eps[DM_MAX_LEVELS];
};

}  // namespace dmwf

struct dm_plan {
  int device = 0;
  int nside = 0, lmax = 0, mmax = 0, batch = 0;
  int64_t npix = 0, nalm = 0;
  int nrings = 0, npairs = 0;
  int fft_M_max = 1;            // largest FFT size over rings
  // flat-sky plans (dm_plan_create_flat, the paper's own setting): rows of an
  // N x N grid are the rings; harmonic modes (kx < N/2, all ky) replace (l, m)
  bool flat = false;
  int flatN = 0;
  double flatL = 0.0;           // side of the patch in radians
  int64_t nmodes = 0;           // N / 2 x N stored modes
  dm_precision prec = DM_FP64;
  std::string err;

  // host copies
  std::vector<dmwf::RingDev> rings_h;
  std::vector<double> cl_h;     // [4][lmax+1]
  bool have_cl = false, have_noise = false;
  bool cov = false;             // correlated 3x3 noise (dm_set_noise_cov), plan-wide
  double *wcov = nullptr;       // [npix][6] W = alpha N^{-1} (xx, yy, zz, xy, xz, yz)
  double *covdraw = nullptr;    // [npix][9] noise draw matrix of constrained realisations (correlated noise)
  std::vector<double> alpha, t_h;   // per RHS: alpha = min N (observed), T_h = alpha Omega

  // schedule
  dm_schedule sched{};
  std::vector<int> forced;      // empty = not forced
  std::vector<double> lambdas;  // per level

  // device tables
  dmwf::RingDev *rings = nullptr;
  dmwf::PairDev *pairs = nullptr;
  double2 *phase = nullptr;     // e^{-i pi q / n} tables
  double2 *bhat = nullptr;      // Bluestein kernel spectra
  double2 *bhatT[2] = {nullptr, nullptr};  // the same transposed for the fixed-size kernels of radix 8, 16
  double2 *chirp = nullptr;     // Bluestein chirps, one table per ring radius
  int64_t ch_total = 0;
  double2 *twid = nullptr;      // stage twiddles: [len - 1 + j] = e^{-i pi j / len}, fft_M_max - 1 entries
  double2 *twr = nullptr;       // pass tables of the fixed-size transforms, M = 2^9 .. 2^12, radix 8 and 16
  int twr_off[2][16] = {{-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1}};  // [LR - 3][LOGM]: offset in twr (-1: not built)
  int twr_words = 0;
  int ring_lr = 3;              // radix 2^ring_lr of the fixed-size ring transforms (0: generic kernels)
  int *ring_order = nullptr;    // [nrings] ring ids grouped by FFT size class
  int *pair_order = nullptr;    // [npairs] the side-0 ring of each pair, grouped by class
  std::vector<int> pair_order_h;
  std::vector<int> ring_order_h;
  std::vector<dmwf::RingClass> ring_classes;
  dmwf::RecCoef *rec = nullptr; // [nalm]
  double *seed = nullptr;       // [mmax+1][npairs][3] : lambda_mm, lp, lm at l0 = max(m, 2)
  int *seed_exp = nullptr;      // [mmax+1][npairs] : scale S (true = v 2^-S), 0 = plain
  double *cl = nullptr;         // [4][lmax+1]
  double *filt = nullptr;       // [B][n_levels][lmax+1][4] per-RHS filters
  int filt_levels = 0;
  double *w = nullptr;          // [B][3][npix] alpha / N (0 masked), per RHS
  uint8_t *mask = nullptr;      // [B][npix]
  double *sigma = nullptr;      // [B][3][npix]

  // workspace (per batch)
  double2 *rc = nullptr;        // [B][3][mmax+1][npairs][2] ring coefficients
  double2 *a = nullptr;         // [B][3][nalm] harmonic iterate
  double2 *apart = nullptr;     // [B][nchunk][3][nalm] analysis partial sums
  int nchunk = 0;               // pair chunks of the analysis
  int nslot = 0;                // chunk slots of apart per RHS (nslot < nchunk: the analysis runs in waves)
  int nchunk32 = 0;             // chunks of apart32 per RHS: nchunk, or 1 (tensor-core analysis only) when that is over 24 GiB
  double *wd = nullptr;         // [B][3][npix] w * d
  double *norms = nullptr;      // [B][3][nrings][2] Cauchy partial sums
  dmwf::SolveState *state = nullptr;   // [B]
  dmwf::LevelDev *lev = nullptr;         // [B] per-RHS stopping schedule
  std::vector<double> eps_final_rhs;     // per RHS (serving sets it per request)
  double *tmpmap = nullptr;     // [B][3][npix] scratch map (CR, host-buffer entry)
  double *tmpmap2 = nullptr;    // [B][3][npix] scratch map
  double2 *tmpalm = nullptr;    // [B][3][nalm] scratch alm (CR)
  uint64_t *seeds_dev = nullptr;  // [B]
  double *coef_tmp = nullptr;   // [lmax+1][4] filter of dm_apply_filter
  bool state_active = false;    // kernels consult state[] (skip finished RHS)
  int64_t bytes = 0;
  // DM_MIXED_FP32 resources (allocated by dm_set_precision)
  bool fp32_ready = false;      // the buffers of the FP32 modes exist (setup_fp32 succeeded)
  // Full FP32 tables: built on first use by the kernels that read them (the
  // CUDA-core FP32 Legendre stages and the stored-table tensor-core tiles).
  // The float-float stages read them when present and otherwise generate
  // them per slab of orders m into ffs / ffs_lo.
  float *ptab = nullptr;        // [3][nalm][npairs] lambda, lam+, lam- in FP32 (FP64 recurrence)
  float *ptab_lo = nullptr;     // [3][nalm][npairs] FP64 value - ptab: float-float tables
  float *ffs = nullptr, *ffs_lo = nullptr;  // slab tables of the float-float stages
  std::vector<int> ffs_m;       // slab boundaries in m (first orders, then mmax + 1)
  int64_t ffs_cap = (int64_t)1 << 30;  // bytes of the largest slab (hi and lo)
  bool ffs_cap_set = false;     // dm_set_ff_slab_bytes was called: slabs of that size, no full tables
  bool ff_legendre = false;     // DM_FLOAT_FLOAT: Legendre stages in float-float
  bool anchor_ff = true;        // mixed-mode anchors in float-float (else FP64)
  bool ff_now = false;          // inside a float-float anchor
  float2 *rc32 = nullptr;       // [B][3][mmax+1][npairs][2]
  float2 *apart32 = nullptr;    // [B][nchunk][3][nalm]
  float *s32 = nullptr;         // [B][3][npix] iteration map
  float *w32 = nullptr;         // [B][3][npix]
  float *wd32 = nullptr;        // [B][3][npix]
  float2 *phase32 = nullptr, *bhat32 = nullptr, *twid32 = nullptr, *twr32 = nullptr, *chirp32 = nullptr;
  float2 *bhatT32[2] = {nullptr, nullptr};
  // FP64 anchor of the mixed iteration (iterative refinement):
  //   a = a_hi + e;  FP32 stages act on e only; g_hi = A W (d - Y a_hi) in FP64
  double2 *a_hi = nullptr;      // [B][3][nalm]
  double2 *g_hi = nullptr;      // [B][3][nalm]
  // FP32 iteration state between anchors: e = a - a_hi, updated as
  //   e <- c + F (e + Omega A r),  c = F (a_hi + g_hi) - a_hi  (FP64-formed per level)
  float2 *e32 = nullptr;        // [B][3][nalm]
  float2 *c32 = nullptr;        // [B][3][nalm]
  int *clev = nullptr;          // [B] level at which c was formed
  float *filt32 = nullptr;      // FP32 copy of filt
  float *shi32 = nullptr;       // [B][3][npix] Y a_hi rounded to FP32 (for ||s||)
  bool anchor_active = false;
  int anchor_every = 256;
  bool use_tc = true;           // tcgen05 Legendre stages when the batch allows
  int *tc_err = nullptr;        // device flag: a bounded tensor-core wait gave up
  int tc_withhold = 0;          // test hook: one withheld arrival in the spin-0 analysis (dm_test_tc_withhold)
  // tiled BF16 hi/lo copies of ptab for the tensor-core stages ([0] = lambda, [1] = lam+/lam-)
  unsigned char *tc_synA[2] = {nullptr, nullptr}, *tc_anaA[2] = {nullptr, nullptr};
  int64_t *tc_soff = nullptr, *tc_aoff = nullptr;  // block offsets per m / per (m, parity)
  unsigned char *tc_synB[2] = {nullptr, nullptr};   // per-iteration synthesis B operand tiles
  // tensor-core Legendre tiles generated in the kernels (dm_legendre_otf.cu):
  // FP32 recurrence from FP32 checkpoints of the FP64 recurrence, one per
  // (m, block of 64 multipoles, ring pair), instead of the stored tables
  int tc_gen = -1;              // 1: generate the tiles in the kernels; 0: stream the stored tables; -1: auto
  int tc_gen_used = -1;         // the resolved choice (tc_generate)
  float4 *ck0 = nullptr;        // [nck][npairs] (lambda_l, lambda_l-1 or D_l, S0, S2): S as int bits, value x 2^-S
  float4 *ck2 = nullptr;        // [nck][npairs] (2lam_l, 2lam_l-1 or D, -2lam_l, -2lam_l-1 or D) / 2, x 2^-S2
  int64_t *cko = nullptr;       // [mmax + 2] first checkpoint block of each m
  float4 *rq0 = nullptr;        // [nalm] FP32 spin-0 coefficients of target l (al, bl, al - 1 - bl, 0)
  float4 *rq2 = nullptr;        // [nalm] FP32 spin-2 coefficients (a, ac, b, 0)
  float2 *rq2d = nullptr;       // [nalm] (a + ac - 1 - b, a - ac - 1 - b) for the difference form of target l
  // solve session (dm_solve_begin / iterate / end)
  double *s64 = nullptr;        // [B][3][npix] FP64 iterate s (FP64 mode) / Y a_hi (mixed)
  double *rhi = nullptr;        // [B][3][npix] FP64 anchor residual w (d - Y a_hi)
  bool session = false;
  int since_anchor = 0;
  int64_t iters_launched = 0;
  int64_t bh_total = 0, ph_total = 0;
  // launch tuning (dm_tune.cu): per ring-size class the radix and lanes per
  // block, per tensor-core kernel its pipeline depth and tiles; 0 or -1 = the
  // built-in heuristic.  tune_only_* restrict a stage call to one launch while
  // the tuner times it.
  int tune_ring_lr[DM_TUNE_MAX_CLASSES];   // -1: the plan's ring_lr
  int tune_ring_G[DM_TUNE_MAX_CLASSES];    // 0: heuristic lanes per block
  int ring_G_used[DM_TUNE_MAX_CLASSES];    // what the last iteration launch used
  int ring_lr_used[DM_TUNE_MAX_CLASSES];
  int tune_ring_fuse[DM_TUNE_MAX_CLASSES];  // fixed-size kernels: 1 fused update pass, 0 separate (default),
                                            // 2 separate with the register-capped radix-16 kernels
  int ring_fuse_used[DM_TUNE_MAX_CLASSES];
  int tune_syn_ns[2] = {0, 0};             // k_syn_tc<PART> stages
  int tune_ana_lt[2] = {0, 0};             // k_ana_tc<PART> l tiles per CTA
  int tune_ana_S[2] = {0, 0};              // k_ana_tc<PART> stages
  int syn_ns_used[2] = {0, 0}, ana_lt_used[2] = {0, 0}, ana_S_used[2] = {0, 0};
  int tune_only_class = -1, tune_only_part = -1;
  bool tuned = false;
  dm_tuning tuning{};
  // progressive working resolution (dm_prog.cu)
  double prog_margin = 0.0;     // > 0: each level at the resolution its l_iter needs
  int prog_lmin = 8;
  std::vector<void *> prog_levels;   // plans of the coarse resolutions (made on first use)
  std::vector<int> prog_counts;      // [B][n_levels] counts of the last progressive solve
  std::vector<int> prog_res;         // [n_levels][2] (nside_k, L_k) of the last progressive solve
  bool prog_notconv = false;
  double lambda_single = 0.0;   // > 0: the lambda of a one-level schedule (a level plan's mu)
  std::vector<double> sigma_h;  // host copy of the plan-wide noise (dm_set_noise_mask)
  std::vector<uint8_t> mask_h;
  bool noise_shared = false;    // every RHS has the plan-wide diagonal noise
  // modified Jacobi refinement (dm_jacobi.cu)
  double2 *jsrc = nullptr;      // [B][3][nalm] harmonic source g of a W~ run
  double2 *jacc = nullptr;      // [B][3][nalm] the refined iterate
  bool src_active = false;      // the iteration adds jsrc before the filter
  // end-of-solve diagnostics (dm_diag.cu): true residual and chi^2 in FP64
  bool diag_on = true;
  double *diag_tab = nullptr;   // [lmax+1][DIAG_TAB_W]: C^1/2, C^+ and range projector per l (tt, te, ee, bb)
  double2 *diag_alm = nullptr;  // [B][3][nalm] analysis of w d, then of w (d - Y a)
  double *diag_part = nullptr;  // per-block partial sums
  double *diag_ao = nullptr;    // [B] alpha Omega
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // ms_total of a solve
  // measurement
  bool prof_on = false;
  dm_profile prof{};
  std::vector<cudaEvent_t> ev;  // 6 per iteration of one poll window
  int64_t launches = 0;
};

namespace dmwf {

// ---- launchers (stream-ordered; return cudaGetLastError()) ----
cudaError_t build_tables(dm_plan *p);                        // geometry, phases, chirps, coefficients, seeds
cudaError_t build_tables_flat(dm_plan *p);                   // rows of a flat N x N grid as rings
cudaError_t build_filter_table(const double *cl4, int64_t n, double mu, double th, double *coef,
                               cudaStream_t st);             // per-index filters of spectra cl4[4][n]
dm_status plan_workspace(dm_plan *p, dm_plan **out);         // dm_api.cu: workspace of a built plan
// flat-sky harmonic stages (dm_flat.cu)
cudaError_t flat_synthesis(dm_plan *p, const double2 *alm, cudaStream_t st);
cudaError_t flat_analysis(dm_plan *p, int epilogue, double2 *out, cudaStream_t st, cudaEvent_t mid);
cudaError_t build_filters(dm_plan *p, int b, cudaStream_t st);  // per-level filters of RHS b
cudaError_t build_noise(dm_plan *p, int b, cudaStream_t st);    // alpha (reduction) and w of RHS b

// ring stage: mode
enum RingMode { RING_FWD_MAP = 0, RING_INV_MAP = 1, RING_ITER = 2, RING_INIT = 3 };
cudaError_t ring_stage(dm_plan *p, int mode, const double *in_map, double *out_map, cudaStream_t st);
// lanes per block of the ring kernel (1..4) for the given shared-memory words
int ring_lanes_per_block(size_t word_bytes, int tw_words, int ph_words, int lane_words, int nlanes, int regs,
                         int nt);
// public-layout permutations of the ring coefficients
cudaError_t rc_to_public(dm_plan *p, double2 *pub, cudaStream_t st);
cudaError_t rc_from_public(dm_plan *p, const double2 *pub, cudaStream_t st);

// Legendre stages on the plan's rc buffer
cudaError_t legendre_synthesis(dm_plan *p, const double2 *alm, cudaStream_t st);
// analysis into apart, then reduce: out = (accumulate ? a_prev : 0) + Omega sum, then filter
enum AnaEpilogue {
  ANA_PLAIN = 0,
  ANA_DM_STEP = 1,
  ANA_FLAT_DRAW = 2  // flat sky only: the constrained-realisation signal draw (dm_flat.cu)
};
cudaError_t legendre_analysis(dm_plan *p, int epilogue, double2 *out, cudaStream_t st, cudaEvent_t mid = nullptr);
cudaError_t apply_filter_level(dm_plan *p, const double *coef, const double2 *in, double2 *out, cudaStream_t st);
cudaError_t build_filter_one(dm_plan *p, double lambda, double th, double *coef, cudaStream_t st);

// solver control
cudaError_t control_init(dm_plan *p, cudaStream_t st);
cudaError_t control_step(dm_plan *p, cudaStream_t st);
cudaError_t prepare_wd(dm_plan *p, const double *d, cudaStream_t st);
cudaError_t cov_prepare_wd(dm_plan *p, const double *d, cudaStream_t st);  // dm_cov.cu
cudaError_t cov_ring_stage(dm_plan *p, cudaStream_t st);
cudaError_t cov_ring_stage32(dm_plan *p, cudaStream_t st);      // the mixed mode's (FP32 state)
cudaError_t anchor_residual_wd_cov(dm_plan *p, const double *s_hi, cudaStream_t st);
cudaError_t setup_fp32(dm_plan *p);
cudaError_t ensure_ptab(dm_plan *p);  // the full FP32 tables, built on first use
// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`, never lowering it.  The limit is a process-wide attribute of
// the function: set per launch, a smaller value set by a plan on another host
// thread between this thread's set and launch would fail the launch; raised
// monotonically under a lock, every launch of at most the granted size holds.
cudaError_t dyn_smem_allow_fn(const void *func, size_t bytes);
template <typename F>
inline cudaError_t dyn_smem_allow(F *func, size_t bytes) {
  return dyn_smem_allow_fn((const void *)func, bytes);
}
// first alm index of order m (m = mmax + 1 = lmax + 1 gives nalm): idx(l, m) = start(m) + l - m
inline int64_t alm_start_h(int lmax, int m) { return (int64_t)m * (2 * lmax + 3 - m) / 2; }
cudaError_t gen_tables32_slab(dm_plan *p, float *hi, float *lo, int m0, int m1, cudaStream_t st);                          // tables and buffers of DM_MIXED_FP32
cudaError_t copy_s32_to_user(dm_plan *p, double *s_out, cudaStream_t st);
// anchor residual: r = w (d - s_hi) (or d on observed pixels when s_hi == nullptr),
// written to p->wd; shi32 = s_hi in FP32
cudaError_t anchor_residual(dm_plan *p, const double *d, const double *s_hi, cudaStream_t st);
cudaError_t anchor_residual_wd(dm_plan *p, const double *s_hi, cudaStream_t st);  // r = wd - w s_hi

// tensor-core Legendre stages (dm_legendre_tc.cu)
bool tc_batch_ok(int B);
size_t tc_table_bytes(int lmax, int mmax, int npairs, int B);
cudaError_t legendre_synthesis_tc(dm_plan *p, const double2 *alm, cudaStream_t st);
cudaError_t legendre_analysis_tc(dm_plan *p, cudaStream_t st);
// tensor-core stages with the Legendre tiles generated in the kernels (dm_legendre_otf.cu)
cudaError_t gen_setup(dm_plan *p);
bool tc_tables_fit(int lmax, int mmax, int npairs, int B);  // auto rule: stored tiles when they fit
bool tc_generate(dm_plan *p);                               // the plan's resolved choice
size_t gen_bytes(int lmax, int mmax, int npairs);
cudaError_t syn_gen_launch(dm_plan *p, bool run0, bool run1, cudaStream_t st);
cudaError_t ana_gen_launch(dm_plan *p, cudaStream_t st);
cudaError_t legendre_synthesis_ff(dm_plan *p, const double2 *alm, cudaStream_t st);
cudaError_t anchor_c32(dm_plan *p, cudaStream_t st);     // c = F (a_hi + g_hi) - a_hi, e = 0
cudaError_t materialize_a(dm_plan *p, cudaStream_t st);  // a = a_hi + e
cudaError_t legendre_analysis_ff_parts(dm_plan *p, cudaStream_t st, int *used);
cudaError_t fold_slots(dm_plan *p, int nused, int m0, int m1, cudaStream_t st);
// Partial sums of the FP64-class analysis over every pair chunk into apart,
// in waves of at most nslot chunks when the plan holds fewer slots than
// chunks: slot 0 keeps the running sum, each later wave fills slots 1 ..
// and is folded into it.  launch(c0, slot0, n, m0, m1) runs the chunks
// [c0, c0 + n) into the slots [slot0, slot0 + n) for the orders [m0, m1).
// Returns the slots that hold the orders' sum (nchunk without waves, else 1).
template <class F>
inline cudaError_t chunk_waves(dm_plan *p, int m0, int m1, cudaStream_t st, F launch, int *used_out) {
  if (p->nslot >= p->nchunk) {
    *used_out = p->nchunk;
    return launch(0, 0, p->nchunk, m0, m1);
  }
  int c0 = 0, used = 0;
  while (c0 < p->nchunk) {
    const int slot0 = used == 0 ? 0 : 1;
    const int n = std::min(p->nslot - slot0, p->nchunk - c0);
    if (cudaError_t e = launch(c0, slot0, n, m0, m1)) return e;
    c0 += n;
    used = slot0 + n;
    if (cudaError_t e = fold_slots(p, used, m0, m1, st)) return e;
    used = 1;
  }
  *used_out = 1;
  return cudaSuccess;
}


// driver (dm_api.cu), shared with the server (dm_serve.cu)
dm_status upload_levels(dm_plan *p);
cudaError_t enqueue_iteration(dm_plan *p, cudaStream_t st, cudaEvent_t *E);
dm_status anchor(dm_plan *p, cudaStream_t st, bool initial, const double *d, bool need_g);
dm_status solve_begin(dm_plan *p, const double *d, cudaStream_t st);
dm_status solve_iterate(dm_plan *p, long max_iters, int *all_done, cudaStream_t st);
dm_status solve_end(dm_plan *p, double *s_out, double *alm_out, cudaStream_t st, bool to_host);
dm_status run_dm(dm_plan *p, const double *d, cudaStream_t st);

// constrained realisations
cudaError_t draw_signal(dm_plan *p, const uint64_t *seeds_dev, double2 *ahat, cudaStream_t st);
cudaError_t draw_white_maps(dm_plan *p, const uint64_t *seeds_dev, double *z, cudaStream_t st);
cudaError_t flat_draw_signal(dm_plan *p, const uint64_t *seeds_dev, double2 *ahat, cudaStream_t st);
cudaError_t draw_noise_add(dm_plan *p, const uint64_t *seeds_dev, const double *shat, double *dhat,
                           cudaStream_t st);
cudaError_t axpy_maps(int64_t n, const double *x, double alpha, double *y, cudaStream_t st);

// progressive working resolution (dm_prog.cu)
dm_status solve_begin_warm(dm_plan *p, const double *d, cudaStream_t st);
dm_status run_progressive(dm_plan *p, const double *d, cudaStream_t st);
void prog_release(dm_plan *p);

// modified Jacobi refinement (dm_jacobi.cu)
cudaError_t jacobi_alloc(dm_plan *p);
cudaError_t jacobi_source(dm_plan *p, const double *d, cudaStream_t st);  // jsrc = P g(jacc)
cudaError_t jacobi_final(dm_plan *p, const double *d, cudaStream_t st);   // s64 = Y a, wd = w d

// launch autotuner (dm_tune.cu)
dm_status autotune(dm_plan *p, cudaStream_t st, std::string &err);

dm_status upload_levels_counts(dm_plan *p, const std::vector<int> &counts);  // per-RHS forced counts [B][n_levels]

// progressive working resolution (dm_prog.cu)
dm_status solve_begin_warm(dm_plan *p, const double *d, cudaStream_t st);
dm_status run_progressive(dm_plan *p, const double *d, cudaStream_t st);
void prog_release(dm_plan *p);

// modified Jacobi refinement (dm_jacobi.cu)
cudaError_t jacobi_alloc(dm_plan *p);
cudaError_t jacobi_source(dm_plan *p, const double *d, cudaStream_t st);  // jsrc = P g(jacc)
cudaError_t jacobi_final(dm_plan *p, const double *d, cudaStream_t st);   // s64 = Y a, wd = w d

// launch autotuner (dm_tune.cu)
dm_status autotune(dm_plan *p, cudaStream_t st, std::string &err);

// end-of-solve diagnostics (dm_diag.cu)
cudaError_t diag_tables(dm_plan *p);
cudaError_t diag_tables_flat(dm_plan *p, const std::vector<double> &cl);  // per mode, cl[4][nmodes]
cudaError_t diagnostics(dm_plan *p, cudaStream_t st, std::vector<double> &resid, std::vector<double> &chi2);

}  // namespace dmwf
