/*
 * dmwf.h -- C ABI of the GB300 (sm_103a) dual messenger Wiener filter for joint
 * T/Q/U CMB maps on the HEALPix sphere.
 *
 * Method: Kodi Ramanah, Lavaux & Wandelt, "Optimal and fast E/B separation with
 * a dual messenger field" (arXiv:1801.05358), Section 2 and Algorithm 1; the
 * constrained realisations of Section 2.2.  The paper is flat-sky; this library
 * carries it onto the HEALPix sphere with spin-0 and spin-2 harmonic transforms.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pixelisation: HEALPix RING order, npix = 12 nside^2, rings 1..4nside-1.
 *  - Maps: [batch][3][npix] float64, components I (T), Q, U.
 *  - Harmonic coefficients: [batch][3][nalm] complex128 (interleaved re, im),
 *    fields T, E, B, m-major: index(l, m) = m (2 lmax + 1 - m) / 2 + l,
 *    0 <= m <= l <= lmax, nalm = (lmax + 1)(lmax + 2) / 2.  Real fields: the
 *    m < 0 coefficients are a_{l,-m} = (-1)^m conj(a_lm) and are not stored.
 *  - Harmonics: Goldberg et al. (1967) spin-weighted harmonics
 *    sY_lm = sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi}; polarisation
 *    (Q + iU) = sum a_{2,lm} 2Y_lm, (Q - iU) = sum a_{-2,lm} -2Y_lm,
 *    a_{+-2} = -(a_E +- i a_B)  (the sphere form of Eqs. 12-16).
 *  - Synthesis Y: alm -> map.  Analysis A = Omega Y^dagger with
 *    Omega = 4 pi / npix (no ring weights).
 *  - Spectra: cl[4][lmax+1] float64 = C^TT, C^EE, C^BB, C^TE (Eq. 10).
 *  - Noise: diagonal N = sigma^2 per pixel and component; masked pixels have
 *    N^{-1} = 0 (Appendix B).  T = alpha 1 with alpha = min N over observed
 *    pixel-components (Section 2), w = alpha / N.
 *  - Device pointers are CUDA device addresses on the plan's device; `stream`
 *    is a cudaStream_t (NULL = legacy default stream).  Calls are ordered on
 *    that stream; a call returns once its work is enqueued unless it says it
 *    synchronises.  The caller owns every buffer it passes; the plan owns its
 *    workspace.  A plan is not thread-safe: one host thread at a time.
 *    Distinct plans may be driven from different host threads at once, each
 *    on its own stream.
 *
 * Errors: every call returns a dm_status.  DM_EINVAL for bad arguments (the
 * plan is left unchanged), DM_ECUDA for a CUDA failure, DM_ENOMEM when device
 * memory runs out, DM_ENOTCONV when max_iter was reached before the last level
 * converged (the last iterate is still written).  dm_last_error() returns a
 * message for the last failure on that plan.
 */
#ifndef DMWF_H
#define DMWF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dm_plan dm_plan;

typedef enum {
  DM_OK = 0,
  DM_EINVAL = 1,
  DM_ENOMEM = 2,
  DM_ECUDA = 3,
  DM_ENOTCONV = 4,
  DM_ETIMEOUT = 5,
  DM_EAGAIN = 6,
  DM_EBUSY = 7
} dm_status;

/* Arithmetic of the Legendre contraction and of map storage.
 * DM_FP64: everything in FP64.
 * DM_MIXED_FP32: FP64 recurrence (Legendre/Wigner values generated in FP64),
 *   FP32 contraction, FP32 ring FFTs and maps on the device; FP64 per-l 3x3
 *   filter, FP64 harmonic state and FP64 convergence norms.
 * DM_FLOAT_FLOAT: the FP64 path with the two Legendre stages computed in
 *   float-float arithmetic (pairs of FP32 numbers, about 48 significant bits)
 *   from FP64-generated tables on the FP32 pipe: FP64-class results (relative
 *   error near 1e-13 per transform) at a fraction of the FP64 cost on GPUs
 *   whose FP64 rate is low.  Not in the paper (an arithmetic choice). */
typedef enum { DM_FP64 = 0, DM_MIXED_FP32 = 1, DM_FLOAT_FLOAT = 2 } dm_precision;

/* Cooling and stopping schedule of Algorithm 1 (Section 3.2).
 * Levels: lambda_k = xi_k / T_h = lambda0^(1 - k/(n_levels-1)), k = 0..n_levels-1,
 * the last level exactly 1 (mu = 0: the Wiener filter itself).
 * iters_per_level > 0: exactly that many iterations per level (no test).
 * Otherwise a level ends when ||s_i - s_{i-1}|| / ||s_i|| < eps_k with
 *   eta > 0 : eps_k = max(eps_final, eps0 * eta^-k), eps_final at the last level;
 *   eta == 0: eps_k = eps0 (eps_final/eps0)^(k/(n_levels-1)).
 * max_iter caps the total; check_every is how often (in iterations) the host
 * reads the device-side convergence state (>= 1). */
typedef struct {
  double lambda0;
  int n_levels;
  int iters_per_level;
  double eps0;
  double eps_final;
  double eta;
  int max_iter;
  int check_every;
} dm_schedule;

#define DM_MAX_LEVELS 64

/* Per-RHS statistics, valid after the call returns.
 * true_resid and chi2 are the paper's quality measures of the final iterate
 * (Section 3.2, Table 1; Appendix C), evaluated on the device in FP64-class
 * arithmetic (FP64, or float-float Legendre stages in DM_FLOAT_FLOAT and for
 * the mixed mode's float-float anchors):
 *  true_resid = ||A x - y|| / ||y||, A = 1 + S^1/2 Y^T N^-1 Y S^1/2,
 *               x = S^-1/2 a, y = S^1/2 Y^T N^-1 d  (with the analysis
 *               A = Omega Y^T standing in for Y^T, as in the iteration);
 *  chi2       = (d - s)^T N^-1 (d - s) + a^T S^+ a  (Eq. 3; observed
 *               pixel-components only, S^+ the per-l pseudo-inverse).
 * Under correlated noise (dm_set_noise_cov) N^-1 is the per-pixel 3 x 3 block
 * on the observed components.  On flat-sky plans S is the per-mode block
 * (<|a_l|^2> = L^2 S) and Omega the pixel area.  Both are NaN when
 * dm_set_diagnostics turned them off.  For a constrained realisation they describe its
 * Wiener-filter solve W(d - dhat).  ms_total is the device time of the call
 * (or from dm_solve_begin to dm_solve_end), diagnostics excluded. */
typedef struct {
  int iters_total;
  int levels_done;
  int iters_per_level[DM_MAX_LEVELS];
  double cauchy_final;
  double true_resid;
  double chi2;
  float ms_total;
} dm_stats;

/* --- plan ------------------------------------------------------------------ */

/* Create a plan for `batch` right-hand sides of one geometry on the current
 * CUDA device.  1 <= nside <= 2048 (a power of two is not required),
 * 2 <= lmax <= 4 nside, 1 <= batch <= 4096, and above nside 1024 at most
 * 2^31 - 1 pixel-components per plan (batch x 3 x 12 nside^2; nside 2048
 * allows 14 RHS).  The mixed and float-float modes also need their FP32
 * hi/lo tables (3 x nalm x 2 nside x 8 bytes) to fit.  Builds the ring geometry, the
 * FFT chirps, the recurrence coefficient and seed tables, and allocates the
 * workspace (DM_ENOMEM if it does not fit). */
dm_status dm_plan_create(int nside, int lmax, int batch, dm_plan **out);
void dm_plan_destroy(dm_plan *plan);
const char *dm_last_error(const dm_plan *plan);
/* Sizes of the plan: npix, nalm, nrings, device bytes held. */
dm_status dm_plan_info(const dm_plan *plan, int64_t *npix, int64_t *nalm, int *nrings, int64_t *workspace_bytes);

/* Arithmetic mode (default DM_FP64); DM_EBUSY while a solve is in progress. */
dm_status dm_set_precision(dm_plan *plan, dm_precision prec);

/* Signal covariance, Eq. 10: host array cl[4][lmax+1] (TT, EE, BB, TE).
 * Each per-l TE block must be positive semi-definite (DM_EINVAL otherwise).
 * DM_EBUSY while a solve is in progress. */
dm_status dm_set_spectra(dm_plan *plan, const double *cl);

/* Noise and mask (shared by every RHS of the plan), host arrays:
 * sigma[3][npix] per-pixel noise std-dev of I, Q, U (> 0 and finite on
 * observed pixels); mask[npix], 1 = observed, 0 = masked; NULL = full sky.
 * Computes alpha = min sigma^2 over observed pixel-components, T_h = alpha
 * Omega and w = alpha / sigma^2 on the device. */
dm_status dm_set_noise_mask(dm_plan *plan, const double *sigma, const uint8_t *mask);

/* Noise and mask of one RHS b (same layout as dm_set_noise_mask), after the
 * plan-wide call; alpha, T_h, w and the per-level filters of that RHS follow
 * it.  DM_EBUSY while a solve is in progress. */
dm_status dm_set_noise_mask_rhs(dm_plan *plan, int b, const double *sigma, const uint8_t *mask);

/* Correlated noise with distinct temperature and polarisation masks, for every
 * RHS of the plan (the 3x3 per-pixel noise covariance of Section 2.1 and
 * Appendix B).  sigma: host [3][npix] (I, Q, U) amplitudes; rho: host [3][npix]
 * correlations (rho_IQ, rho_IU, rho_QU), N = Sigma C Sigma with C the
 * unit-diagonal correlation matrix; mask_t: host [npix], 1 = temperature
 * observed (NULL = all); mask_p: the same for Q and U.  Masked components
 * carry Sigma^{-1} = 0 (Appendix B).  alpha is the smallest eigenvalue of N
 * over the observed components, and the messenger update is Appendix B's
 * t = (Nbar^{-1} + T^{-1})^{-1} (T^{-1} s + Nbar^{-1} d), applied as
 * s + alpha N^{-1} (d - s).  Copied at the call.  Solves then run in DM_FP64
 * or DM_FLOAT_FLOAT (DM_EINVAL in DM_MIXED_FP32 at dm_solve_begin); per-RHS
 * noise returns DM_EINVAL.  Constrained realisations draw the noise whose
 * covariance the solve's precision inverts (Eq. 18): Sigma L z with C = L L^T
 * on fully observed pixels, and on partly masked ones the draw conditioned
 * on zero noise on the masked components (x_o - C_om C_mm^{-1} x_m), from the
 * unit normals described at dm_draw_cr_inputs.
 * dm_set_noise_mask returns the plan to diagonal noise.  DM_EINVAL for a
 * correlation matrix that is not positive definite, sigma <= 0 or non-finite
 * on an observed component, or no observed component; DM_EBUSY during a
 * solve. */
dm_status dm_set_noise_cov(dm_plan *plan, const double *sigma, const double *rho, const uint8_t *mask_t,
                           const uint8_t *mask_p);

/* Schedule (defaults: lambda0 1000, 10 levels, 10 iterations per level).
 * DM_EBUSY while a solve is in progress. */
dm_status dm_set_schedule(dm_plan *plan, const dm_schedule *sched);

/* Force the per-level iteration counts (length n_levels of the schedule),
 * overriding iters_per_level and the Cauchy test; NULL clears it.  Used to
 * replay a recorded run.  DM_EBUSY while a solve is in progress. */
dm_status dm_set_forced_iters(dm_plan *plan, const int *iters);

/* --- the hot path -------------------------------------------------------- */

/* Wiener filter by the dual messenger iteration (Algorithm 1).
 * d: device [batch][3][npix] data maps (masked pixels ignored).
 * s_out: device [batch][3][npix] Wiener-filtered maps (s = Y a).
 * alm_out: device [batch][3][nalm] complex128 or NULL.
 * stats: host [batch] or NULL.  Synchronises the stream before returning. */
dm_status dm_wiener_filter(dm_plan *plan, const double *d, double *s_out, double *alm_out,
                           dm_stats *stats, void *stream);

/* Same, with HOST buffers (pinned memory recommended): copies d in, runs,
 * copies s_out (and alm_out if non-NULL) back. */
dm_status dm_wiener_filter_host(dm_plan *plan, const double *d_host, double *s_host, double *alm_host,
                                dm_stats *stats, void *stream);

/* The same solve in three calls, so that a caller can advance it in pieces
 * (serving, checkpointed runs, steady-state timing):
 *  dm_solve_begin   sets s_0 = 0, t_0 = d (d must stay valid until the call
 *                   returns; the plan keeps w d and its own iterate);
 *  dm_solve_iterate runs up to max_iters iterations, stops early once every
 *                   RHS met its stopping rule (*all_done = 1); synchronises;
 *  dm_solve_end     writes s_out / alm_out (device, may be NULL) and stats.
 * DM_EBUSY when a solve is already in progress on the plan.  A solve that
 * fails (a CUDA error, DM_ETIMEOUT) ends its session, in these calls and in
 * dm_wiener_filter / dm_constrained_realization, so the plan stays usable. */
dm_status dm_solve_begin(dm_plan *plan, const double *d, void *stream);
dm_status dm_solve_iterate(dm_plan *plan, int max_iters, int *all_done, void *stream);
dm_status dm_solve_end(dm_plan *plan, double *s_out, double *alm_out, dm_stats *stats, void *stream);

/* End-of-solve diagnostics (default on): with a non-NULL stats argument the
 * solve calls evaluate true_resid and chi2 of dm_stats, at the cost of two
 * FP64-class analyses and map reductions per call (Section 3.2, Appendix C).
 * 0 turns them off (the fields are then NaN). */
dm_status dm_set_diagnostics(dm_plan *plan, int on);

/* Mixed precision refinement: the FP32 stages act on the correction
 * e = a - a_hi around an FP64 anchor a_hi, and A W (d - Y a_hi) is recomputed
 * with the FP64 transforms every anchor_every iterations (default 256) and at
 * the end, so the iteration keeps the FP64 fixed point (classical mixed
 * precision iterative refinement; no counterpart in the paper). */
dm_status dm_set_refinement(dm_plan *plan, int anchor_every);

/* Arithmetic of those anchors: DM_FLOAT_FLOAT (default; FP64-class accuracy
 * on the FP32 pipe) or DM_FP64 (FP64 pipe); DM_EINVAL for other values. */
dm_status dm_set_anchor_precision(dm_plan *plan, dm_precision prec);

/* Tensor cores for the mixed-precision Legendre stages (default on): with a
 * batch of 8, 16, 32 or 64 RHS the contractions over l and over ring pairs
 * run as tcgen05 GEMMs with BF16 hi/lo split operands and FP32 accumulation
 * (three products per K step); other batches use the FP32 CUDA-core kernels.
 * A pipeline wait that gives up (after 1 s) makes the solve calls return
 * DM_ETIMEOUT; the single-stage calls (dm_alm2map, dm_legendre_synthesis, ...)
 * return without synchronising and do not check it.  Each solve starts with
 * the flag cleared. */
dm_status dm_set_tensor_cores(dm_plan *plan, int on);

/* Source of the tensor cores' Legendre operand (default -1: stored tiles when
 * they and the FP32 tables they are cut from take at most 40 GiB, as at
 * nside 512 / lmax 1024 (26 GB), else generated tiles).
 * 1: the kernels generate each tile from checkpoints of the FP64 recurrence
 *    (the state at every 64th multipole of each (m, ring pair), stored in
 *    FP32 with a power-of-two scale: 32 bytes per checkpoint, about 150 MB at
 *    nside 512 / lmax 1024) and advance it in FP32 with a float-float
 *    product by cos(theta), the Legendre functions' recurrence in l of
 *    Section 2.3 run inside the contraction;
 * 0: they stream tiles of stored BF16 hi/lo tables (16 GB at nside 512 /
 *    lmax 1024), built on first use.
 * Both give the same products to within the BF16 hi/lo rounding.  Without
 * stored tiles the plan keeps no full FP32 tables either: the float-float
 * anchors generate theirs per slab of orders (1 GiB).  DM_EINVAL for a null
 * plan, DM_EBUSY during a solve session. */
dm_status dm_set_tc_tiles(dm_plan *plan, int generate);

/* Memory for the float-float stages' per-slab Legendre tables, used when the
 * plan has no full FP32 tables (DM_FLOAT_FLOAT, and DM_MIXED_FP32's anchors
 * with generated tiles): each stage call generates the tables of one slab of
 * orders m (FP64 recurrence, hi and lo in FP32) and contracts it before the
 * next.  bytes: the largest slab (default 1 GiB; at least one order m is
 * always taken).  By default a plan keeps the full tables instead when they
 * fit in one slab, and in DM_FLOAT_FLOAT when they take at most 32 GiB;
 * after this call only the first rule applies.  Takes effect at the next stage call; DM_EINVAL for a null
 * plan or bytes < 1, DM_EBUSY during a solve session. */
dm_status dm_set_ff_slab_bytes(dm_plan *plan, int64_t bytes);

/* Memory for the partial sums of the FP64 and float-float analysis: one
 * slot per RHS and chunk of 64 ring pairs (3 nalm FP64 complex values).  By
 * default a plan holds every chunk while that takes at most 24 GiB, else as
 * many slots as fit in it (at least 2); with fewer slots than chunks the
 * analysis runs the chunks in waves, slot 0 keeping the running sum.  slots:
 * 2 .. chunks (clamped).  Reallocates the partial-sum buffer; DM_EINVAL for a
 * null plan or slots < 2, DM_EBUSY during a solve session. */
dm_status dm_set_analysis_slots(dm_plan *plan, int slots);

/* Tuning: the ring transforms of an iteration for rings whose FFT size M is a
 * power of two in [512, 4096] run as fixed-size kernels of radix 2^lr with
 * M / 2^lr threads per ring and (RHS, field) lane; lr = 3 (radix 8, the
 * default) or 4 (radix 16); lr = 0 selects the generic radix-2^2 kernels for
 * every size.  The results agree to rounding.  DM_EINVAL for other lr. */
dm_status dm_set_ring_radix(dm_plan *plan, int lr);

/* Constrained realisations, Section 2.2, Eq. 19:
 * s_CR = W(d - dhat) + shat with shat = Y ahat, ahat ~ S, dhat = shat + nhat,
 * nhat ~ N on observed pixels, drawn from seeds[batch] (host) with the
 * Philox4x32-10 generator described at dm_draw_cr_inputs.  One dual messenger
 * run per realisation.  Buffers as in dm_wiener_filter; s_cr_out device. */
dm_status dm_constrained_realization(dm_plan *plan, const double *d, const uint64_t *seeds,
                                     double *s_cr_out, double *alm_cr_out, dm_stats *stats, void *stream);

/* The random inputs of a constrained realisation (step a9), per RHS b with
 * key = (seed_b low 32 bits, seed_b high 32 bits):
 *  ahat: for alm index i, Philox counters (i, j, 0, 0), j = 0, 1, 2 give unit
 *   normals for T, E, B: two 53-bit uniforms u1 = words 0,1 and u2 = words 2,3
 *   ((hi >> 5) * 2^26 + (lo >> 6) + 0.5) * 2^-53, Box-Muller z0 = r cos(2 pi u2),
 *   z1 = r sin(2 pi u2), r = sqrt(-2 ln u1); re from z0, im from z1.  ahat = L z
 *   with L the Cholesky factor of [[TT, TE], [TE, EE]] and sqrt(BB); m = 0 real
 *   (full variance), m > 0 re and im each at half variance.
 *  nhat: for pixel p, counters (p, 0, 1, 0) -> (I, Q), (p, 1, 1, 0) -> (U, -),
 *   times sigma, zero on masked pixels (under dm_set_noise_cov these three
 *   normals z give the correlated draw described there, zero on masked
 *   components).
 * Outputs (device, any may be NULL): ahat [batch][3][nalm] complex128,
 * shat = Y ahat and dhat = (shat + nhat) on observed pixels, [batch][3][npix]. */
dm_status dm_draw_cr_inputs(dm_plan *plan, const uint64_t *seeds, double *ahat, double *shat, double *dhat,
                            void *stream);

/* Progressive working resolution (the speed-up proposed in Section 4, with
 * l_iter of Section 2): with margin > 0 the solve calls (dm_wiener_filter,
 * dm_wiener_filter_host, dm_constrained_realization) run each cooling level
 * k at the smallest resolution whose band limit stays a margin above that
 * level's l_iter: L_k = min(lmax, max(lmin, ceil((1 + margin) l_iter(mu_k)))),
 * l_iter(mu) the largest l whose TE block or BB has an eigenvalue above
 * mu_k = (lambda_k - 1) T_h, and nside_k the smallest power of two with
 * 2 nside_k >= L_k; the last level runs at full resolution.  A coarse level
 * sees per Stokes component the inverse-noise weighted mean of the observed
 * children of each coarse pixel (noise variance 1 / sum N^-1), its own alpha,
 * w and T_h, and the filter of threshold mu_k; the harmonic iterate carries
 * over between levels (modes above L_k dropped or zero) and the usual step
 * continues from it.  Each resolution gets a plan of the same batch and
 * precision, made on first use and kept until the spectra, noise or
 * arithmetic change.  Needs a power-of-two nside and plan-wide diagonal
 * noise (dm_set_noise_mask); stats report the count of every level.
 * margin = 0 (default) turns it off.  No counterpart in the paper's runs. */
dm_status dm_set_progressive(dm_plan *plan, double margin, int lmin);
/* (nside_k, L_k) of every level of the last progressive solve (host arrays of
 * the schedule's n_levels); DM_EINVAL before one ran. */
dm_status dm_get_progressive_levels(const dm_plan *plan, int *nside_k, int *lmax_k);

/* The modified Jacobi refinement of Appendix A after a Wiener-filter solve:
 * the usual solve of d (as dm_wiener_filter), then n_refine steps
 *   a <- a + W~(P g(a)),  g(a) = A(w (d - Y a)) - alpha Omega C^+ a,
 * where W~ is the dual messenger iteration at the per-level counts the solve
 * took (per RHS), driven by the harmonic source g instead of data (from
 * a = 0: a <- F_k [a + g - A(w Y a)]), C^+ the per-l pseudo-inverse of the
 * signal covariance and P the projector onto its range.  g vanishes at the
 * Wiener filter, so the refined solution converges to it for any counts.
 * Buffers as in dm_wiener_filter (d must stay valid until the call returns);
 * stats report iters_total = (1 + n_refine) x the solve's count and the
 * diagnostics of the refined a.  Diagonal noise only (DM_EINVAL under
 * dm_set_noise_cov).  Synchronises. */
dm_status dm_jacobi_refine(dm_plan *plan, const double *d, int n_refine, double *s_out, double *alm_out,
                           dm_stats *stats, void *stream);

/* --- transform stages (the steps of the iteration, exposed for testing) ---- */

/* Synthesis map = Y alm (Legendre synthesis + inverse ring FFT), device buffers. */
dm_status dm_alm2map(dm_plan *plan, const double *alm, double *map, void *stream);
/* Analysis alm = A map = Omega Y^dagger map (ring FFT + Legendre analysis). */
dm_status dm_map2alm(dm_plan *plan, const double *map, double *alm, void *stream);
/* Ring DFTs alone: rc[batch][3][nrings][lmax+1] complex128,
 * rc = sum_j f_j e^{-i m phi_j} per ring (forward); inverse is the real map
 * f_j = Re rc_0 + 2 sum_{m>0} Re(rc_m e^{i m phi_j}). */
dm_status dm_ring_fft_forward(dm_plan *plan, const double *map, double *rc, void *stream);
dm_status dm_ring_fft_inverse(dm_plan *plan, const double *rc, double *map, void *stream);
/* Legendre stages alone, rc in the layout above:
 * synthesis rc^T = sum_l aT lambda, rc^Q = -sum_l (aE lam+ + i aB lam-),
 * rc^U = -sum_l (aB lam+ - i aE lam-), lam+- = (2lambda +- -2lambda)/2;
 * analysis is its Omega-scaled adjoint (ring sums). */
dm_status dm_legendre_synthesis(dm_plan *plan, const double *alm, double *rc, void *stream);
dm_status dm_legendre_analysis(dm_plan *plan, const double *rc, double *alm, void *stream);
/* Per-l filter of level lambda (Eq. 8): alm_out = F alm_in with
 * F = V diag(f_e) V^T, f_e = max(S_e, mu)/(max(S_e, mu) + T_h), mu = (lambda-1) T_h. */
dm_status dm_apply_filter(dm_plan *plan, double lambda, const double *alm_in, double *alm_out, void *stream);
/* Allocation-free variant of dm_legendre_analysis (same inputs, same
 * outputs, FP64), for callers that must not allocate device memory at the
 * moment they call: work recorded into a CUDA graph by stream capture, a
 * real-time loop where cudaMalloc/cudaFree could synchronise the device, or
 * an application that fixes the library's device-memory budget at start-up.
 * The paper has no counterpart; this is a property of the library.
 * The per-chunk partial sums go to one file-scope device array of
 * 64 MiB (held on every GPU that loads the library until exit) instead of
 * the plan's workspace; plans needing more (batch x ceil(2 nside / 64) x 3 x
 * nalm x 16 bytes) get DM_EINVAL with a message.  The first call on each
 * device looks the array's address up (cudaGetSymbolAddress) with that device
 * current: make it before any stream capture.  The address is cached for the
 * life of the process: after cudaDeviceReset on a device, do not call this
 * entry point on that device again.  Calls share the array, so
 * calls that overlap on the GPU race and must be serialised by the caller;
 * every value the call reads from the array it wrote first, so nothing needs
 * clearing between calls.  No cudaMalloc, cudaFree or allocating library call
 * is made. */
dm_status dm_legendre_analysis_noalloc(dm_plan *plan, const double *rc, double *alm, void *stream);

/* --- launch tuning ----------------------------------------------------- */

#define DM_TUNE_MAX_CLASSES 12

/* Launch configuration of the iteration's kernels (no counterpart in the
 * paper; a property of this library).  Ring stage: one launch per FFT-size
 * class of rings (classes ordered by decreasing FFT size); per class the
 * radix of the fixed-size transforms (3: radix 8, 4: radix 16, 0: the generic
 * radix-4 kernels; classes whose size is not a power of two in [512, 4096]
 * always run the generic ones) and the (RHS, field) lanes per block.
 * Tensor-core stages (DM_MIXED_FP32 with 8, 16, 32 or 64 RHS): pipeline
 * stages of the spin-0 and spin-2 synthesis kernels, l tiles per CTA and
 * pipeline stages of the two analysis kernels.  A value of 0 (-1 for a
 * radix) means the built-in heuristic.  The ms_ fields report the stage time
 * per iteration of the pick and of the heuristic, as measured by
 * dm_autotune (0 when not measured). */
typedef struct {
  int n_ring_classes;
  int ring_radix_lr[DM_TUNE_MAX_CLASSES];
  int ring_lanes[DM_TUNE_MAX_CLASSES];
  int ring_fused[DM_TUNE_MAX_CLASSES];  /* fixed-size kernels: 1 = last inverse pass, messenger update and
                                           first forward pass fused in registers, 0 = separate passes,
                                           2 = separate passes with the FP32 radix-16 kernels of up to 2048
                                           points compiled for 80 registers a thread (three blocks of 256
                                           threads per SM; other launches take 0), -1 = default (separate) */
  int syn_stages[2];
  int ana_ltiles[2];
  int ana_stages[2];
  float ms_ring, ms_ring_default;
  float ms_synthesis, ms_synthesis_default;
  float ms_analysis, ms_analysis_default;
  int from_cache;  /* 1: taken from the process-wide cache without measuring */
} dm_tuning;

/* Time the candidate launch configurations of the plan's current precision
 * on its own buffers with CUDA events on `stream` and keep the fastest per
 * launch.  Results are cached per process for (device, nside, lmax, batch,
 * precision, tensor cores); a later plan of the same kind takes them without
 * measuring unless force != 0.  Outside a solve only (DM_EBUSY during one);
 * it overwrites the plan's iteration buffers, so call it before
 * dm_solve_begin.  Results of a solve do not depend on the configuration
 * beyond rounding.  Synchronises. */
dm_status dm_autotune(dm_plan *plan, int force, void *stream);
/* The configuration in use (after dm_autotune or dm_set_tuning; zeros and
 * -1 radixes when neither ran). */
dm_status dm_get_tuning(const dm_plan *plan, dm_tuning *out);
/* Apply a configuration (e.g. one stored from an earlier dm_get_tuning);
 * out-of-range values fall back to the heuristic; DM_EBUSY during a solve. */
dm_status dm_set_tuning(dm_plan *plan, const dm_tuning *t);

/* alpha and T_h of the noise model of RHS 0 (host outputs). */
dm_status dm_noise_info(const dm_plan *plan, double *alpha, double *t_h);

/* --- measurement --------------------------------------------------------- */

/* Per-stage device time of the dual messenger iterations, measured with CUDA
 * events recorded on the caller's stream around every stage launch, and the
 * number of kernels this library launched.  Enabling resets the counters. */
typedef struct {
  int64_t launches;        /* kernels launched by this plan since enabling */
  int64_t iterations;      /* dual messenger iterations timed */
  double ms_analysis;      /* Legendre analysis (a2) */
  double ms_reduce;        /* chunk reduction + harmonic step + filter (a2/a3) */
  double ms_synthesis;     /* Legendre synthesis (a4) */
  double ms_ring;          /* inverse FFT, update, norms, forward FFT (a5, a6, a7, a1) */
  double ms_control;       /* Cauchy ratio and level control (a7, a8) */
  int64_t anchors;         /* FP64 anchors of the mixed mode */
  double ms_anchor;        /* their total device time */
} dm_profile;

dm_status dm_profile_enable(dm_plan *plan, int on);
dm_status dm_profile_read(const dm_plan *plan, dm_profile *out);

/* ALU roofline denominators of the current device, measured with independent
 * FMA chains on every SM (about 0.2 s): FP64 and FP32 TFLOP/s (FMA = 2 flops).
 * The paper has no counterpart; it is the peak the FP64 Legendre stage is
 * compared against. */
dm_status dm_measure_alu_peaks(double *fp64_tflops, double *fp32_tflops);

/* --- the flat-sky setting (Section 2.1, Section 3.1) ----------------------- */

/* A plan for the paper's own flat-sky problem: an N x N grid (N a power of two,
 * 16 <= N <= 2048) of a square patch of side L radians, batch RHS.  Maps are
 * [batch][3][N * N] float64 row-major (pixel (y, x) at (y L/N, x L/N)).
 * Transforms: a_l = Omega_p sum_x m(x) e^{-i l.x} with Omega_p = (L/N)^2 and
 * l = 2 pi k / L, m(x) = L^-2 sum_l a_l e^{i l.x}; polarisation by the E/B
 * rotation of Eqs. 13-16, E = Q cos 2phi + U sin 2phi,
 * B = -Q sin 2phi + U cos 2phi, phi the angle of l from the l_x axis.  The
 * Nyquist row and column are outside the harmonic space.  Harmonic layout
 * (alm_out of the solve calls): [batch][3][N/2][N] complex128, kx = 0 .. N/2-1
 * major, ky in FFT order (0 .. N/2-1, then -N/2 .. -1); the modes kx < 0 are
 * the complex conjugates of (-kx, -ky).  The pair is exact (F^dagger F = 1),
 * so the iteration is Algorithm 1 as printed.  Solves (dm_wiener_filter,
 * dm_wiener_filter_host, dm_solve_*), the transform stages (dm_alm2map,
 * dm_map2alm, the ring and column stages), the schedule calls,
 * dm_autotune, the end-of-solve diagnostics and constrained realisations
 * (dm_constrained_realization, dm_draw_cr_inputs) work on it, in DM_FP64.
 * Its constrained-realisation signal draw takes unit white-noise maps z
 * instead of per-mode normals: for pixel p = y N + x, counters (p, 0, 2, 0)
 * -> (I, Q) and (p, 1, 2, 0) -> (U, -), Box-Muller as at dm_draw_cr_inputs;
 * ahat = (L/N) FFT2(z), unrotated, times the per-mode Cholesky factor of the
 * TE block and sqrt(BB), zero on the Nyquist row (so <a a^H> = L^2 S); the
 * noise draw is that of dm_draw_cr_inputs, zero on each masked component.
 * dm_jacobi_refine works on it too (the source with per-mode spectra and
 * the pixel area for Omega).  The sphere-only calls (spectra per l, HEALPix
 * noise setters, dm_apply_filter) return DM_EINVAL. */
dm_status dm_plan_create_flat(int N, double L, int batch, dm_plan **out);
/* Spectra per Fourier mode, host S[4][N][N] (TT, EE, BB, TE) in numpy FFT
 * order (axis 0 = ky, axis 1 = kx), <|a_l|^2> = L^2 C per mode; each 2x2 TE
 * block positive semi-definite. */
dm_status dm_set_spectra_flat(dm_plan *plan, const double *S);
/* Diagonal noise with distinct temperature and polarisation masks, host
 * sigma[3][N * N], mask_t / mask_p [N * N] (1 = observed, NULL = all):
 * alpha = min sigma^2 over observed components, w = alpha / sigma^2 there and
 * 0 on masked components (N^{-1} = 0), T_h = alpha Omega_p.  Shared by every
 * RHS. */
dm_status dm_set_noise_flat(dm_plan *plan, const double *sigma, const uint8_t *mask_t, const uint8_t *mask_p);

/* --- testing hook --------------------------------------------------------- */

/* Failure test of the tensor-core pipeline's bounded waits (no counterpart in
 * the paper): while on, the spin-0 tensor-core analysis of the mixed mode
 * withholds one plain mbarrier arrival (with stored tiles the first converter
 * thread of its first CTA, with generated tiles the first lane of its first
 * worker warp; first K step), so the MMA warp's wait gives up after 1 s with
 * no copy or MMA in flight on that barrier; the CTA then drains its copies,
 * frees its tensor memory and exits, and the solve calls return
 * DM_ETIMEOUT.  The plan and the CUDA context stay usable: turn it off and
 * the next solve is normal.  Not for production use. */
dm_status dm_test_tc_withhold(dm_plan *plan, int on);

/* --- serving: continuous batching of requests of different geometries ---- */

/* A server keeps one plan ("pool") per (nside, lmax, spectra) whose RHS are
 * slots.  A worker thread admits queued requests into free slots, or into a new
 * pool while the device-memory budget allows (idle pools are released to make
 * room), sets each slot up alone (its noise, mask, tolerance, data and, for a
 * constrained realisation, its Philox draws), then advances every pool with
 * busy slots by iters_per_round iterations on the pool's own stream so pools
 * overlap on the device, and retires converged slots into the caller's buffer.
 * A request's messenger state stays on the device from admission to
 * retirement, and its result does not depend on the other requests sharing the
 * device. */
typedef struct dm_server dm_server;

typedef enum { DM_REQ_WF = 0, DM_REQ_CR = 1 } dm_request_kind;

typedef struct {
  size_t hbm_budget_bytes;   /* device memory the pools may reserve */
  int slots_per_plan;        /* RHS slots per pool (1..1024) */
  int iters_per_round;       /* iterations between admissions (>= 1) */
  dm_precision prec;         /* arithmetic of every pool */
  dm_schedule sched;         /* cooling schedule (eps_final is per request) */
  int anchor_every;          /* mixed-precision refinement period (0 = 256) */
  int max_pending;           /* queue bound; dm_serve_submit returns DM_EBUSY beyond it (0 = 100000) */
  double strict_tol;         /* requests with tol < strict_tol run in pools of strict_prec (0 = never) */
  dm_precision strict_prec;  /* DM_FP64 or DM_FLOAT_FLOAT: a mixed-mode Cauchy ratio cannot resolve
                                tolerances near the FP32 rounding of the iteration state */
} dm_server_config;

typedef struct {
  int nside, lmax;           /* geometry, 1 <= nside <= 1024, 2 <= lmax <= 4 nside */
  int kind;                  /* dm_request_kind */
  double tol;                /* final Cauchy threshold eps_final */
  uint64_t seed;             /* Philox key of the constrained-realisation draws */
  const double *cl;          /* host [4][lmax+1], copied at submit */
  const double *sigma;       /* host [3][npix], copied at submit */
  const uint8_t *mask;       /* host [npix] or NULL, copied at submit */
  const double *d;           /* host [3][npix], copied at submit */
  double *s_out;             /* host [3][npix]: written before the ticket completes; must stay valid until then */
} dm_request;

typedef struct {
  dm_status status;          /* DM_OK, DM_ENOTCONV, DM_ENOMEM (never fits), DM_EAGAIN (cancelled), ... */
  int iters;                 /* dual messenger iterations run */
  double cauchy_final;
  double latency_ms;         /* submit to completion (host wall clock) */
  double queue_ms;           /* submit to admission */
} dm_result;

typedef struct {
  int64_t pending, busy_slots, pools, bytes_reserved, rounds, admitted, retired;
} dm_server_info_t;

dm_status dm_server_create(const dm_server_config *cfg, dm_server **out);
/* Queue a request; *ticket identifies it.  DM_EINVAL for a bad request (sizes,
 * kind, tolerance, sigma not finite and > 0 on an observed pixel, or a mask
 * with no observed pixel), DM_EBUSY when the queue is full.  A request the
 * plan setup rejects later completes with that status; one that can never fit
 * the memory budget completes with DM_ENOMEM. */
dm_status dm_serve_submit(dm_server *srv, const dm_request *req, uint64_t *ticket);
/* DM_OK and *out once the request completed (the ticket is then released),
 * DM_EAGAIN while it is queued or running, DM_EINVAL for an unknown ticket. */
dm_status dm_serve_poll(dm_server *srv, uint64_t ticket, dm_result *out);
/* Remove a request that is still queued (its result reports DM_EAGAIN);
 * DM_EBUSY once admitted. */
dm_status dm_serve_cancel(dm_server *srv, uint64_t ticket);
dm_status dm_server_info(dm_server *srv, dm_server_info_t *out);
/* Completes every queued and running request, then frees the pools. */
void dm_server_destroy(dm_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* DMWF_H */
