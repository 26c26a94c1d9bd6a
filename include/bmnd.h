/*
 * bmnd.h - C ABI of the B300 (sm_103a) BMND denoiser.
 *
 * BMND (arXiv 2609.34622) denoises an array y with any number of axes in two
 * stages (Sec. 3, "Method Overview"): stage 1 matches patches against the
 * observation, filters each group by hard thresholding of its separable
 * transform against propagated noise variances (Sec. 5) and aggregates the
 * filtered patches by variance-weighted, Kaiser-windowed overlap-add (Sec. 7);
 * stage 2 repeats matching on the stage-1 estimate (the pilot) and applies
 * empirical Wiener shrinkage to the observation's coefficients (Sec. 6).
 * Optionally each stage is made to conserve the observed total (Sec. 8).
 *
 * Conventions for every entry point:
 *  - Arrays are float32, C-contiguous (last axis fastest), in DEVICE memory of
 *    the context's device, unless an argument says "host".
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *    is the legacy default stream).  Inputs must stay valid and unmodified,
 *    and outputs unread, until the stream reaches the end of the call's work.
 *  - Scratch memory is owned by the context and reused between calls; two
 *    calls on one context must not run concurrently (different contexts may).
 *  - Errors are reported by return code.  BMND_EINVAL is returned before any
 *    work is enqueued; bmnd_last_error() gives a one-line reason.  No call
 *    traps, asserts or aborts on the device.
 *  - Processing units follow the paper's experiment section: Poisson data are
 *    y = s_P K with K the event counts; Gaussian data are y = x + n.
 */
#ifndef BMND_H
#define BMND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BMND_MAX_NDIM 8

typedef struct bmnd_ctx bmnd_ctx;

typedef enum {
    BMND_OK = 0,
    BMND_EINVAL = 1,        /* invalid argument (nothing enqueued)             */
    BMND_ENOMEM = 2,        /* device memory or scratch budget exhausted       */
    BMND_ECUDA = 3,         /* a CUDA runtime call failed                      */
    BMND_ETIMEOUT = 4,      /* a bounded device-side wait gave up              */
    BMND_EUNSUPPORTED = 5   /* valid request this build does not implement     */
} bmnd_status;

/* Observation model (Sec. 3.1 / 3.2).
 * kind = BMND_NOISE_GAUSSIAN: additive white Gaussian noise with standard
 *   deviation `sigma` >= 0 (Def. "Additive Gaussian observation model").
 * kind = BMND_NOISE_POISSON: scaled Poisson, y = s_P K, with
 *   `poisson_scale` = s_P > 0 (Def. "Scaled-Poisson observation model"). */
enum { BMND_NOISE_GAUSSIAN = 0, BMND_NOISE_POISSON = 1 };
typedef struct {
    int kind;
    double sigma;
    double poisson_scale;
} bmnd_noise;

enum { BMND_SCHEDULE_GENERATED = 0, BMND_SCHEDULE_OFF = 1, BMND_SCHEDULE_SPARSE = 2,
       BMND_SCHEDULE_BALANCED = 3 };
enum { BMND_POWER_CLASSIC = 0, BMND_POWER_NOISE_FLOOR = 1, BMND_POWER_VARIANCE_SCALED = 2 };
enum { BMND_GROUP_HAAR = 0, BMND_GROUP_DCT = 1 };
enum { BMND_WEIGHT_CLASSIC = 0, BMND_WEIGHT_VARIANCE = 1, BMND_WEIGHT_RISK = 2 };
enum { BMND_SCOPE_PATCH = 0, BMND_SCOPE_GROUP = 1 };
/* Stage-1 matching distance (Sec. 4.2) and acceptance policy (Sec. 4.3). */
enum { BMND_METRIC_SSD = 0, BMND_METRIC_DEVIANCE = 1, BMND_METRIC_PEARSON = 2, BMND_METRIC_ANSCOMBE = 3 };
enum { BMND_POLICY_FIXED = 0, BMND_POLICY_REFERENCE = 1, BMND_POLICY_STANDARDIZED = 2 };
/* Stage-1 thresholding rule (Def. "Coefficient thresholding"). */
enum { BMND_HT_HARD = 0, BMND_HT_SOFT = 1 };
/* Aggregation-weight domain (Sec. 7.3). */
enum { BMND_DOMAIN_COEFFICIENT = 0, BMND_DOMAIN_WINDOWED = 1 };
/* Spatial transform of the hard-threshold stage (App. A). */
enum { BMND_SPATIAL_DCT = 0, BMND_SPATIAL_BIOR15 = 1 };
/* The finite-count moment tables cover pooled counts 0..BMND_MOMENT_NMAX; a
 * pooled count above it uses the moments at BMND_MOMENT_NMAX. */
#define BMND_MOMENT_NMAX 4096

/* Algorithm profile.  bmnd_default_params() fills the standard configuration
 * of App. A ("Standard Configuration"):
 *   lambda_ht 3.0 (hard-threshold multiplier, Def. "Coefficient thresholding")
 *   gamma_ht 3.0 (SSD noise-bias factor in stage 1, Def. "Noise-bias-corrected
 *     SSD"); gamma_wie 0.0 (plain SSD on the pilot in stage 2)
 *   tau_ht, tau_wie <= 0: matching thresholds 3000 P / 255^2 and 400 P / 255^2
 *     for P patch entries (App. A lists 2.9527 and 0.3937 for P = 64)
 *   s_v 0.4 (Wiener variance scale, Def. "Practical Wiener gain")
 *   kaiser_beta 2.0; shift_density 2.0 and passes 2 (generated schedule,
 *     Sec. 4.1); power_mode classic (Def. "Pilot-power modes");
 *   group_transform Haar; min_group 2; weight_model variance, weight_scope
 *     patch (Defs. "Coefficient-domain hard-thresholding / Wiener weighting
 *     models").
 *   match_metric SSD (App. A); match_policy fixed; match_t 3.0; beta_s 0.1
 *     and kappa_s 1.0 (Sec. 9.4); ht_rule hard (App. A); weight_domain
 *     coefficient (App. A); cov_planes 0 (the diagonal variance model; App. A
 *     lists 4 exact covariance planes); spatial_transform DCT (App. A lists
 *     bior1.5 for the hard-threshold stage).
 *
 * spatial_transform = BMND_SPATIAL_BIOR15 transforms the patch axes of stage
 * 1 by the biorthogonal spline wavelet bior1.5 (App. A, "Transforms" row):
 * periodic extension, full depth on every patch axis, whose sides must be
 * powers of two (BMND_EINVAL otherwise); coefficient variances are
 * sum_i T_ki^2 m_v(u_i) with the non-orthonormal analysis T (Lemma
 * "Covariance propagation"), the inverse is its synthesis matrix, and the
 * windowed weighting models use that synthesis.  Stage 2 keeps the DCT.  It
 * runs in the generic kernels.
 *
 * cov_planes = k_ex > 0 (scaled-Poisson noise only, at most 32) gives the
 * coefficients of the first k_ex planes of the group-axis transform, in both
 * stages, the partial shared-source variance of Def. "Partial shared-source
 * Poisson variance model": entries of overlapping members that come from
 * the same location add their transform weights before squaring (Def.
 * "Effective transform weights").  It runs in the generic kernels.
 *
 * weight_domain = BMND_DOMAIN_WINDOWED measures the weighting models of both
 * stages in the windowed synthesized domain (Def. "Windowed synthesized-
 * domain weighting models"): with the diagonal filters and noise model here,
 * tr(H F Sigma F^H) weights each coefficient's term by the diagonal of the
 * windowed synthesis metric H (Def. "Windowed synthesis metrics"), i.e. by
 * sum_p |U_pq|^2 w_p^2 over the spatial inverse transform U and the Kaiser
 * aggregation window w of a patch.
 *
 * ht_rule = BMND_HT_SOFT replaces the stage-1 hard threshold by the soft one
 * of Eq. (soft-threshold), C_k = sgn(Y_k) [|Y_k| - lambda_ht sigma_k]_+: the
 * attenuation a_k = C_k / Y_k then enters the hard-thresholding weighting
 * models as |a_k|^2 (classic) or |a_k|^2 sigma_k^2 (variance).
 *
 * Poisson-aware stage-1 matching (Secs. 4.2-4.3; scaled-Poisson noise only,
 * BMND_EINVAL otherwise).  With match_metric != SSD, stage 1 ranks the
 * candidates of a reference p by one of the distances built from the raw
 * counts r_i = [p_i / s_P]_+, c_i = [q_i / s_P]_+ (Eq. raw-counts):
 * P d_m = sum_i phi_m(r_i, c_i) with phi the Poisson deviance (Eq. deviance),
 * the Pearson statistic (Eq. pearson) or half the squared Anscombe difference
 * (Eq. anscombe-distance); gamma_ht is not used.  Acceptance (then the group
 * rules of App. A as for SSD):
 *   fixed:        d_m < tau_ht, or, with tau_ht <= 0, d_m < 1 + t sqrt(2/P)
 *                 (the high-count null, mean 1 and variance 2 per entry,
 *                 Thm. "Common high-count limit");
 *   reference:    d_m < T_ref(p; t) of Eq. (reference-threshold), with the
 *                 exact moments mu_m, v_m of Prop. "Universal finite-count
 *                 moments" at the pooled-count estimate 2 r_i rounded to the
 *                 nearest integer, plus beta_s r-bar^kappa_s;
 *   standardized: candidates ranked and accepted by Z_m < t of Eq.
 *                 (standardized-distance), n_i = r_i + c_i rounded.
 * Stage 2 keeps plain SSD on the pilot with tau_wie (App. B).
 *
 * Decisions.  Every ranking and acceptance comparison of matching, and the
 * hard threshold |Y_k| > lambda sigma_k, is the comparison of the
 * double-precision definition: scores are screened in float32 with an error
 * bound, and what the bound cannot separate is re-evaluated exactly (integer
 * sums for dyadic data and for the Poisson distances on count data) or in
 * double precision; groups and kept coefficients therefore differ from those
 * of the definition only at ties in real arithmetic. */
typedef struct {
    double lambda_ht;
    double gamma_ht;
    double gamma_wie;
    double tau_ht;
    double tau_wie;
    double s_v;
    double kaiser_beta;
    double shift_density;
    int passes;
    int schedule;
    int power_mode;
    int group_transform;
    int min_group;
    int weight_model;
    int weight_scope;
    int match_metric;
    int match_policy;
    double match_t;
    double beta_s;
    double kappa_s;
    int ht_rule;
    int weight_domain;
    int cov_planes;
    int spatial_transform;
} bmnd_params;

void bmnd_default_params(bmnd_params *p);

/* Finite-count null moments of a Poisson matching distance (Prop. "Universal
 * finite-count moments"; Prop. "Exact Pearson moments" for Pearson): writes
 * mu_m(n) and v_m(n), n = 0..count-1, rounded to float32, into the HOST
 * arrays mu[count] and v[count] -- the tables stage-1 matching reads.
 * metric is BMND_METRIC_DEVIANCE, _PEARSON or _ANSCOMBE; 1 <= count <=
 * BMND_MOMENT_NMAX + 1.  Host computation only (no device, no context).
 * Errors: BMND_EINVAL for a bad metric, count or null pointer. */
bmnd_status bmnd_match_moments(int metric, int count, float *mu, float *v);

/* Create a context on CUDA device `device`.  `scratch_budget_bytes` caps the
 * device scratch the context may hold (0 = no cap).  On success *ctx owns
 * that scratch until bmnd_destroy().  Errors: BMND_EINVAL (null ctx, bad
 * device), BMND_ECUDA. */
bmnd_status bmnd_create(bmnd_ctx **ctx, int device, size_t scratch_budget_bytes);

/* Release the context and its scratch (synchronizes the context's device). */
bmnd_status bmnd_destroy(bmnd_ctx *ctx);

/* One-line description of the last error on this context ("" if none). */
const char *bmnd_last_error(const bmnd_ctx *ctx);

/* Denoise y (both stages, App. A profile).  This is the paper's problem
 * statement (Sec. 3: recover x from y) with the two-stage algorithm.
 *   y, out       device float32 arrays of prod(shape) elements; out must not
 *                overlap y.
 *   ndim, shape  1 <= ndim <= BMND_MAX_NDIM, shape[d] >= 1 (host array).
 *   noise        observation model (see bmnd_noise).
 *   patch, step, search  host int[ndim]: patch size j_d (1 <= j_d <= shape[d],
 *                j_d <= 32), reference step h_d (1 <= h_d <= j_d), search window
 *                w_d (odd, >= 1) centred on the reference origin (Sec. 4.1/4.2).
 *   group_size   host int[2]: maximum group size in stage 1 / stage 2, a power
 *                of two in [1, 32] for the Haar group transform.
 *   stages       1 (hard thresholding only) or 2.
 *   mass_conserve bit 0: conserve mass in stage 1, bit 1: in stage 2 (Sec. 8).
 * Errors: BMND_EINVAL for any violated constraint above, BMND_EUNSUPPORTED if
 * more than 6 axes have length > 1, BMND_ENOMEM, BMND_ECUDA. */
bmnd_status bmnd_denoise(bmnd_ctx *ctx, const float *y, int ndim, const int64_t *shape,
                         bmnd_noise noise, const int *patch, const int *step, const int *search,
                         const int *group_size, int stages, int mass_conserve, float *out,
                         void *stream);

/* Same as bmnd_denoise with an explicit profile (NULL = defaults). */
bmnd_status bmnd_denoise_ex(bmnd_ctx *ctx, const float *y, int ndim, const int64_t *shape,
                            bmnd_noise noise, const int *patch, const int *step, const int *search,
                            const int *group_size, int stages, int mass_conserve,
                            const bmnd_params *params, float *out, void *stream);

/* One stage.  stage = 1: hard thresholding, matching on y.  stage = 2: Wiener
 * shrinkage of y's coefficients, matching on `pilot` (a device array like y,
 * the stage-1 estimate; Def. "Paired pilot and observation groups").
 * `group_max` is that stage's maximum group size; `mass_conserve` 0/1 applies
 * the two-sweep correction of Sec. 8 to this stage. */
bmnd_status bmnd_stage(bmnd_ctx *ctx, const float *y, const float *pilot, int ndim,
                       const int64_t *shape, bmnd_noise noise, const int *patch, const int *step,
                       const int *search, int group_max, int stage, int mass_conserve,
                       const bmnd_params *params, float *out, void *stream);

/* Reference schedule (Sec. 4.1, Def. "Clipped reference origin" and the
 * schedule selected by params->schedule).  Writes the distinct reference
 * origins as C-order linear indices into the DEVICE array `origins`
 * (capacity `cap`), in an order grouped by tile, and their number into the
 * HOST int64 *n_refs (the call synchronizes `stream` to read it back).
 * Returns BMND_ENOMEM if cap < *n_refs (nothing written past cap). */
bmnd_status bmnd_schedule(bmnd_ctx *ctx, int ndim, const int64_t *shape, const int *patch,
                          const int *step, const bmnd_params *params, int64_t *origins,
                          int64_t cap, int64_t *n_refs, void *stream);

/* Block matching only (Sec. 4.2-4.4 with the group rules of App. A) for every
 * scheduled reference.  `guide` is y (stage 1, noise-bias corrected SSD with
 * gamma_ht) or the pilot (stage 2, plain SSD).  Outputs (DEVICE, capacity
 * `cap` references): origins[cap] reference linear origins, groups[cap *
 * group_max] member linear origins in group order (reference first, unused
 * slots -1), counts[cap] group sizes.  *n_refs (HOST) receives the number of
 * references (the call synchronizes `stream`). */
bmnd_status bmnd_match(bmnd_ctx *ctx, const float *guide, int ndim, const int64_t *shape,
                       bmnd_noise noise, const int *patch, const int *step, const int *search,
                       int group_max, int stage, const bmnd_params *params, int64_t *origins,
                       int64_t *groups, int32_t *counts, int64_t cap, int64_t *n_refs,
                       void *stream);

/* Reference coverage of the schedule params selects (Sec. 9.3, "Shift
 * Schedule Analysis"): C(x), the number of scheduled reference patches that
 * contain location x, for every x of an array of the given shape (patch,
 * step and params->schedule / shift_density / passes as for bmnd_schedule).
 *   coverage  DEVICE int32[prod(shape)], C-order, or NULL (map not written).
 *   n_refs    HOST: number of distinct scheduled origins |R|.
 *   cv        HOST: CV(C) = sigma_C / mu_C over all locations (population
 *             standard deviation; 0 when mu_C = 0).
 * Synchronizes `stream` to return n_refs and cv.  Errors: BMND_EINVAL for the
 * shape / patch / step constraints of bmnd_denoise or null n_refs / cv,
 * BMND_ENOMEM, BMND_ECUDA. */
bmnd_status bmnd_coverage(bmnd_ctx *ctx, int ndim, const int64_t *shape, const int *patch, const int *step,
                          const bmnd_params *params, int32_t *coverage, int64_t *n_refs, double *cv,
                          void *stream);

/* One job of a batched call. */
typedef struct {
    const float *y;
    float *out;
    int ndim;
    int64_t shape[BMND_MAX_NDIM];
    bmnd_noise noise;
    int patch[BMND_MAX_NDIM];
    int step[BMND_MAX_NDIM];
    int search[BMND_MAX_NDIM];
    int group_size[2];
    int stages;
    int mass_conserve;
} bmnd_job;

/* Denoise n_jobs independent arrays in shared launches: every kernel of a
 * stage covers the tiles of all jobs at once (a flat (job, tile) work list).
 * Each job's result equals that of bmnd_denoise_ex on the job alone.  Jobs
 * with different numbers of non-singleton axes are accepted: the stage
 * kernels are compiled per rank, so each rank class runs as its own batch,
 * one class after another on `stream`.  All jobs use the same stage count.
 * Errors as bmnd_denoise, reported for the first invalid job. */
bmnd_status bmnd_denoise_batch(bmnd_ctx *ctx, int n_jobs, const bmnd_job *jobs,
                               const bmnd_params *params, void *stream);

/* bmnd_denoise_batch with host arrays (the paper has no counterpart: a
 * convenience for callers whose data live in host memory).  jobs[i].y and
 * jobs[i].out are HOST pointers (float32, C-order; pinned memory makes the
 * copies asynchronous DMA, pageable memory is staged by the driver).  The
 * call copies every y to context-owned device buffers (grown on use, held
 * until bmnd_destroy), runs bmnd_denoise_batch on them on `stream`, copies
 * every result back and waits for the stream: on return the outputs are
 * in host memory.  Errors: as bmnd_denoise_batch; BMND_ENOMEM when the
 * device buffers cannot be allocated; BMND_ECUDA on a failed copy. */
bmnd_status bmnd_denoise_batch_host(bmnd_ctx *ctx, int n_jobs, const bmnd_job *jobs,
                                    const bmnd_params *params, void *stream);

/* Plan of one array (diagnostics; no counterpart in the paper): info[0] the
 * number of tiles, info[1] the cells of a tile's region (the partial each
 * tile writes and the reduce kernel reads, float2 each), info[2] the
 * reference capacity of a tile, info[3] the number of non-singleton axes,
 * info[4..7] the tile core along those axes (0 past them).  Arguments as
 * bmnd_denoise_ex; nothing is launched.  Errors: those of bmnd_denoise_ex's
 * argument checks. */
bmnd_status bmnd_plan_info(bmnd_ctx *ctx, int ndim, const int64_t *shape, const int *patch, const int *step,
                           const int *search, const int *group_size, int stages, int mass_conserve,
                           const bmnd_params *params, int64_t info[8]);

/* FP32 FMA throughput of a device in TFLOP/s (measurement only; no
 * counterpart in the paper): a kernel of independent fused multiply-add
 * chains on every SM, timed with CUDA events (best of three after a
 * warm-up), 2 flops per FMA.  It allocates and frees a small output array.
 * Errors: BMND_EINVAL (bad device or null tflops), BMND_ENOMEM, BMND_ECUDA. */
bmnd_status bmnd_fp32_fma_peak(int device, double *tflops);

/* Per-kernel timing, for measurement only (the paper has no counterpart).
 * With profiling enabled, every kernel launched by the context is bracketed by
 * CUDA events recorded on the launch stream.  bmnd_kernel_stats() synchronizes
 * the context's device, folds the recorded pairs into per-kind totals and
 * returns, for one kind, the number of launches and their summed duration in
 * milliseconds since the last reset (reset != 0 clears all totals after
 * reading).  Kinds: */
enum { BMND_KERNEL_SCHEDULE = 0, BMND_KERNEL_STAGE1 = 1, BMND_KERNEL_STAGE2 = 2,
       BMND_KERNEL_REDUCE = 3, BMND_KERNEL_MC_SWEEP = 4,
       BMND_KERNEL_MATCH = 5,  /* match-only stage launches of bmnd_match */
       BMND_KERNEL_KINDS = 6 };
bmnd_status bmnd_set_profiling(bmnd_ctx *ctx, int enable);
bmnd_status bmnd_kernel_stats(bmnd_ctx *ctx, int kind, int reset, int64_t *launches,
                              double *total_ms);

/* Counters of the decisions taken in double precision (diagnostics; no
 * counterpart in the paper).  The kernels score candidates and compare
 * coefficients with the hard threshold in FP32, each with an error bound;
 * wherever the bound cannot separate two candidates' scores, a score from
 * the acceptance threshold or a coefficient from lambda sigma_k, the
 * decision is re-taken in double precision as the definitions read
 * (Eq. ssd, Def. "Noise-bias-corrected SSD", App. A group rules, Eq.
 * hard-threshold).  counts[0]: candidates rescored; counts[1]: windows scored
 * entirely in double precision (an ambiguous run longer than the warp's
 * list); counts[2]: coefficients decided in double precision.  Synchronizes
 * the context's device; totals since the context was created or since the
 * last reset (reset != 0 clears them after reading).
 * Errors: BMND_EINVAL for a null context or counts, BMND_ECUDA. */
bmnd_status bmnd_decision_stats(bmnd_ctx *ctx, int reset, uint64_t counts[3]);

/* ---- Serving loop --------------------------------------------------------
 * A request server (the paper has no counterpart; it serves the data-parallel
 * path to many concurrent requests).  A worker thread admits submitted jobs in
 * arrival order while the device-memory budget and the slot count allow,
 * copies each admitted job's input to the device and builds its reference
 * schedule.  Jobs go to one of two lanes by their estimated GPU time (1 ms):
 * each lane has its own stream (the small-job lane at the higher priority)
 * and keeps up to two steps queued, in which its jobs run both stages.  The
 * small-job lane batches all its waiting jobs into a step, jobs of the same
 * kernel class sharing one launch of each kernel; the large-job lane runs one
 * job per step, the shortest estimate first, aged by the time waited, with
 * one CTA per tile, so that the small-job lane's CTAs take SMs between its
 * tiles.
 * When a job's step is done its output is copied to the host and its memory
 * is released.  Each job owns its tiles and partial sums, so its result is
 * bitwise the same as bmnd_denoise on the job alone.
 * Jobs use the App. A profile. */
typedef struct bmnd_server bmnd_server;
typedef struct {
    size_t mem_budget_bytes;  /* device memory for admitted jobs (0: 8 GiB)   */
    int max_slots;            /* jobs admitted at the same time (0: 256)      */
} bmnd_server_config;
typedef struct {
    int64_t submitted, completed, failed;
    double p50_ms, p99_ms, mean_ms;  /* latency: submission to result on the host */
    double voxels_per_s;             /* completed voxels / (last completion - first submission) */
    int64_t steps;                   /* server steps (shared launches)            */
    double mean_jobs_per_step;
} bmnd_server_stats;

/* Create a server on `device` (allocates the budget up front).  Errors:
 * BMND_EINVAL, BMND_ENOMEM, BMND_ECUDA. */
bmnd_status bmnd_server_create(bmnd_server **srv, int device, const bmnd_server_config *cfg);
/* Submit a job; job->y and job->out are HOST arrays that must stay valid
 * until bmnd_server_wait returns for the ticket.  Invalid jobs (as for
 * bmnd_denoise) and jobs larger than the budget are rejected here. */
bmnd_status bmnd_server_submit(bmnd_server *srv, const bmnd_job *job, int64_t *ticket);
/* Wait for a ticket (timeout_ms < 0: no limit; BMND_ETIMEOUT if it runs out);
 * returns the job's status and its latency in *latency_ms (may be NULL).  A
 * ticket can be waited for once. */
bmnd_status bmnd_server_wait(bmnd_server *srv, int64_t ticket, int timeout_ms, double *latency_ms);
bmnd_status bmnd_server_get_stats(bmnd_server *srv, bmnd_server_stats *stats);
/* Finish all submitted jobs, stop the worker and release everything. */
bmnd_status bmnd_server_destroy(bmnd_server *srv);

/* ---- Tile autotuning ------------------------------------------------------
 * Times the computation of bmnd_denoise_ex on this array with several tile
 * cores (the part of the array whose reference patches one CTA owns; the
 * planner's choice, powers of two per axis for one or two axes, steps of one
 * and two around the planner's choice for more), each also with one resident
 * CTA per SM where the shared memory would allow two (the stage kernels then
 * keep the whole register file instead of a cap of 128 per thread), and keeps
 * the fastest in the context, keyed by shape, patch, step, search, group sizes, stages, mass
 * conservation and profile (not the noise level).  Later calls on this
 * context with the same key -- bmnd_denoise, bmnd_denoise_ex, the batched
 * and graph entry points -- plan with that core.  The paper has no
 * counterpart: tiling is an execution choice and changes the output only by
 * the order of floating-point additions.
 *   - Synchronous: it runs each candidate three times on `stream` and waits.
 *   - out receives the estimate with the chosen core.
 *   - core (host int[ndim], may be NULL) receives the chosen core per axis
 *     (1 for axes of length 1); the CTAs-per-SM choice is kept with it but
 *     not reported.
 * Errors: those of bmnd_denoise_ex. */
bmnd_status bmnd_autotune(bmnd_ctx *ctx, const float *y, int ndim, const int64_t *shape, bmnd_noise noise,
                          const int *patch, const int *step, const int *search, const int *group_size, int stages,
                          int mass_conserve, const bmnd_params *params, float *out, void *stream, int *core);

/* Batched autotuning: as bmnd_autotune, but timing bmnd_denoise_batch on the
 * whole batch `jobs` (where the arrays share the SMs, which a single array
 * timed alone does not show).  The fastest core is kept for the problem key
 * of jobs[0] and applies to every job of that key; jobs of other keys keep
 * their cores.  Every job's out receives its estimate with the chosen
 * cores; core (host int[jobs[0].ndim], may be NULL) receives jobs[0]'s.
 * Synchronous.  Errors: those of bmnd_denoise_batch. */
bmnd_status bmnd_autotune_batch(bmnd_ctx *ctx, int n_jobs, const bmnd_job *jobs, const bmnd_params *params,
                                void *stream, int *core);

/* ---- Replayable graphs ----------------------------------------------------
 * The computation of bmnd_denoise_ex (both stages, Sec. 4-5 as for that call)
 * on one array, recorded once as a CUDA graph and replayed: for arrays that
 * are denoised again and again with the same shape and parameters (frames of
 * a detector, slices of a series), where the host-side planning and the
 * dozen launches of a call would otherwise be repeated.  The paper has no
 * counterpart: this is an execution convenience.
 *   - bmnd_graph_create plans the array, allocates the graph's own scratch
 *     and descriptor table (device memory, held until bmnd_graph_destroy),
 *     uploads the table (synchronously) and records the launches with stream
 *     capture on a private stream.  Call it outside any stream capture.
 *   - y and out are device arrays BOUND at creation: refill y (float32,
 *     C-order, shape as given) and launch again to denoise new data; out
 *     receives the estimate.  They must stay allocated while the graph lives.
 *   - bmnd_graph_launch enqueues the graph on `stream`; launches of one graph
 *     share its scratch, so they must not overlap on the GPU (launch on one
 *     stream, or order them).  A replay gives bitwise the output of
 *     bmnd_denoise_ex on the same input.
 *   - bmnd_graph_destroy waits for the device to be idle, then frees it.
 *   - Replays read tables owned by the context (the DCT matrices, and the
 *     finite-count moment tables of a Poisson matching distance): destroy
 *     every graph of a context before the context.
 * Errors: those of bmnd_denoise_ex; BMND_ENOMEM / BMND_ECUDA when the scratch
 * cannot be allocated or the recording fails (bmnd_last_error of ctx says). */
typedef struct bmnd_graph bmnd_graph;
bmnd_status bmnd_graph_create(bmnd_ctx *ctx, const float *y, int ndim, const int64_t *shape, bmnd_noise noise,
                              const int *patch, const int *step, const int *search, const int *group_size,
                              int stages, int mass_conserve, const bmnd_params *params, float *out,
                              bmnd_graph **graph);
bmnd_status bmnd_graph_launch(bmnd_graph *graph, void *stream);
bmnd_status bmnd_graph_destroy(bmnd_graph *graph);

/* Allocation-free denoising (the paper has no counterpart: this is a
 * deployment convenience).  Same computation and arguments as bmnd_denoise
 * with the parameters that bmnd_default_params sets, but no context and no
 * allocation: it calls no
 * cudaMalloc, cudaFree, pinned-host or other allocating routine.  It is meant
 * for callers that cannot allocate device memory: code running while another
 * component owns the device allocator, services working inside a memory
 * budget that is already committed, or environments where cudaMalloc is
 * unavailable or would synchronize the device at the wrong moment.
 *
 * Scratch: one file-scope device array of 64 MiB, held by every GPU that
 * loads the library until the process exits.  Arrays whose plan needs more
 * scratch are rejected with BMND_ENOMEM before any work is enqueued (a 1-D
 * signal of 262144 samples and a 2-D 512x512 image fit; a 2048x2048 image
 * does not).
 *   - The first call on a device (the current device) performs a one-time,
 *     synchronous set-up: it resolves the array's device address, copies the
 *     float and double DCT tables into the array, uploads the butterfly-DCT
 *     constants to the device's constant bank and reads the device limits.
 *     A process may call this entry point without ever creating a context.
 *   - Calls must not be recorded by stream capture (each call copies its
 *     two-entry job table from host stack memory): a call on a capturing
 *     stream returns BMND_EUNSUPPORTED before enqueueing anything.
 *   - Every call shares the array, which keeps the previous call's contents;
 *     the call clears what must start at zero.  Calls whose work overlaps on
 *     the GPU (different streams, or host threads on one device) race on the
 *     array and give wrong results: serialize them.
 *   - errbuf/errlen (may be NULL/0) receive a one-line message on error.
 * Errors: as bmnd_denoise, plus BMND_ENOMEM when the array is too small and
 * BMND_EUNSUPPORTED on a capturing stream. */
bmnd_status bmnd_denoise_noalloc(const float *y, int ndim, const int64_t *shape, bmnd_noise noise,
                                 const int *patch, const int *step, const int *search,
                                 const int *group_size, int stages, int mass_conserve, float *out,
                                 void *stream, char *errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif
#endif /* BMND_H */
