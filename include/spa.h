/*
 * spa.h -- C ABI of the GB300 sparsity-path-analysis (SPA) library.
 *
 * The library runs the sequential Monte Carlo sweep over the scale c of a
 * generalised-t prior on logistic-regression coefficients (Lee, Caron, Doucet &
 * Holmes, arXiv:1106.0322, Sections 2-5) on one NVIDIA GB300 (sm_103a). Every step
 * of the sweep runs in the library's own CUDA kernels: the genotype store, the
 * split-BF16 tcgen05 likelihood GEMM with a fused softplus epilogue (or a plain
 * FP32 SIMT comparator), the prior incremental weight, the FP64 log-sum-exp / ESS,
 * systematic resampling, the random-walk / MALA moves and the per-scale summaries.
 *
 * Conventions for every function:
 *   - Return value: SPA_OK (0) or one of the SPA_E* codes below. No exception, no
 *     abort and no exit crosses this boundary; spa_last_error() gives a message.
 *   - Pointers are HOST pointers unless the name ends in _device, where they are
 *     device pointers of the current CUDA device.
 *   - Inputs are read during the call and never retained; the library copies what it
 *     keeps. Outputs are caller-allocated buffers of the documented size.
 *   - Matrices are row-major. Genotypes G are n x p (individual-major); particle
 *     matrices B are N x p (particle-major).
 *   - A context is not thread-safe: use one context per host thread. Distinct
 *     contexts may be used concurrently.
 *   - The library owns all device memory it allocates and frees it in spa_destroy.
 */
#ifndef SPA_H
#define SPA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status codes */
#define SPA_OK 0
#define SPA_EINVAL 1      /* invalid argument: sizes < 1, nu <= 0 or NaN, genotype not in
                             {0,1,2}, phenotype not in {0,1}, a monomorphic marker (sd 0),
                             a non-positive or non-finite scale, NULL pointer */
#define SPA_ENOMEM 2      /* device or host allocation failed */
#define SPA_ECUDA 3       /* a CUDA runtime call failed (message in spa_last_error) */
#define SPA_ETIMEOUT 4    /* a bounded device-side wait gave up (the kernel returned early) */
#define SPA_ENUMERIC 5    /* NaN/Inf in a log-likelihood or a log-weight, or ESS < 1 */
#define SPA_EUNSUPPORTED 6 /* configuration not supported (e.g. no sm_100-family GPU) */

/* ------------------------------------------------------------------ configuration */
#define SPA_MOVE_RW 0       /* joint random-walk Metropolis-Hastings */
#define SPA_MOVE_MALA 1     /* Metropolis-adjusted Langevin, driven by the adjoint kernel */
#define SPA_MOVE_SITE 2     /* the paper's own kernel (Section 4.1, "Further details"): per move,
                               a cycle of single-coordinate random-walk Metropolis updates
                               j = 1..p with proposal sd site_sd, each an O(n) update of X beta;
                               runs on CUDA cores (FP32), the precision field is ignored */

#define SPA_PREC_SPLIT_BF16 0 /* tcgen05: X exact in BF16, beta = hi + lo BF16, FP32 accumulate */
#define SPA_PREC_FP32 1       /* plain FP32 SIMT (FFMA) comparator path */

#define SPA_INIT_PRIOR_IS 0       /* prior draws at c_1 weighted by the likelihood */
#define SPA_INIT_RESAMPLE_MOVE 1  /* the same, then resampled and burn_in_steps x M moves */

#define SPA_MAX_QUANTILES 8
#define SPA_MAX_DELTAS 8

typedef struct spa_config {
    int32_t move_kind;       /* SPA_MOVE_RW (default), SPA_MOVE_MALA or SPA_MOVE_SITE */
    int32_t precision;       /* SPA_PREC_SPLIT_BF16 (default) or SPA_PREC_FP32 */
    int32_t init_mode;       /* SPA_INIT_PRIOR_IS (default) or SPA_INIT_RESAMPLE_MOVE */
    int32_t burn_in_steps;   /* blocks of M moves at c_1 for SPA_INIT_RESAMPLE_MOVE (default 0) */
    int32_t n_quantiles;     /* number of weighted quantile levels (default 3) */
    double quantiles[SPA_MAX_QUANTILES]; /* levels in (0,1) (default 0.05, 0.5, 0.95) */
    int32_t n_deltas;        /* number of concentration thresholds (default 2) */
    double deltas[SPA_MAX_DELTAS];       /* Delta > 0 of V = 1 - Pr(|beta_j| < Delta) (0.05, 0.1) */
    double ess_frac;         /* resample when ESS < ess_frac * N (default 0.75, Section 4) */
    double rw_scale;         /* RW: sigma_j = rw_scale/sqrt(p) * max(sd_W(beta_j), sd_floor*c) (2.38) */
    double mala_h;           /* MALA: initial lambda in h = lambda * p^(-1/6) (1.65) */
    double sd_floor;         /* floor of the proposal scale relative to c (default 1e-3) */
    double site_sd;          /* SITE: proposal sd of one coordinate (0.5: the paper's variance 0.25) */
    int32_t map_path;        /* nonzero: record each step's particle of highest posterior density,
                                for spa_map_path after the run (default 0) */
    void* stream;            /* cudaStream_t to run on; NULL: the context's own stream */
} spa_config;

/* Per-scale outputs of a sweep, caller-allocated (any pointer may be NULL to skip it).
 * t indexes the schedule, j the marker, q the quantile level, d the threshold. */
typedef struct spa_result {
    double* mean;         /* [T*p]    weighted posterior mean of beta_j at c_t          */
    double* quantile;     /* [T*p*Q]  weighted quantiles (index (t*p + j)*Q + q)        */
    double* conc;         /* [T*p*D]  concentration 1 - Pr(|beta_j| < Delta_d)          */
    double* ess;          /* [T]      effective sample size after reweighting           */
    double* log_z_inc;    /* [T]      log Z_t/Z_{t-1}; entry 0 is log Z_1 (prior IS)    */
    double* accept_rate;  /* [T]      fraction of accepted proposals in step t's moves  */
    uint8_t* resampled;   /* [T]      1 if the particles were resampled at step t       */
} spa_result;

typedef struct spa_ctx spa_ctx;

/* Fills *cfg with the defaults listed above. */
void spa_config_default(spa_config* cfg);

/* --------------------------------------------------------------------- lifecycle */

/* Create a context for one hit region (Section 3 data, Section 2 model).
 *   G   n*p genotypes in {0,1,2}, row-major (individual i, marker j)
 *   y   n phenotypes in {0,1} (case = 1)
 *   nu  Gt degrees of freedom a > 0 (eq. gent_prior, q = 1); +INFINITY selects the
 *       double-exponential prior (the a -> infinity limit, Section 5.4)
 * Copies G and y to the device, standardises the columns (Section 3: mean 0, unit
 * population sd) and builds the exact BF16 GEMM operand. Errors: SPA_EINVAL for bad
 * sizes or values (including a monomorphic column), SPA_ENOMEM, SPA_ECUDA,
 * SPA_EUNSUPPORTED if the current device is not compute capability 10.x. */
int spa_create(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, double nu, spa_ctx** out);

/* Replace the genotypes and phenotypes of an existing context (same n, p). */
int spa_set_data(spa_ctx* ctx, const int8_t* G, const uint8_t* y);

/* Set / read the configuration. spa_set_config validates it (SPA_EINVAL). */
int spa_set_config(spa_ctx* ctx, const spa_config* cfg);
int spa_get_config(const spa_ctx* ctx, spa_config* cfg);

/* Free every device and host resource of the context. NULL is ignored. */
void spa_destroy(spa_ctx* ctx);

/* Message for the last failing call on this context, or, for ctx == NULL, the last
 * failure of a context-free call on this host thread. Never NULL. */
const char* spa_last_error(const spa_ctx* ctx);

/* --------------------------------------------------------------------- the sweep */

/* Run the SMC sampler over the prior scale (Section 4) with targets
 * pi_t(beta) = p(beta | X, y, a, c_t), t = 0..T-1:
 *   t = 0   N draws from Gt(a, c_0), weighted by the likelihood (log Z_1 estimate);
 *   t >= 1  reweight by gamma_t/gamma_{t-1} (the prior ratio, Section 4 with the
 *           reversal backward kernel), log Z_t/Z_{t-1} = log sum_i W_{t-1} w_t;
 *   every t resample (systematic) if ESS < ess_frac*N, then moves_per_step MCMC
 *           moves invariant for pi_t (resample before move, Section 4), then the
 *           per-scale summaries of Section 5 into *out (host buffers).
 *   scale_schedule  T values c_t > 0 (any order; the paper sweeps b_t = a c_t down)
 *   N               particles (1 .. 2^22); moves_per_step >= 0; seed keys Philox.
 * Blocks until the results are on the host. SPA_ENUMERIC if a log-likelihood or a
 * weight became non-finite, SPA_ETIMEOUT if a device wait gave up. */
int spa_run(spa_ctx* ctx, const double* scale_schedule, int64_t T, int64_t N,
            int32_t moves_per_step, uint64_t seed, spa_result* out);

/* As spa_run, but the schedule and every spa_result array are DEVICE pointers and the
 * call only enqueues the sweep on the configured stream (no host synchronisation).
 * Inside the sweep each step's summaries run on a second stream owned by the context and
 * are joined back before the sweep's last kernel. Work enqueued on the configured stream
 * after the call therefore sees the whole sweep, outputs included. Device-side errors are
 * reported by the next spa_sync(). */
int spa_run_device(spa_ctx* ctx, const double* scale_schedule_device, int64_t T, int64_t N,
                   int32_t moves_per_step, uint64_t seed, spa_result* out_device);

/* Wait for work enqueued on the context's stream and report device-side errors. */
int spa_sync(spa_ctx* ctx);

/* Batched sweeps over R independent regions (Section 5 runs the sweep per region; each
 * context keeps its own data, nu and config). */
typedef struct spa_batch_args {
    const double* const* schedules;  /* R host pointers, schedule of region r      */
    const int64_t* T;                /* [R] schedule lengths                        */
    const int64_t* N;                /* [R] particle counts                         */
    const int32_t* moves_per_step;   /* [R]                                         */
    const uint64_t* seeds;           /* [R]                                         */
} spa_batch_args;
/* One-shot batch: spa_batch_create + spa_batch_run + spa_batch_destroy. outs: R results
 * (or NULL). */
int spa_run_batch(spa_ctx* const* ctxs, int32_t R, const spa_batch_args* args, spa_result* outs);

/* A reusable batch: the R sweeps are captured into ONE CUDA graph whose R branches (one
 * per context, on the context's stream) run concurrently on the GPU, and every
 * spa_batch_run is a single graph launch on the batch's own stream. Each region's
 * likelihood tile configuration comes from the tile table or the tuner. In this branch form
 * each region's likelihood and adjoint launches are sized for an eighth of the SMs (an
 * equal share when fewer than 8 regions), so that the regions share the GPU; the partials,
 * and so the results, do not depend on the grid.
 * With the environment variable SPA_BATCH_MODE=lockstep at creation, a batch whose regions
 * share T, N, moves_per_step, the move kind (RW or MALA), the start and the burn-in, on the
 * tensor cores, is captured in lock step instead: at every likelihood evaluation all regions
 * wait for each other and one persistent grouped launch per tile class evaluates every
 * region's particles (a device table of all regions' particle-tile x n-tile units). The
 * results are the same bit for bit; on the 64-region MALA workload the branch form is faster
 * (1.84 s against 2.26 s per batch), so it is the default.
 * Contexts must be distinct and outlive the batch; their schedules (args->schedules,
 * copied here), T, N and moves_per_step are fixed at creation. Results are bit-identical
 * to spa_run of each context with the same seed.
 * Errors: SPA_EINVAL (NULL or repeated contexts, bad sizes or schedule values),
 * SPA_ENOMEM, SPA_ECUDA; the message is spa_last_error(NULL). */
typedef struct spa_batch spa_batch;
int spa_batch_create(spa_ctx* const* ctxs, int32_t R, const spa_batch_args* args, spa_batch** out);
/* Run all R sweeps once. seeds: R seeds, or NULL for the seeds given at creation.
 * outs: R caller-allocated results (fields may be NULL), or NULL. Blocks until done.
 * SPA_EINVAL if a context's workspace, run buffers or config changed since creation
 * (spa_run with other shapes, spa_set_config, spa_loglik with another N); a device error
 * of region r is reported as that region's code, with spa_last_error(ctxs[r]). */
int spa_batch_run(spa_batch* batch, const uint64_t* seeds, spa_result* outs);
/* Kernel launches in one spa_batch_run (all regions). */
int64_t spa_batch_launch_count(const spa_batch* batch);
void spa_batch_destroy(spa_batch* batch);

/* Number of kernels the last spa_run / spa_run_device of this context launched. */
int64_t spa_last_launch_count(const spa_ctx* ctx);

/* Failure detection (the paper has no counterpart; the sweep must never hang the GPU).
 * Every mbarrier wait in the context's tensor-core kernels (likelihood, adjoint) is bounded.
 * When a wait runs out, the kernel sets an error bit, waits (at most 100 ms) for its own TMA
 * copies and MMAs in flight, frees its TMEM and returns; later waits of the same sweep give
 * up at once, the rest of the sweep runs on to its end, and the call that reads the error
 * word (spa_run, spa_sync, spa_loglik, ...) returns SPA_ETIMEOUT. The context stays usable:
 * the next sweep starts with a clear error word.
 * spa_set_wait_limit sets that bound for later launches of this context (limit_ns = 0: the
 * default, 4 s). A short limit lets a deployment fail fast on a wait that cannot complete.
 * It replaces the context's captured sweep graph. Errors: SPA_EINVAL for a NULL ctx.
 * Host-side fault injection, for tests of the error paths: the environment variable
 * SPA_FAULT, read at each call that can inject, holds a comma-separated list of
 *   alloc       every device allocation by the library fails (the call returns SPA_ENOMEM)
 *   nan_weight  the first log-weight of a sweep is set to NaN after the initial weighting
 *               (SPA_ENUMERIC, from the device-side finiteness check of the log-sum-exp)
 *   stall       each tensor-core likelihood launch first waits on a barrier that nothing
 *               arrives at, so that wait runs out after the wait limit (set a short one
 *               with spa_set_wait_limit first) and the call returns SPA_ETIMEOUT
 * A wait that runs out is the only way the timeout path is reached: mbarrier waits that
 * will complete suspend the thread until they do, so a short limit alone does not end them.
 * None of these faults, traps or hangs the GPU. */
int spa_set_wait_limit(spa_ctx* ctx, uint64_t limit_ns);

/* Individuals per n-tile (128, 224 or 256) of the tensor-core likelihood kernel for the
 * context's current workspace (its tile configuration's, below), or 0 before the first run.
 * The environment variable SPA_LOGLIK_BN=128|256, read when a workspace is created, fixes
 * it. The width does not change any result (partial sums are per 32 individuals either way). */
int spa_loglik_tile_width(const spa_ctx* ctx);

/* The likelihood kernel's tile configuration for the context's current workspace (-1 before
 * the first run), and where it came from (*source, may be NULL): 0 fixed (the environment,
 * spa_set_tile_config, or n <= 128), 1 the tile table, 2 timed by the tuner. Configurations:
 *   0: n-tiles of 256, 3 G stages, 16 epilogue warps   1: 128, 4 stages, 16 warps
 *   2: 256, 3 stages, 8 warps                          3: 128, 6 stages, 16 warps (p <= 255)
 *   4: 256, 6 stages, 8 warps, the particle operand held in tensor memory (p <= 255)
 *   5: 128, 12 stages, 16 warps, the particle operand held in tensor memory (p <= 255)
 *   6: 224, 4 stages, 8 warps, a compact resident particle operand (p <= 255 with the last of
 *      four k-blocks at most 32 columns wide: (p + 1) mod 64 in 1..32, or p < 192)
 * A shape takes SPA_TILE_CONFIG=0..6 (or SPA_LOGLIK_BN) from the environment, else the value
 * fixed by spa_set_tile_config, else the nearest shape of the tile table (a JSON file written
 * by the package's tune_tiles.py on a GB300: SPA_TILE_TABLE, else tuning/loglik_tiles.json
 * beside the package), else the tuner times every valid configuration once per process. No
 * configuration changes any result: the partial sums are per 32 individuals whatever the tile. */
int spa_loglik_tile_config(const spa_ctx* ctx, int32_t* source);
/* Fix the tile configuration (0..6; -1 returns to the table and tuner) for later runs of the
 * context: it replaces the context's workspace and captured graph. An invalid configuration
 * for the shape (3..6 with p > 255, 6 with a wide last k-block) is ignored at the next run.
 * SPA_EINVAL if out of range. */
int spa_set_tile_config(spa_ctx* ctx, int32_t cfg);

/* Enqueue `reps` launches of the context's likelihood kernel (split-BF16 tcgen05 or
 * FP32 SIMT, per the configuration) on `stream` over the particles last packed for
 * N (by spa_run / spa_loglik with the same N), in the launch configuration the sweep
 * uses. No host synchronisation; for timing the kernel with events on `stream`.
 * SPA_EINVAL if no workspace of N particles exists. */
int spa_loglik_repeat(spa_ctx* ctx, int64_t N, int32_t reps, void* stream);

/* The same for MALA's per-move gradient kernels on the tensor cores: `reps` times the
 * residual likelihood pass (softplus partials and r = y - logit^{-1}(eta) as BF16 hi | lo),
 * the adjoint GEMM C = R G and the gradient finish, over the proposals last packed for N, in
 * the sweep's launch configuration. SPA_EINVAL unless the context's last sweep was a
 * split-BF16 MALA sweep of N particles. */
int spa_grad_repeat(spa_ctx* ctx, int64_t N, int32_t reps, void* stream);

/* Scale-marginalised summaries (Section 4, eq. all_particles). With a uniform prior on
 * log b and a log-spaced schedule (as spa_run's geometric schedules are), the particle
 * systems of all steps mix with weights proportional to Z_t / Z_1, each estimated by the
 * running product of the Z_t / Z_{t-1} increments:
 *   post_c[t] = exp(L_t - max L) / sum_s exp(L_s - max L),  L_t = sum_{s=1..t} log_z_inc[s]
 * (log_z_inc[0] is common to every L_t and does not enter), which is also the posterior of
 * the scale on the schedule's grid. mean_out[j] = sum_t post_c[t] mean[t][j] and
 * conc_out[j][d] = sum_t post_c[t] conc[t][j][d] are the mixture's means and V(Delta).
 * Inputs are one sweep's spa_result arrays: log_z_inc [T], mean [T][p], conc [T][p][D]
 * (D = the config's n_deltas, 0..SPA_MAX_DELTAS; conc and conc_out may be NULL when
 * D = 0). Outputs: post_c [T], mean_out [p], conc_out [p][D]. All FP64, formed on the GPU.
 * spa_marginal takes host pointers and blocks; spa_marginal_device takes device pointers and
 * only enqueues on `stream`. Errors: SPA_EINVAL (NULL pointers, T or p < 1, D out of
 * range), SPA_ENOMEM, SPA_ECUDA. */
int spa_marginal(const double* log_z_inc, const double* mean, const double* conc, int64_t T, int64_t p, int32_t D,
                 double* post_c, double* mean_out, double* conc_out);
int spa_marginal_device(const double* log_z_inc, const double* mean, const double* conc, int64_t T, int64_t p,
                        int32_t D, double* post_c, double* mean_out, double* conc_out, void* stream);

/* MAP estimates by EM (Section 2.1). The scale-mixture representation makes each EM step
 * a weighted-L1 logistic regression, beta <- argmax l(beta) - sum_j w_j |beta_j| with
 * w_j = (a+1)/(a c + |beta_j|) (double exponential: 1/c), iterated until no coordinate
 * moves by more than tol (or max_em steps). The inner problem is solved on the GPU by
 * proximal-gradient steps with momentum and restarts, in FP32, to a tenth of tol.
 *
 * spa_map: S independent solves at scale c > 0 from beta0 [S][p] (host, FP32); beta_out
 * [S][p] receives the modes and logpost [S] (may be NULL) l + log p at them (FP64, the
 * constant -p log 2c included). Blocks until done.
 *
 * spa_map_path (Section 4.1): after a spa_run / spa_run_device of T steps with
 * config.map_path set, at each step t the EM starts from the step's particle of highest
 * posterior density and (t > 0) from the previous step's MAP, and the mode with the higher
 * log posterior is kept: map_out [T][p] (host, FP32), logpost [T] (host, may be NULL).
 * The rule is the recurrence S_0 = A_0, S_t = better(A_t, EM(c_t, S_{t-1})) with A_t the
 * mode from step t's best particle; it is solved by parallel rounds over t (all A_t, then
 * EM(c_t, S_{t-1}) again wherever S_{t-1} changed, until a round changes nothing), which
 * gives bit for bit what walking the steps in order gives. Blocks until done.
 *
 * spa_map_path_rounds: the number of rounds after the first that the last spa_map_path on
 * ctx took (1 when no step's chained start beat its best-particle start in a way that moved
 * a later step; at most T); -1 for a NULL ctx.
 *
 * Errors: SPA_EINVAL (NULL arguments, S or T < 1, c <= 0, max_em < 1, tol <= 0, no recorded
 * run of T steps with map_path, or n + 5p too large for one block's shared memory),
 * SPA_ENOMEM, SPA_ECUDA. */
int spa_map(spa_ctx* ctx, const float* beta0, int32_t S, double c, int32_t max_em, double tol, float* beta_out,
            double* logpost);
int spa_map_path(spa_ctx* ctx, int64_t T, int32_t max_em, double tol, float* map_out, double* logpost);
int spa_map_path_rounds(const spa_ctx* ctx);

/* spa_map_path_given: the same MAP path rule and solver from caller-given starts instead of a
 * recorded run: sched [T] the scales c_t > 0 (host), best [T][p] step t's best particle (host,
 * FP32). At t = 0 the EM starts from best[0]; at each later t from best[t] and from the MAP
 * kept at t - 1, and the mode with the higher log posterior is kept (a tie keeps the one from
 * best[t]). Outputs as spa_map_path. It lets the path be checked against an independent walk
 * of the rule from the same starts. Errors: SPA_EINVAL (NULL arguments, T < 1, a schedule
 * value not finite and > 0, max_em < 1, tol <= 0, n + 5p too large), SPA_ENOMEM, SPA_ECUDA. */
int spa_map_path_given(spa_ctx* ctx, const double* sched, const float* best, int64_t T, int32_t max_em, double tol,
                       float* map_out, double* logpost);

/* ------------------------------------------------------- per-step entry points */

/* Log-likelihood l(beta) = sum_i [y_i eta_i - log(1 + exp(eta_i))], eta = X beta
 * (Section 2, standardised X of Section 3) for N particles B (N*p floats), with the
 * context's precision: split-BF16 tcgen05 or plain FP32. ll_out: N doubles.
 * Split-BF16 bound: |err| <= (2^-15 + (2p+2) 2^-23) * sum_i (sum_j |g_ij bt_j| + |o|)
 *   + 2^-20 n + 2^-21 sum_i softplus(eta_i), with bt_j = beta_j/s_j, o = -sum_j m_j bt_j. */
int spa_loglik(spa_ctx* ctx, const float* B, int64_t N, double* ll_out);
int spa_loglik_device(spa_ctx* ctx, const float* B_device, int64_t N, double* ll_device,
                      void* stream);

/* Gradient of the log posterior at scale c, grad l(beta) + grad log p(beta | a, c)
 * (grad l = X^T (y - logit^{-1}(eta)); the prior term -(a+1) sgn(beta_j)/(a c + |beta_j|),
 * or -sgn(beta_j)/c for the double exponential, with sgn(0) = 0). c == 0 returns the
 * likelihood gradient alone. ll_out: N doubles (may be NULL); grad_out: N*p floats. */
int spa_grad(spa_ctx* ctx, const float* B, int64_t N, double c, double* ll_out, float* grad_out);
int spa_grad_device(spa_ctx* ctx, const float* B_device, int64_t N, double c, double* ll_device,
                    float* grad_device, void* stream);

/* Systematic resampling (Section 4 resamples when ESS < 3N/4; the scheme is systematic):
 * A_k = min{i : C_i > (k+u)/N}, clamped to N-1, C the cumulative sum of W formed in
 * blocks of 256 (running sum in each block, running sum of block totals before it,
 * C_i = carry + local_i), target ((double)k + u)/(double)N rounded to nearest.
 *   W  N normalised weights (doubles), u in [0,1); idx_out: N int32 ancestor indices.
 * Bit-exact given W and u. */
int spa_resample_systematic(const double* W, int64_t N, double u, int32_t* idx_out);

/* Allocation-free variant of spa_resample_systematic (the paper has no counterpart: it
 * is a deployment convenience). For callers that cannot call cudaMalloc: a process whose
 * device memory is held by another allocator's pool, a latency-critical path where an
 * allocation would synchronise the device, a service that must not grow its device
 * footprint after start-up. The caller passes DEVICE buffers; the call allocates nothing.
 *   W_device    N normalised weights (doubles, device memory)
 *   u           the uniform in [0,1)
 *   idx_device  N int32 ancestor indices (device memory), bit-identical to
 *               spa_resample_systematic's for the same W and u
 *   stream      cudaStream_t to enqueue on (NULL: the legacy default stream); returns
 *               without synchronising
 * The kernel's scratch (N + ceil(N/256) + 1 doubles) is a fixed device array of
 * SPA_NOALLOC_RESAMPLE_MAX_N + 1025 doubles (about 2.1 MB), held by every GPU that loads
 * the library until the process exits. N > SPA_NOALLOC_RESAMPLE_MAX_N is rejected with
 * SPA_EINVAL (message in spa_last_error(NULL)); a device that is not compute capability
 * 10.x with SPA_EUNSUPPORTED; a failed CUDA call with SPA_ECUDA and CUDA's error string.
 * The first call on a device looks the array's address up (cudaGetSymbolAddress) with that
 * device current: make that first call before any stream capture. The address is kept per
 * device together with the unique ID of the CUDA context it belongs to; after a
 * cudaDeviceReset the next call sees a new context and looks the address up again (that
 * call, too, must come before any capture). All calls share the array: calls whose kernels
 * overlap on the GPU (different streams, no ordering between them) race and must be
 * serialised by the caller. Nothing needs to start at zero: each call writes every entry it
 * reads. */
#define SPA_NOALLOC_RESAMPLE_MAX_N 262144
int spa_resample_systematic_noalloc(const double* W_device, int64_t N, double u, int32_t* idx_device,
                                    void* stream);

/* log Gt(beta | a, c) = -log(2c) - (a+1) log1p(|beta|/(a c)) per element (eq. gent_prior,
 * q = 1, mu = 0); nu = +INFINITY gives -log(2c) - |beta|/c. out: k doubles. */
int spa_prior_logpdf(double nu, double c, const float* beta, int64_t k, double* out);

/* Incremental log-weight per particle for a scale change c_prev -> c_new:
 * sum_j log p(beta_j | c_new) - log p(beta_j | c_prev) (Section 4: the likelihood
 * cancels under the reversal backward kernel). B: N*p floats; out: N doubles. */
int spa_incr_weight(double nu, double c_prev, double c_new, const float* B, int64_t N, int64_t p,
                    double* out);

/* Log-sum-exp and effective sample size (sum W)^2 / sum W^2 of N log-weights. */
int spa_lse_ess(const double* logw, int64_t N, double* lse_out, double* ess_out);

/* Weighted per-marker summaries of particles (Section 5.1-5.2): mean, quantiles
 * Q_q = beta_(k*) with k* = min{k : cumulative sorted weight >= q}, and concentration
 * 1 - Pr(|beta_j| < Delta). B: N*p floats, W: N normalised weights.
 * Outputs: mean[p], quant[p*nq], conc[p*nd] (doubles). */
int spa_summaries(const float* B, const double* W, int64_t N, int64_t p, const double* q,
                  int32_t nq, const double* deltas, int32_t nd, double* mean, double* quant,
                  double* conc);

/* The random streams (Philox4x32-10, Salmon et al. SC'11), for stream tests:
 *   spa_philox4x32_10: count counters (4 uint32 each) under one key -> 4*count outputs;
 *   spa_normals: the p move normals of (particle, step t, move m) under seed;
 *   spa_prior_sample: the N*p initial draws from Gt(a, c) under seed. */
int spa_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out);
int spa_normals(uint64_t seed, uint32_t particle, uint32_t t, uint32_t m, int64_t p, float* out);
int spa_prior_sample(uint64_t seed, double nu, double c, int64_t N, int64_t p, float* out);

#ifdef __cplusplus
}
#endif

#endif /* SPA_H */
