// spa_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace spa {

constexpr double LN2 = 0.69314718055994530941723212145818;
constexpr double LOG2E = 1.4426950408889634073599246810019;

// Launch helpers return cudaGetLastError() of the launch.

// Set the message spa_last_error(NULL) returns on this thread ("msg" followed by value
// when value >= 0). Writes into fixed storage; never allocates.
void set_thread_error(const char* msg, int64_t value = -1);

// ----------------------------------------------------------- genotype store
// Integer column sums of G (S1 = sum g, S2 = sum g^2, SY = sum y g) and the case count,
// with device-side validation of G in {0,1,2} and y in {0,1} (DERR_INPUT).
cudaError_t launch_store_sums(const int8_t* G, const uint8_t* y, int64_t n, int64_t p,
                              unsigned long long* sums /* [3p + 1], zeroed */, uint32_t* err,
                              cudaStream_t st);
// Means m_j, population sds s_j and v_j = sum_i y_i x_ij from the integer sums; per-column
// FP32 constants; the BF16 GEMM operand [n][Kp] = (g_i0..g_i,p-1, 1, 0...); the FP32
// standardised X [n][p].
cudaError_t launch_store_finish(const int8_t* G, int64_t n, int64_t p, int Kp, const unsigned long long* sums,
                                double* mean, double* sd, double* v, float* l2e_over_s, float* mean_f, float* colf,
                                __nv_bfloat16* Gbf, float* Xf, uint32_t* err, cudaStream_t st);

cudaError_t launch_store_pack_t(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, int64_t n_r,
                                __nv_bfloat16* GT, float* yv, cudaStream_t st);
// XT2 [p][n] = X^T log2(e) (single-coordinate moves).
cudaError_t launch_store_xt2(const float* Xf, int64_t n, int64_t p, float* XT2, cudaStream_t st);
// y as a bitmask: bit (i % 32) of word i / 32 is y_i; words cover `words` * 32 individuals.
cudaError_t launch_store_ybits(const uint8_t* y, int64_t n, int64_t words, uint32_t* ybits, cudaStream_t st);

// ------------------------------------------------------------- SMC kernels
// Precision plan: GB300's CUDA-core FP64 rate is a small fraction of FP32 and an FP64 warp
// instruction costs a full warp issue even with one active lane, so per-element work is
// FP32 with compensated (TwoSum) sums, and FP64 appears only in thread-per-particle code
// (the weights, log-likelihoods, log-priors, MH ratios) and in the resampling sums.
struct PriorArgs {
    float a;   // degrees of freedom (ignored for the double exponential)
    int de;    // 1: double-exponential prior
};

// Normalised weights in the forms their consumers need.
struct WeightArrays {
    double* logw;    // log W_i, normalised (log-sum-exp 0)
    double* W;       // W_i (resampling cumulative sum)
    float* Wf;       // W_i in FP32 (column moments, weighted means)
    uint32_t* wfix;  // round(W_i 2^31) (exact integer sums for quantiles and concentrations)
};

cudaError_t launch_init_prior(float* beta, int64_t N, int p, PriorArgs pr, const double* sched, int t0,
                              const uint64_t* seed, cudaStream_t st);

// ------------------------------------------------------------- moves
// A move is a proposal for every particle (beta' in beta_p, its GEMM row in A), the GEMM
// for the proposals' log-likelihood partials, and the Metropolis-Hastings test. The test of
// move m runs at the start of move m+1's proposal kernel (the accepted proposal is written
// back as the state while it is read), and the last move of a step ends with a commit
// kernel, so that between steps beta (and gl) hold the particles.
//
// Log-likelihoods and log-priors in the MH test are compensated FP32 pairs (s, c), value
// s + c: llq in partial units (ln 2 * nats for the tensor-core path, nats for the FP32
// path) and lpq = sum_j log1p(|b_j|/(a c_t)) (Gt) or sum_j |b_j| (double exponential) at
// the current scale; log alpha = sp_scale (l' - l) + coef(c_t) (q' - q) with
// coef = -(a+1) or -1/c, formed in FP32 from the pairs.
struct MhState {
    float2* llq;               // current log-likelihood pair (partial units)
    float2* lpq;               // current log-prior term sum pair at c_t
    const float2* lpt_p;       // proposal's log-prior term sum pair
    const float2* ydq;         // proposal's linear term y . eta (partial units)
    const float* partial;      // proposal's softplus partials [n_parts][ld_part]
    int n_parts;
    int64_t ld_part;
    float sp_scale;            // natural-log units per partial unit
    double sp_scale_d;         // the same in FP64 (for the log-weights)
    unsigned long long* acc_count;
    // log of each pending proposal's accept uniform, [2][ld_lu]: the kernel that proposes
    // move m writes row m & 1 for its block's particles, the MH test of move m reads it
    float* lu;
    int64_t ld_lu;
};

struct MoveArgs {
    float* beta;                 // particle states
    float* beta_p;               // proposals
    __nv_bfloat16* A;            // GEMM rows, NULL on the FP32 path
    int ldA, Kp;
    float2* lpt_p;
    float2* ydq;
    const float* sigma;          // RW: per-coordinate step; MALA: D_j
    const float* sqrt_D;         // MALA: sqrt(D_j) and 1/D_j (written beside D_j)
    const float* inv_D;
    const float* l2e_over_s;
    const float* mean_f;
    const float* vy;             // v_j in partial units (y . eta = beta . v)
    MhState mh;
    // MALA only
    float* gl;                   // grad l of the states
    const float* gl_p;           // grad l of the proposals
    float2* fwd;                 // forward-move residual sum of the proposals
    const float* h;              // step size
};

// The paper's single-coordinate cycle (move kind 2): M cycles over j = 0..p-1 per launch.
struct SiteArgs {
    float* beta;                      // particle states [N][p], updated in place
    float2* llq;                      // at the end of the step: log-likelihood (partial units)
    float2* lpq;                      //   and log-prior term sum pair, as the MH state keeps them
    float inv_sp_scale;               // partial units per nat
    const float* XT2;                 // [p][n] standardised genotypes times log2(e)
    const float* vy;                  // v = X^T y (nats)
    float sd;                         // proposal standard deviation
    unsigned long long* acc_count;   // accepted coordinate updates (may be NULL)
};
constexpr size_t SITE_SMEM_MAX = 220 * 1024;  // eta2 and beta rows of a block's particles
// Particles per block (one warp each) for n individuals and p markers; 0 if one does not fit.
int site_warps_per_block(int64_t n, int p);
cudaError_t launch_move_site(const SiteArgs& a, int64_t N, int p, int64_t n, PriorArgs pr, const float4* stepk, int t,
                             uint32_t m0, int M, const uint64_t* seed, cudaStream_t st);

// The reweighting kernel's constants of step t >= 1 (entry 0 unused).
struct ReweightK {
    float k1, kc, kac, inv_ac;  // c_{t-1} - c_t, c_t, a c_{t-1}, 1/(a c_t)
    double lbase;               // -p log(c_t / c_{t-1})
    double dinv;                // 1/c_t - 1/c_{t-1}
};
// The per-step constants of a schedule sched [T]: the move kernels' (a c_t, log-prior
// coefficient, 1/c_t, 1/(a c_t)) into out [T] and, with rk != NULL, the reweighting
// kernel's into rk [T] (p markers).
cudaError_t launch_step_constants(PriorArgs pr, const double* sched, int T, int p, float4* out, ReweightK* rk,
                                  cudaStream_t st);
// Random-walk move (decide: MH test of the pending proposal first; noise = 0: pack beta
// unchanged, for the log-likelihood entry points and t = 0).
cudaError_t launch_move_rw(const MoveArgs& a, bool decide, int64_t N, int p, PriorArgs pr, const float4* stepk, int t,
                           uint32_t m, uint32_t m_prev, const uint64_t* seed, int noise, uint32_t* err, cudaStream_t st);
// MALA move: needs grad l of the states in gl, D_j (sigma) and h from launch_colstats kind 1.
cudaError_t launch_move_mala(const MoveArgs& a, bool decide, int64_t N, int p, PriorArgs pr, const float4* stepk, int t,
                             uint32_t m, uint32_t m_prev, const uint64_t* seed, uint32_t* err, cudaStream_t st);
// MH test of the pending proposals, then accepted rows (and gradients) into the state.
cudaError_t launch_move_commit(const MoveArgs& a, bool mala, int64_t N, int p, PriorArgs pr, const float4* stepk, int t,
                               uint32_t m_prev, const uint64_t* seed, uint32_t* err, cudaStream_t st);
// The packed particles' log-likelihoods as the state (llq, lpq), and in FP64 to logw
// (prior-IS weights) and/or ll_out; either may be NULL.
cudaError_t launch_finish_loglik(const MhState& s, int64_t N, double* logw, double* ll_out, uint32_t* err,
                                 cudaStream_t st);
// lambda *= exp(acceptance - 0.574) (MALA step adaptation) and a device scalar store.
cudaError_t launch_adapt_lambda(double* lam, const unsigned long long* acc, double denom, cudaStream_t st);
cudaError_t launch_set_f64(double* ptr, double v, cudaStream_t st);

// logw += log p(beta | c_t) - log p(beta | c_{t-1}); the log-prior pair lpq refreshed at c_t.
cudaError_t launch_reweight(const float* beta, double* logw, float2* lpq, int64_t N, int p, PriorArgs pr,
                            const ReweightK* rk, int t, uint32_t* err, cudaStream_t st);

// Log-sum-exp and ESS of logw (per-CTA partial (max, sum e, sum e^2) combined in block order
// by the last CTA), then normalisation into W, Wf, wfix.
// mode 0: step t >= 1 (log_z[t] = LSE); 1: prior-IS start (log_z[0] = LSE - log N);
// 2: resample-move start (log_z[0] = LSE - log N, resampling forced, ESS not recorded).
constexpr int LSE_BLOCKS = 128;
constexpr int LSE_SCRATCH = 3 * LSE_BLOCKS + 4;  // doubles
cudaError_t launch_lse_ess(const WeightArrays& w, int64_t N, double* scratch, unsigned int* counter, int t, int mode,
                           double ess_frac, double* ess_out, double* logz_out, uint8_t* resampled_out, int* flag,
                           uint32_t* err, cudaStream_t st, bool pdl = true);
// Wf and wfix from a given W (for the summaries entry point).
cudaError_t launch_weight_forms(const double* W, int64_t N, float* Wf, uint32_t* wfix, cudaStream_t st);

cudaError_t launch_mark_uniform(int64_t N, int t, double* ess_out, uint8_t* resampled_out, int* flag, cudaStream_t st);

// Systematic resampling: ancestor indices (bit-exact blocked cumulative sum: block-local sums
// over the SMs, the carries in block order, then a parallel binary search that adds them),
// gather of particle rows into scratch and copy back. All no-ops when *flag == 0. cum holds
// N + ceil(N/256) + 1 doubles (local sums, carries, u).
cudaError_t launch_resample_index(const double* W, int64_t N, double* cum, int32_t* idx, const int* flag,
                                  int t, const uint64_t* seed, double u_override, cudaStream_t st);
cudaError_t launch_gather(const int32_t* idx, const float* beta, float* beta_tmp, const float2* llq, const float2* lpq,
                          float2* llq_tmp, float2* lpq_tmp, const float* g, float* g_tmp, int64_t N, int p,
                          const int* flag, cudaStream_t st);
cudaError_t launch_copyback(float* beta, const float* beta_tmp, float2* llq, float2* lpq, const float2* llq_tmp,
                            const float2* lpq_tmp, float* g, const float* g_tmp, const WeightArrays& w, int64_t N, int p,
                            const int* flag, cudaStream_t st);

// Weighted column moments -> per-coordinate proposal scales. kind 0 (RW):
// sigma_j = lam/sqrt(p) max(sd_j, floor c) into scale_out [p]; kind 1 (MALA):
// D_j = max(var_j, (floor c)^2), sqrt(D_j) and 1/D_j into scale_out [3p].
constexpr int COLSTAT_SPLITS = 128;
// With lam_dev (MALA) it also writes h = lambda p^{-1/6} to h_out.
cudaError_t launch_colstats(const float* beta, const float* Wf, int64_t N, int p, float4* part, float* scale_out,
                            int kind, double lam_const, const double* lam_dev, double sd_floor,
                            const double* sched, int t, float* h_out, cudaStream_t st);

// Per-scale summaries of Section 5 for step t.
struct SummaryArgs {
    int nq;
    double q[8];
    int nd;
    double delta[8];
    // filled by launch_summaries: the smallest float >= delta[d], and ceil(q 2^31)
    float dthr[8];
    unsigned long long target[8];
};
// keysT: N * p words of scratch (the transposed keys; two kernels).
cudaError_t launch_summaries(const float* beta, const float* Wf, const uint32_t* wfix, int64_t N, int p,
                             const SummaryArgs& s, int t, double* mean, double* quant, double* conc, uint32_t* keysT,
                             cudaStream_t st);
// The two halves of launch_summaries, for running the summaries beside the next step: the
// key transpose (with WfS != NULL also a copy of the weights into WfS, wfixS), then the
// summaries from keys and weights. pdl: launch with programmatic stream serialization.
cudaError_t launch_keys(const float* beta, const float* Wf, const uint32_t* wfix, int64_t N, int p, uint32_t* keysT,
                        float* WfS, uint32_t* wfixS, bool pdl, cudaStream_t st);
cudaError_t launch_summaries_keys(const uint32_t* keysT, const float* Wf, const uint32_t* wfix, int64_t N, int p,
                                  const SummaryArgs& s, int t, double* mean, double* quant, double* conc, bool pdl,
                                  cudaStream_t st);

// Scale-marginalised summaries (mixture over the steps with weights Z_t / Z_1).
cudaError_t launch_marginal(const double* log_z_inc, const double* mean, const double* conc, int64_t T, int64_t p,
                            int D, double* post_c, double* mean_out, double* conc_out, cudaStream_t st);

cudaError_t launch_accept_rate(const unsigned long long* acc_count, int T, double denom, double* rate,
                               cudaStream_t st);

// Opt the summaries kernel into its dynamic shared memory (once per device, before any capture).
cudaError_t smc_init_attributes();

// Stream-test helpers.
cudaError_t launch_philox(const uint32_t* ctr, uint2 key, int64_t count, uint32_t* out, cudaStream_t st);
cudaError_t launch_normals(uint64_t seed, uint32_t particle, uint32_t t, uint32_t m, int64_t p, float* out,
                           cudaStream_t st);
cudaError_t launch_prior_sample(uint64_t seed, PriorArgs pr, double c, int64_t N, int64_t p, float* out,
                                cudaStream_t st);
cudaError_t launch_prior_logpdf(PriorArgs pr, double c, const float* beta, int64_t k, double* out,
                                cudaStream_t st);

// ------------------------------------------------------------ MAP by EM
// Section 2.1 (EM with weighted-L1 logistic steps), Section 4.1 (the MAP path).
struct MapData {
    const float* Xf;    // [n][p] standardised genotypes
    const float* XT2;   // [p][n] the same times log2(e)
    const uint8_t* y;   // [n]
    int64_t n;
    int p;
    const float* lip;   // ||X||_2^2 / 4 (launch_map_lipschitz)
    PriorArgs pr;
};
constexpr size_t MAP_SMEM_MAX = 200 * 1024;
bool map_fits(int64_t n, int p);  // the solve's shared-memory plan fits one block
cudaError_t map_init_attributes();
cudaError_t launch_map_lipschitz(const MapData& d, float* lip, cudaStream_t st);
// S independent EM solves from beta0 [S][p] at scale c.
cudaError_t launch_map(const MapData& d, const float* beta0, int S, double c, int max_em, float tol, float* beta_out,
                       double* lp_out, cudaStream_t st);
// The MAP path over T steps from the recorded best particles best [T][p], as Jacobi rounds
// of its recurrence: A / lpA the modes from the best particles (round 0), S / lpS / chg two
// ping-pong copies ([2][T][p], [2][T], [2][T]) of the kept modes and of whether each changed
// in the round that wrote it, n_changed the count of changes of one round (zeroed by the
// caller). Round k writes copy k & 1.
struct MapRoundBufs {
    float* A;
    double* lpA;
    float* S;
    double* lpS;
    int* chg;
    int* n_changed;
};
cudaError_t launch_map_round(const MapData& d, const float* best, const double* sched, int T, int round, int max_em,
                             float tol, const MapRoundBufs& b, cudaStream_t st);
// Step t's particle of highest posterior density into best[t].
cudaError_t launch_best_particle(const MhState& s, const float* beta, int64_t N, int p, PriorArgs pr,
                                 const double* sched, int t, float* best, cudaStream_t st);

// ------------------------------------------------------------ likelihood
// tcgen05 split-BF16 GEMM with the fused softplus reduction: partial[c * N_pad + i] receives
// -sum over the 32-individual chunk c of log2(1 + 2^eta2), eta2 = eta log2(e), so that
// l = ln(2) * (sum of the partials + beta . v log2(e)) with v = X^T y.
// Tile configurations of the likelihood kernel (the tuner chooses one per shape):
//   config  n-tile width BN  G stages  epilogue warps  particle operand (K <= 256)
//   0       256              3         16              shared memory
//   1       128              4         16              shared memory
//   2       256              3         8               shared memory
//   3       128              6         16              shared memory (resident only)
//   4       256              6         8               tensor memory (resident only)
//   5       128              12        16              tensor memory (resident only)
//   6       224              4         8               shared memory, compact (resident, and the
//                                                      last of four k-blocks at most 32 wide)
// Configurations 3-6 need the particle operand resident (K <= 256). The residual (MALA)
// variant uses the configuration's BN with 3 or 4 stages, 8 epilogue warps and A in shared
// memory. Every configuration gives the same partial sums bit for bit (one per 32 individuals).
constexpr int TC_CONFIGS = 7;
int tc_config_bn(int cfg);
// whether configuration cfg can run the kernel for p markers (K = p + 1)
bool tc_config_valid(int cfg, int64_t p);
struct TcPlan {
    int cfg;         // tile configuration
    int BN;          // individuals per n-tile (128 or 256)
    int n_tiles;     // ceil(n / BN)
    int m_tiles;     // N_pad / 128
    int kblocks;     // active 64-wide k-blocks of each half
    int ksteps;      // active 16-wide k-steps of each half: ceil((p+1)/16)
    int grid;        // persistent CTAs
    int n_parts;     // partial sums per particle = ceil(n / 32), whatever BN
    int tw;          // width of a narrow last k-block (16 or 32 columns), or 0
};
// The likelihood kernel's tensor maps: A and G with 64-column boxes (128-byte swizzle) and,
// when the plan has a narrow last k-block, the same with tw-column boxes.
struct TcMaps {
    CUtensorMap A, B, At, Bt;
    const __nv_bfloat16* Araw = nullptr;  // the particle operand the maps A, At describe
};
// cfg: the tile configuration (the tuner's choice); -1 picks by the size of n.
TcPlan tc_plan(int64_t n, int p, int64_t N_pad, int num_sms, int cfg = -1);
// Opt the tensor-core kernels into their dynamic shared memory (once per device, before any capture).
cudaError_t tc_init_attributes();
bool tc_make_map_A(CUtensorMap* map, const __nv_bfloat16* A, int64_t N_pad, int Kp);
bool tc_make_map_B(CUtensorMap* map, const __nv_bfloat16* Gbf, int64_t n, int Kp, int BN);
bool tc_make_map_A_tail(CUtensorMap* map, const __nv_bfloat16* A, int64_t N_pad, int Kp, int tw);
bool tc_make_map_B_tail(CUtensorMap* map, const __nv_bfloat16* Gbf, int64_t n, int Kp, int BN, int tw);
// Residual mode of the likelihood kernel (the adjoint's first half): also writes
// r = y - logit^{-1}(eta) as BF16 hi | lo rows of R [N_pad][2 n_r] and its row sums.
struct ResidArgs {
    __nv_bfloat16* R;        // [N_pad][2 n_r], columns >= n stay zero
    int64_t n_r;             // round_up(n, 64)
    float* rsum_part;        // same layout as the softplus partials
};
// ybits: y as a bitmask, one word per 32 individuals (ceil(n_tiles * BN / 32) words, zero beyond n).
// wait_ns: the limit of each bounded mbarrier wait (0: the default, WAIT_LIMIT_DEFAULT_NS).
// stall != 0 (injected, for tests of the timeout path): the MMA issuer first waits on a
// barrier that nothing arrives at, so that wait runs out and the kernel returns early.
cudaError_t launch_loglik_tc(const TcMaps& maps, const TcPlan& plan, int64_t n, int Kp, const uint32_t* ybits,
                             float* partial, int64_t N_pad, uint32_t* err, cudaStream_t st,
                             const ResidArgs* resid = nullptr, uint64_t wait_ns = 0, int stall = 0);

// One region's entry in a grouped likelihood launch (many regions' units in one persistent
// launch). The table lives in device memory; CUtensorMap is aligned to 64 bytes or more, so
// every entry and each of its maps keeps that alignment.
struct TcRegion {
    CUtensorMap A, B, At, Bt;  // as TcMaps, for this region's buffers and its plan's BN
    float* partial;            // [n_parts][N_pad] softplus partials
    const uint32_t* ybits;
    __nv_bfloat16* R;          // residual mode: [N_pad][2 n_r]
    float* rsum_part;
    int64_t N_pad, n_r;
    int64_t unit0;             // global index of the region's first unit
    int tw, n_tiles, m_tiles, kblocks, ksteps, Kp, n;
};
// Units of region r: m_tiles x n_tiles in row-major order, global indices from unit0. CTA b
// of `grid` takes the global units [cta_units[b], cta_units[b + 1]). All regions of one launch
// share the tile configuration, the residual mode and the A-resident mode (kblocks <= 4).
cudaError_t launch_loglik_tc_grouped(const TcRegion* regs, int R, const int64_t* cta_units, int grid, int cfg, bool ar,
                                     bool resid, uint32_t* err, cudaStream_t st, uint64_t wait_ns = 0);
// Whether a plan's particle operand stays resident in shared memory (K <= 256).
bool tc_plan_resident(const TcPlan& plan);

// The adjoint's second half: C = R G (tcgen05, split-BF16 R, exact G^T [p][n_r]) into
// gpart[ksplit][N_pad][p], then grad l = (sum C - m_j sum r) / s_j (+ prior gradient).
struct AdjPlan {
    int64_t n_r;
    int kblocks, BN2, p_tiles, m_tiles, ksplit, grid;
};
AdjPlan adj_plan(int p, int64_t n, int64_t N_pad, int num_sms);
bool adj_make_map_R(CUtensorMap* map, const __nv_bfloat16* R, int64_t N_pad, int64_t n_r);
bool adj_make_map_GT(CUtensorMap* map, const __nv_bfloat16* GT, int p, int64_t n_r, int BN2);
// max_ctas > 0 caps the grid (the CTAs then loop over the output tiles; the partials do not
// change), else one CTA per output tile and K-split. r_last_use_hint reads R under an L2
// evict-first policy (R is dead after this kernel): measured faster for a region that has
// the GPU to itself, slower for a batch's regions side by side.
cudaError_t launch_adjoint_tc(const CUtensorMap& mapR, const CUtensorMap& mapGT, const AdjPlan& a, int p, float* gpart,
                              int64_t N_pad, uint32_t* err, cudaStream_t st, uint64_t wait_ns = 0, int max_ctas = 0,
                              bool r_last_use_hint = false);
cudaError_t launch_grad_finish(const float* gpart, int ksplit, const float* rsum_part, int n_parts, int64_t N_pad,
                               int64_t N, int p, const float* mean_f, const float* inv_sd, const float* B, PriorArgs pr,
                               double c, float* grad, cudaStream_t st);

// Plain FP32 SIMT path: partial[nt * N_pad + i] = -sum over 64-individual tile nt of
// softplus(eta_r) (natural units; the linear half beta . v is added by the move kernels).
constexpr int SIMT_TILE_N = 64;
cudaError_t launch_loglik_simt(const float* beta_p, const float* Xf, const uint8_t* y, int64_t N, int64_t n, int p,
                               float* partial, int64_t N_pad, cudaStream_t st);

// Plain FP32 gradient: eta = B X^T materialised, r = y - logit^{-1}(eta); grad = r X
// (+ prior gradient at c when c > 0); ll = sum y eta - softplus(eta).
cudaError_t launch_grad_simt(const float* B, const float* Xf, const uint8_t* y, int64_t N, int64_t n, int p,
                             float* eta_scratch, float* grad, double* ll, PriorArgs pr, double c, cudaStream_t st);

}  // namespace spa
