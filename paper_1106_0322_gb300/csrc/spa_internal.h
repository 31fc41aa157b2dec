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
                                double* mean, double* sd, double* v, float* l2e_over_s, float* mean_f,
                                __nv_bfloat16* Gbf, float* Xf, uint32_t* err, cudaStream_t st);

cudaError_t launch_store_pack_t(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, int64_t n_r,
                                __nv_bfloat16* GT, float* yv, cudaStream_t st);
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

// Random-walk proposal (noise = 1) or plain packing of beta (noise = 0): writes beta_p, the
// compensated sum of the proposal's log-prior terms (log1p(|b|/(a c)), or |b| for the double
// exponential) to lpt_p, and (A != NULL) the split-BF16 GEMM row [hi(bt) | lo(bt)] with
// bt_j = beta'_j log2(e)/s_j and the offset o = -sum_j m_j bt_j in column p.
cudaError_t launch_propose_rw(const float* beta, float* beta_p, __nv_bfloat16* A, int ldA, int Kp, float2* lpt_p,
                              const float* sigma, const float* l2e_over_s, const float* mean_f, int64_t N, int p,
                              PriorArgs pr, const double* sched, int t, uint32_t m, const uint64_t* seed, int noise,
                              cudaStream_t st);

// Finish log-likelihoods from the GEMM partial sums (l = sp_scale * sum of partials) and
// log-priors from lpt_p (without the constant -p log(2c), which cancels at a fixed scale),
// then store them (mode 0) or run the Metropolis-Hastings test (mode 1).
struct AcceptArgs {
    float* beta;
    const float* beta_p;
    double* ll;
    double* lp;
    const float2* lpt_p;
    const float* partial;
    int n_parts;
    int64_t ld_part;
    double sp_scale;
    double* logw;                    // mode 0: logw = ll (prior-IS weights); may be NULL
    unsigned long long* acc_count;  // mode 1: accepted-proposal counter; may be NULL
};
cudaError_t launch_accept(const AcceptArgs& a, int64_t N, int p, PriorArgs pr, const double* sched, int mode, int t,
                          uint32_t m, const uint64_t* seed, uint32_t* err, cudaStream_t st);

// MALA proposal (needs grad l at beta in gl, D_j from launch_colstats kind 1, lambda on the
// device) and its MH test with the Langevin q-correction; accepted rows move beta and gl.
// h = lambda p^{-1/6} comes from launch_colstats (h_out). fwd receives the compensated sum
// of (beta' - beta - drift)^2 / D per particle.
cudaError_t launch_propose_mala(const float* beta, const float* gl, float* beta_p, __nv_bfloat16* A, int ldA, int Kp,
                                float2* lpt_p, float2* fwd, const float* D, const float* h, const float* l2e_over_s,
                                const float* mean_f, int64_t N, int p, PriorArgs pr, const double* sched, int t,
                                uint32_t m, const uint64_t* seed, cudaStream_t st);
cudaError_t launch_accept_mala(const AcceptArgs& a, float* gl, const float* gl_p, const float2* fwd, const float* D,
                               const float* h, int64_t N, int p, PriorArgs pr, const double* sched, int t, uint32_t m,
                               const uint64_t* seed, uint32_t* err, cudaStream_t st);
// lambda *= exp(acceptance - 0.574) (MALA step adaptation) and a device scalar store.
cudaError_t launch_adapt_lambda(double* lam, const unsigned long long* acc, double denom, cudaStream_t st);
cudaError_t launch_set_f64(double* ptr, double v, cudaStream_t st);

// logw += log p(beta | c_t) - log p(beta | c_{t-1}); lp refreshed at c_t (without -p log(2c)).
cudaError_t launch_reweight(const float* beta, double* logw, double* lp, int64_t N, int p, PriorArgs pr,
                            const double* sched, int t, uint32_t* err, cudaStream_t st);

// Log-sum-exp and ESS of logw (per-CTA partial (max, sum e, sum e^2) combined in block order
// by the last CTA), then normalisation into W, Wf, wfix.
// mode 0: step t >= 1 (log_z[t] = LSE); 1: prior-IS start (log_z[0] = LSE - log N);
// 2: resample-move start (log_z[0] = LSE - log N, resampling forced, ESS not recorded).
constexpr int LSE_BLOCKS = 128;
constexpr int LSE_SCRATCH = 3 * LSE_BLOCKS + 4;  // doubles
cudaError_t launch_lse_ess(const WeightArrays& w, int64_t N, double* scratch, unsigned int* counter, int t, int mode,
                           double ess_frac, double* ess_out, double* logz_out, uint8_t* resampled_out, int* flag,
                           uint32_t* err, cudaStream_t st);
// Wf and wfix from a given W (for the summaries entry point).
cudaError_t launch_weight_forms(const double* W, int64_t N, float* Wf, uint32_t* wfix, cudaStream_t st);

cudaError_t launch_mark_uniform(int64_t N, int t, double* ess_out, uint8_t* resampled_out, int* flag, cudaStream_t st);

// Systematic resampling: ancestor indices (bit-exact blocked cumulative sum, then a parallel
// binary search), gather of particle rows into scratch and copy back. All no-ops when
// *flag == 0. cum holds N + ceil(N/256) + 1 doubles.
cudaError_t launch_resample_index(const double* W, int64_t N, double* cum, int32_t* idx, const int* flag,
                                  int t, const uint64_t* seed, double u_override, cudaStream_t st);
cudaError_t launch_gather(const int32_t* idx, const float* beta, float* beta_tmp, const double* ll,
                          const double* lp, double* ll_tmp, double* lp_tmp, const float* g, float* g_tmp,
                          int64_t N, int p, const int* flag, cudaStream_t st);
cudaError_t launch_copyback(float* beta, const float* beta_tmp, double* ll, double* lp, const double* ll_tmp,
                            const double* lp_tmp, float* g, const float* g_tmp, const WeightArrays& w, int64_t N,
                            int p, const int* flag, cudaStream_t st);

// Weighted column moments -> per-coordinate proposal scales. kind 0 (RW):
// sigma_j = lam/sqrt(p) max(sd_j, floor c); kind 1 (MALA): D_j = max(var_j, (floor c)^2).
constexpr int COLSTAT_SPLITS = 32;
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
};
cudaError_t launch_summaries(const float* beta, const float* Wf, const uint32_t* wfix, int64_t N, int p,
                             const SummaryArgs& s, int t, double* mean, double* quant, double* conc, cudaStream_t st);

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

// ------------------------------------------------------------ likelihood
// tcgen05 split-BF16 GEMM with the fused log-likelihood reduction: partial[(nt*2 + h)*N_pad + i]
// receives the sum over the h-th half of n-tile nt of y_r eta2 - log2(1 + 2^eta2), eta2 =
// eta log2(e), so that l = ln(2) * (sum of the partials).
struct TcPlan {
    int BN;          // individuals per n-tile (128 or 256)
    int n_tiles;     // ceil(n / BN)
    int m_tiles;     // N_pad / 128
    int kblocks;     // active 64-wide k-blocks of each half
    int ksteps;      // active 16-wide k-steps of each half: ceil((p+1)/16)
    int grid;        // persistent CTAs
    int n_parts;     // partial sums per particle = 2 * n_tiles
};
TcPlan tc_plan(int64_t n, int p, int64_t N_pad, int num_sms);
// Opt the tensor-core kernels into their dynamic shared memory (once per device, before any capture).
cudaError_t tc_init_attributes();
bool tc_make_map_A(CUtensorMap* map, const __nv_bfloat16* A, int64_t N_pad, int Kp);
bool tc_make_map_B(CUtensorMap* map, const __nv_bfloat16* Gbf, int64_t n, int Kp, int BN);
// Residual mode of the likelihood kernel (the adjoint's first half): also writes
// r = y - logit^{-1}(eta) as BF16 hi | lo rows of R [N_pad][2 n_r] and its row sums.
struct ResidArgs {
    __nv_bfloat16* R;        // [N_pad][2 n_r], columns >= n stay zero
    int64_t n_r;             // round_up(n, 64)
    float* rsum_part;        // same layout as the softplus partials
};
// ybits: y as a bitmask, one word per 32 individuals (ceil(n_tiles * BN / 32) words, zero beyond n).
cudaError_t launch_loglik_tc(const CUtensorMap& mapA, const CUtensorMap& mapB, const TcPlan& plan, int64_t n,
                             int Kp, const uint32_t* ybits, float* partial, int64_t N_pad, uint32_t* err, cudaStream_t st,
                             const ResidArgs* resid = nullptr);

// The adjoint's second half: C = R G (tcgen05, split-BF16 R, exact G^T [p][n_r]) into
// gpart[ksplit][N_pad][p], then grad l = (sum C - m_j sum r) / s_j (+ prior gradient).
struct AdjPlan {
    int64_t n_r;
    int kblocks, BN2, p_tiles, m_tiles, ksplit, grid;
};
AdjPlan adj_plan(int p, int64_t n, int64_t N_pad, int num_sms);
bool adj_make_map_R(CUtensorMap* map, const __nv_bfloat16* R, int64_t N_pad, int64_t n_r);
bool adj_make_map_GT(CUtensorMap* map, const __nv_bfloat16* GT, int p, int64_t n_r, int BN2);
cudaError_t launch_adjoint_tc(const CUtensorMap& mapR, const CUtensorMap& mapGT, const AdjPlan& a, int p, float* gpart,
                              int64_t N_pad, uint32_t* err, cudaStream_t st);
cudaError_t launch_grad_finish(const float* gpart, int ksplit, const float* rsum_part, int n_parts, int64_t N_pad,
                               int64_t N, int p, const double* mean, const double* sd, const float* B, PriorArgs pr,
                               double c, float* grad, cudaStream_t st);

// Plain FP32 SIMT path: partial[nt * N_pad + i] = sum over 64-individual tile nt of
// y_r eta_r - softplus(eta_r) (natural units).
constexpr int SIMT_TILE_N = 64;
cudaError_t launch_loglik_simt(const float* beta_p, const float* Xf, const uint8_t* y, int64_t N, int64_t n, int p,
                               float* partial, int64_t N_pad, cudaStream_t st);

// Plain FP32 gradient: eta = B X^T materialised, r = y - logit^{-1}(eta); grad = r X
// (+ prior gradient at c when c > 0); ll = sum y eta - softplus(eta).
cudaError_t launch_grad_simt(const float* B, const float* Xf, const uint8_t* y, int64_t N, int64_t n, int p,
                             float* eta_scratch, float* grad, double* ll, PriorArgs pr, double c, cudaStream_t st);

}  // namespace spa
