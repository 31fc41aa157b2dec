/*
 * spa_oracle.c -- FP64 CPU oracle for the sparsity-path-analysis (SPA) sweep.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg load this library. The product (the
 * CUDA library) never calls it, and the two share no code, headers or constants
 * generators: this file is a plain, slow, index-order restatement of the method of
 * Lee, Caron, Doucet & Holmes, "Bayesian Sparsity-Path-Analysis of Genetic
 * Association Signal using Generalized t Priors" (arXiv:1106.0322).
 *
 * Conventions: everything in double precision; sums run in increasing index
 * order; the only parallelism is an OpenMP loop over particles whose iterations
 * are independent, so results do not depend on the thread count. Build with
 * -ffp-contract=off so no multiply-add is fused behind our back.
 *
 * Parity status of each function (pins live in tests/test_oracle_*.py):
 *   or_philox4x32_10      pinned: published known-answer values of Philox4x32-10
 *   or_prior_logpdf       pinned: quadrature (integrates to 1), tail CDF, moments,
 *                         scale-mixture identity (Section 2, eq. scalemix), DE limit
 *   or_loglik / or_grad   pinned: l(0) = -n log 2, label-flip symmetry, brute-force
 *                         product of Bernoulli probabilities, central differences
 *   or_log_incr_weight    pinned: constant schedule gives 0, telescoping sums
 *   or_lse_ess            pinned: scipy logsumexp, equal / one-hot weights
 *   or_resample_systematic pinned: brute-force definition, count bounds, identity map
 *   or_weighted_quantile  pinned: brute-force definition on small inputs
 *   or_run                pinned: p <= 2 grid quadrature of every pi_t (posterior
 *                         means, quantiles, concentrations) and of Z_t / Z_1
 *   or_map                pinned: the double-exponential case against scikit-learn's L1
 *                         logistic regression; the EM fixed point's optimality (KKT)
 *                         conditions; monotone increase of the EM objective
 *   or_map_path           pinned: for the double exponential (a unique mode) every step's
 *                         MAP is scikit-learn's L1 logistic regression at c_t; for one
 *                         marker with a spike and a slab mode, the kept mode is the global
 *                         maximum of the log posterior on a fine grid at every c_t
 *   or_run's best output  pinned: the recorded particle has the largest l + log p of the
 *                         final particles of a one-step run (brute force)
 *   or_marginal           pinned: equal evidence gives the plain average, one dominant
 *                         step gives its summary, shift invariance of log Z, and the
 *                         p <= 2 quadrature of the scale-marginalised posterior
 *   The paper's own SPA curves cannot pin anything: its figures and data are absent.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Counter-based random numbers: Philox4x32 with 10 rounds (Salmon, Moraes,   */
/* Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).        */
/* One round maps counter (x0,x1,x2,x3) with key (k0,k1) to                   */
/*   (hi(B*x2) ^ x1 ^ k0, lo(B*x2), hi(A*x0) ^ x3 ^ k1, lo(A*x0))             */
/* with multipliers A = 0xD2511F53, B = 0xCD9E8D57; the key is bumped by the   */
/* Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.                    */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prodA = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prodB = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hiA = (uint32_t)(prodA >> 32), loA = (uint32_t)prodA;
        uint32_t hiB = (uint32_t)(prodB >> 32), loB = (uint32_t)prodB;
        uint32_t y0 = hiB ^ x1 ^ k0;
        uint32_t y1 = loB;
        uint32_t y2 = hiA ^ x3 ^ k1;
        uint32_t y3 = loA;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Random-stream layout shared (by specification, not by code) with the GPU path.
 * key = (seed low 32 bits, seed high 32 bits); the counter names the draw:
 *   init prior draws   (j/2, particle, 0, 1<<16)      u[2(j%2)] -> V_j, u[2(j%2)+1] top bit -> sign
 *   move normals       (j/4, particle, t, 2<<16 | m)  Box-Muller pairs (u0,u1), (u2,u3)
 *   MH uniform         (0,   particle, t, 3<<16 | m)  u0
 *   resampling uniform (0,   0,        t, 4<<16)      u0                                   */
enum { OR_TAG_INIT = 1, OR_TAG_NORMAL = 2, OR_TAG_ACCEPT = 3, OR_TAG_RESAMPLE = 4, OR_TAG_SITE = 5 };

static void or_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* Uniform on the open interval (0,1) from the top 23 bits: (k + 1/2) 2^-23, a value
 * that single precision also holds exactly. */
static double or_u01_open(uint32_t u) { return ((double)(u >> 9) + 0.5) * (1.0 / 8388608.0); }
/* Uniform on [0,1) from the top 24 bits. */
static double or_u01(uint32_t u) { return (double)(u >> 8) * (1.0 / 16777216.0); }

/* Four standard normals by the Box-Muller transform of two uniform pairs. */
static void or_normals4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[4])
{
    uint32_t u[4];
    or_draw(seed, c0, c1, c2, c3, u);
    const double two_pi = 6.283185307179586476925286766559;
    for (int h = 0; h < 2; ++h) {
        double u1 = or_u01_open(u[2 * h]);
        double u2 = or_u01_open(u[2 * h + 1]);
        double r = sqrt(-2.0 * log(u1));
        double th = two_pi * u2;
        z[2 * h] = r * cos(th);
        z[2 * h + 1] = r * sin(th);
    }
}

/* Exposed so the tests can compare streams bit for bit with the GPU path. */
void or_normals(uint64_t seed, uint32_t particle, uint32_t t, uint32_t m, int64_t p, double* z)
{
    for (int64_t j = 0; j < p; j += 4) {
        double z4[4];
        or_normals4(seed, (uint32_t)(j / 4), particle, t, ((uint32_t)OR_TAG_NORMAL << 16) | m, z4);
        for (int k = 0; k < 4 && j + k < p; ++k) z[j + k] = z4[k];
    }
}

/* ------------------------------------------------------------------------- */
/* Section 3: columns of X are standardised to mean zero and unit standard    */
/* deviation (population sd, denominator n).                                  */
/* ------------------------------------------------------------------------- */
int or_standardise(const int8_t* G, int64_t n, int64_t p, double* mean, double* sd)
{
    for (int64_t j = 0; j < p; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += (double)G[i * p + j];
        double m = s / (double)n;
        double v = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double d = (double)G[i * p + j] - m;
            v += d * d;
        }
        mean[j] = m;
        sd[j] = sqrt(v / (double)n);
        if (!(sd[j] > 0.0)) return -1;
    }
    return 0;
}

static double* or_make_x(const int8_t* G, int64_t n, int64_t p)
{
    double* mean = (double*)malloc(sizeof(double) * (size_t)p);
    double* sd = (double*)malloc(sizeof(double) * (size_t)p);
    double* X = (double*)malloc(sizeof(double) * (size_t)(n * p));
    if (!mean || !sd || !X || or_standardise(G, n, p, mean, sd) != 0) {
        free(mean); free(sd); free(X);
        return NULL;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < p; ++j)
            X[i * p + j] = ((double)G[i * p + j] - mean[j]) / sd[j];
    free(mean); free(sd);
    return X;
}

/* ------------------------------------------------------------------------- */
/* Section 2: logistic likelihood f(y|X,beta) = prod_i p_i^y_i (1-p_i)^(1-y_i),*/
/* p_i = logit^{-1}(x_i beta), no intercept. Its log is                       */
/*   l(beta) = sum_i [ y_i eta_i - log(1 + exp(eta_i)) ],  eta = X beta,      */
/* with log(1+e^x) evaluated as max(x,0) + log1p(exp(-|x|)).                  */
/* ------------------------------------------------------------------------- */
static double or_softplus(double x) { return (x > 0.0 ? x : 0.0) + log1p(exp(-fabs(x))); }
static double or_sigmoid(double x)
{
    if (x >= 0.0) return 1.0 / (1.0 + exp(-x));
    double e = exp(x);
    return e / (1.0 + e);
}

static double or_loglik_x(const double* X, const uint8_t* y, int64_t n, int64_t p, const double* beta,
                          double* eta_scratch)
{
    double ll = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double eta = 0.0;
        for (int64_t j = 0; j < p; ++j) eta += X[i * p + j] * beta[j];
        if (eta_scratch) eta_scratch[i] = eta;
        ll += (double)y[i] * eta - or_softplus(eta);
    }
    return ll;
}

/* grad l(beta)_j = sum_i x_ij (y_i - logit^{-1}(eta_i)). */
static void or_grad_x(const double* X, const uint8_t* y, int64_t n, int64_t p, const double* eta,
                      double* grad)
{
    for (int64_t j = 0; j < p; ++j) grad[j] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = (double)y[i] - or_sigmoid(eta[i]);
        for (int64_t j = 0; j < p; ++j) grad[j] += X[i * p + j] * r;
    }
}

/* Log-likelihood of N particles B (N x p, particle-major). */
int or_loglik(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, const double* B, int64_t N,
              double* ll_out)
{
    double* X = or_make_x(G, n, p);
    if (!X) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k) ll_out[k] = or_loglik_x(X, y, n, p, B + k * p, NULL);
    free(X);
    return 0;
}

/* Log-likelihood and its gradient for N particles. */
int or_loglik_grad(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, const double* B, int64_t N,
                   double* ll_out, double* grad_out)
{
    double* X = or_make_x(G, n, p);
    if (!X) return -1;
    int fail = 0;
#pragma omp parallel
    {
        double* eta = (double*)malloc(sizeof(double) * (size_t)n);
        if (!eta) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(static)
        for (int64_t k = 0; k < N; ++k) {
            if (!eta) continue;
            ll_out[k] = or_loglik_x(X, y, n, p, B + k * p, eta);
            or_grad_x(X, y, n, p, eta, grad_out + k * p);
        }
        free(eta);
    }
    free(X);
    return fail ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Section 2, eq. gent_prior with q = 1, mu = 0: the centred L1 generalised t  */
/*   Gt(a,c):  p(beta_j) = 1/(2c) (1 + |beta_j|/(a c))^{-(a+1)},              */
/* and its a -> infinity limit, the double exponential p = exp(-|beta|/c)/(2c)*/
/* (Section 5.4). a = +infinity selects the latter.                           */
/* ------------------------------------------------------------------------- */
static double or_logprior1(double a, double c, double b)
{
    double x = fabs(b);
    if (isinf(a)) return -log(2.0 * c) - x / c;
    return -log(2.0 * c) - (a + 1.0) * log1p(x / (a * c));
}

/* d/d beta_j of the log prior; the derivative at 0 is taken as 0. */
static double or_dlogprior1(double a, double c, double b)
{
    double s = (b > 0.0) ? 1.0 : ((b < 0.0) ? -1.0 : 0.0);
    if (isinf(a)) return -s / c;
    return -(a + 1.0) * s / (a * c + fabs(b));
}

void or_prior_logpdf(double a, double c, const double* beta, int64_t k, double* out)
{
    for (int64_t i = 0; i < k; ++i) out[i] = or_logprior1(a, c, beta[i]);
}

static double or_logprior(double a, double c, const double* beta, int64_t p)
{
    double s = 0.0;
    for (int64_t j = 0; j < p; ++j) s += or_logprior1(a, c, beta[j]);
    return s;
}

/* Section 4: with the backward kernel taken as the reversal of K_t, the      */
/* incremental weight is gamma_t(beta)/gamma_{t-1}(beta): the likelihood      */
/* cancels and only the ratio of priors at the two scales is left.            */
double or_log_incr_weight(double a, double c_prev, double c_new, const double* beta, int64_t p)
{
    return or_logprior(a, c_new, beta, p) - or_logprior(a, c_prev, beta, p);
}

/* A draw from Gt(a,c) by inversion: |beta| has tail P(|beta| > x) = (1 + x/(a c))^{-a}
 * (integrate eq. gent_prior), so |beta| = a c (V^{-1/a} - 1) for V uniform on (0,1);
 * for the double exponential |beta| = -c log V. The sign is a fair coin. */
double or_prior_draw(uint64_t seed, uint32_t particle, int64_t j, double a, double c)
{
    uint32_t u[4];
    or_draw(seed, (uint32_t)(j / 2), particle, 0u, (uint32_t)OR_TAG_INIT << 16, u);
    int h = (int)(j % 2);
    double V = or_u01_open(u[2 * h]);
    double mag = isinf(a) ? -c * log(V) : a * c * (pow(V, -1.0 / a) - 1.0);
    return (u[2 * h + 1] >> 31) ? -mag : mag;
}

void or_prior_sample(uint64_t seed, double a, double c, int64_t N, int64_t p, double* out)
{
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < p; ++j) out[i * p + j] = or_prior_draw(seed, (uint32_t)i, j, a, c);
}

/* ------------------------------------------------------------------------- */
/* Weights: log-sum-exp and the effective sample size (Liu & Chen) used for  */
/* the resampling test of Section 4: ESS = (sum W)^2 / sum W^2.               */
/* ------------------------------------------------------------------------- */
void or_lse_ess(const double* logw, int64_t N, double* lse_out, double* ess_out)
{
    double m = -INFINITY;
    for (int64_t i = 0; i < N; ++i)
        if (logw[i] > m) m = logw[i];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double e = exp(logw[i] - m);
        s1 += e;
        s2 += e * e;
    }
    if (lse_out) *lse_out = m + log(s1);
    if (ess_out) *ess_out = (s1 * s1) / s2;
}

/* ------------------------------------------------------------------------- */
/* Systematic resampling. One uniform u in [0,1); the k-th offspring takes    */
/* ancestor A_k = min{ i : C_i > (k+u)/N }, clamped to N-1, where C is the    */
/* cumulative sum of the normalised weights. The cumulative sum is formed in  */
/* a fixed association order so two implementations can agree to the bit:    */
/* blocks of 256 weights in index order, a running sum inside each block, a   */
/* running sum of block totals before it, and C_i = carry(block) + local_i.   */
/* The target is (double)k + u, then divided by (double)N, each correctly     */
/* rounded, with no fused multiply-add.                                       */
/* ------------------------------------------------------------------------- */
void or_cumsum_blocked(const double* W, int64_t N, double* C)
{
    const int64_t B = 256;
    double carry = 0.0;
    for (int64_t b0 = 0; b0 < N; b0 += B) {
        double local = 0.0;
        int64_t b1 = (b0 + B < N) ? b0 + B : N;
        for (int64_t i = b0; i < b1; ++i) {
            local += W[i];
            C[i] = carry + local;
        }
        carry = carry + local;
    }
}

int or_resample_systematic(const double* W, int64_t N, double u, int32_t* idx)
{
    double* C = (double*)malloc(sizeof(double) * (size_t)N);
    if (!C) return -1;
    or_cumsum_blocked(W, N, C);
    int64_t i = 0;
    for (int64_t k = 0; k < N; ++k) {
        volatile double num = (double)k + u;
        double target = num / (double)N;
        while (i < N && !(C[i] > target)) ++i;
        idx[k] = (int32_t)(i < N ? i : N - 1);
        if (i >= N) i = N - 1;  /* stay clamped for the remaining k */
    }
    free(C);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Section 5: weighted quantile of a marginal, Q_q = beta_(k*) with           */
/* k* = min{k : sum_{l<=k} W_(l) >= q} over the values sorted ascending (ties  */
/* by particle index).                                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    double v;
    int64_t i;
} or_pair;

static int or_pair_cmp(const void* a, const void* b)
{
    const or_pair* x = (const or_pair*)a;
    const or_pair* y = (const or_pair*)b;
    if (x->v < y->v) return -1;
    if (x->v > y->v) return 1;
    return (x->i < y->i) ? -1 : (x->i > y->i);
}

static void or_quantiles_sorted(const or_pair* s, const double* W, int64_t N, const double* q, int nq,
                                double* out)
{
    for (int k = 0; k < nq; ++k) {
        double cum = 0.0;
        out[k] = s[N - 1].v;
        for (int64_t l = 0; l < N; ++l) {
            cum += W[s[l].i];
            if (cum >= q[k]) {
                out[k] = s[l].v;
                break;
            }
        }
    }
}

int or_weighted_quantile(const double* vals, const double* W, int64_t N, const double* q, int nq,
                         double* out)
{
    or_pair* s = (or_pair*)malloc(sizeof(or_pair) * (size_t)N);
    if (!s) return -1;
    for (int64_t i = 0; i < N; ++i) {
        s[i].v = vals[i];
        s[i].i = i;
    }
    qsort(s, (size_t)N, sizeof(or_pair), or_pair_cmp);
    or_quantiles_sorted(s, W, N, q, nq, out);
    free(s);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The SMC sampler over the prior scale (Section 4).                          */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t move_kind;      /* 0: joint random-walk Metropolis; 1: MALA; 2: the paper's cycle
                               of single-coordinate random-walk updates */
    int32_t init_mode;      /* 0: prior importance sampling at c_1; 1: the same, then an
                               unconditional resample and burn-in moves at c_1 */
    int32_t burn_in_steps;  /* init_mode 1: blocks of M moves run before step 1's statistics */
    int32_t n_quantiles;
    double quantiles[8];
    int32_t n_deltas;
    double deltas[8];
    double ess_frac;        /* resample when ESS < ess_frac * N (3/4 in the paper) */
    double rw_scale;        /* random walk: sigma_j = rw_scale / sqrt(p) * max(sd_j, sd_floor * c) */
    double mala_h;          /* MALA: h = lambda_t * p^(-1/6), lambda_0 = mala_h, then
                               lambda_{t+1} = lambda_t * exp(acceptance_t - 0.574) */
    double sd_floor;
    double site_sd;         /* single-coordinate moves: proposal sd (0.5, variance 0.25) */
    int32_t n_threads;      /* OpenMP threads; <= 0 keeps the runtime default */
} or_config;

typedef struct {
    double* mean;           /* [T * p] */
    double* quantile;       /* [T * p * n_quantiles] */
    double* conc;           /* [T * p * n_deltas] */
    double* ess;            /* [T] */
    double* log_z_inc;      /* [T] */
    double* accept_rate;    /* [T] */
    uint8_t* resampled;     /* [T] */
    double* final_beta;     /* [N * p], may be NULL */
    double* final_logw;     /* [N], may be NULL */
    double* best;           /* [T * p], may be NULL: after the moves of step t, the particle of
                               highest posterior density l + log p(. | a, c_t) (ties: the
                               lowest index), the start of Section 4.1's MAP tracking */
} or_result;

typedef struct {
    const double* X;
    const uint8_t* y;
    int64_t n, p, N;
    double a;
    uint64_t seed;
    int move_kind;
    double* beta;   /* N x p */
    double* ll;     /* N */
    double* lp;     /* N */
    double* gl;     /* N x p, gradient of the log-likelihood (MALA) */
} or_state;

/* Weighted column mean and variance with normalised weights W. */
static void or_col_moments(const or_state* s, const double* W, double* mu, double* var)
{
    for (int64_t j = 0; j < s->p; ++j) {
        double m = 0.0;
        for (int64_t i = 0; i < s->N; ++i) m += W[i] * s->beta[i * s->p + j];
        double v = 0.0;
        for (int64_t i = 0; i < s->N; ++i) {
            double d = s->beta[i * s->p + j] - m;
            v += W[i] * d * d;
        }
        mu[j] = m;
        var[j] = v;
    }
}

/* The paper's own kernel (Section 4.1, "Further details"): a cycle of single-  */
/* coordinate random-walk Metropolis updates, j = 1..p in order, each proposing  */
/* beta_j' = beta_j + site_sd * xi, the cycle repeated M times. eta = X beta is   */
/* carried along and changed by x_.j * delta when an update is accepted, so one  */
/* update costs O(n). The normal is Box-Muller's cosine branch on the first two  */
/* words of the Philox block (j, particle, t, TAG_SITE << 16 | m); the third word */
/* is the update's uniform. Returns the number of accepted coordinate updates.   */
static int64_t or_site_moves(or_state* s, double c, uint32_t t, uint32_t m0, int32_t M, const or_config* cfg)
{
    const int64_t p = s->p, n = s->n, N = s->N;
    int64_t accepted = 0;
#pragma omp parallel reduction(+ : accepted)
    {
        double* eta = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            double* b = s->beta + i * p;
            or_loglik_x(s->X, s->y, n, p, b, eta);
            for (int32_t mm = 0; mm < M; ++mm) {
                const uint32_t m = m0 + (uint32_t)mm;
                for (int64_t j = 0; j < p; ++j) {
                    uint32_t u[4];
                    or_draw(s->seed, (uint32_t)j, (uint32_t)i, t, ((uint32_t)OR_TAG_SITE << 16) | m, u);
                    const double z = sqrt(-2.0 * log(or_u01_open(u[0]))) *
                                     cos(6.283185307179586476925286766559 * or_u01_open(u[1]));
                    const double delta = cfg->site_sd * z;
                    const double bn = b[j] + delta;
                    double dl = 0.0;
                    for (int64_t r = 0; r < n; ++r) {
                        const double x = s->X[r * p + j];
                        const double e0 = eta[r], e1 = e0 + x * delta;
                        dl += (double)s->y[r] * x * delta - (or_softplus(e1) - or_softplus(e0));
                    }
                    const double dlp = or_logprior1(s->a, c, bn) - or_logprior1(s->a, c, b[j]);
                    if (log(or_u01_open(u[2])) < dl + dlp) {
                        b[j] = bn;
                        for (int64_t r = 0; r < n; ++r) eta[r] += s->X[r * p + j] * delta;
                        ++accepted;
                    }
                }
            }
            s->ll[i] = or_loglik_x(s->X, s->y, n, p, b, eta);
            s->lp[i] = or_logprior(s->a, c, b, p);
        }
        free(eta);
    }
    return accepted;
}

/* M moves of an MCMC kernel with invariant distribution pi_t (Section 4.1)  */
/* applied to every particle; returns the number of accepted proposals.      */
static int64_t or_moves(or_state* s, double c, uint32_t t, uint32_t m0, int32_t M, const double* W,
                        const or_config* cfg, double lam)
{
    if (s->move_kind == 2) return or_site_moves(s, c, t, m0, M, cfg);
    const int64_t p = s->p, n = s->n, N = s->N;
    double* mu = (double*)malloc(sizeof(double) * (size_t)p);
    double* var = (double*)malloc(sizeof(double) * (size_t)p);
    double* scale = (double*)malloc(sizeof(double) * (size_t)p);
    uint8_t* acc = (uint8_t*)calloc((size_t)N, 1);
    int64_t accepted = 0;
    or_col_moments(s, W, mu, var);
    const double floor_sd = cfg->sd_floor * c;
    const double h = lam * pow((double)p, -1.0 / 6.0);
    for (int64_t j = 0; j < p; ++j) {
        double sd = sqrt(var[j]);
        if (s->move_kind == 0)
            scale[j] = lam / sqrt((double)p) * (sd > floor_sd ? sd : floor_sd);
        else
            scale[j] = (var[j] > floor_sd * floor_sd) ? var[j] : floor_sd * floor_sd;  /* D_j */
    }
    for (int32_t mm = 0; mm < M; ++mm) {
        const uint32_t m = m0 + (uint32_t)mm;
#pragma omp parallel
        {
            double* z = (double*)malloc(sizeof(double) * (size_t)p);
            double* bp = (double*)malloc(sizeof(double) * (size_t)p);
            double* glp = (double*)malloc(sizeof(double) * (size_t)p);
            double* eta = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(static)
            for (int64_t i = 0; i < N; ++i) {
                double* b = s->beta + i * p;
                or_normals(s->seed, (uint32_t)i, t, m, p, z);
                double log_alpha;
                double llp, lpp;
                if (s->move_kind == 0) {
                    /* joint random walk: beta' = beta + sigma * xi */
                    for (int64_t j = 0; j < p; ++j) bp[j] = b[j] + scale[j] * z[j];
                    llp = or_loglik_x(s->X, s->y, n, p, bp, NULL);
                    lpp = or_logprior(s->a, c, bp, p);
                    log_alpha = (llp + lpp) - (s->ll[i] + s->lp[i]);
                } else {
                    /* MALA: beta' = beta + (h^2/2) D grad log pi_t(beta) + h D^{1/2} xi */
                    const double* gl = s->gl + i * p;
                    double fwd = 0.0, bwd = 0.0;
                    for (int64_t j = 0; j < p; ++j) {
                        double g = gl[j] + or_dlogprior1(s->a, c, b[j]);
                        double mean = b[j] + 0.5 * h * h * scale[j] * g;
                        bp[j] = mean + h * sqrt(scale[j]) * z[j];
                        double d = bp[j] - mean;
                        fwd += d * d / scale[j];
                    }
                    llp = or_loglik_x(s->X, s->y, n, p, bp, eta);
                    or_grad_x(s->X, s->y, n, p, eta, glp);
                    lpp = or_logprior(s->a, c, bp, p);
                    for (int64_t j = 0; j < p; ++j) {
                        double g = glp[j] + or_dlogprior1(s->a, c, bp[j]);
                        double mean = bp[j] + 0.5 * h * h * scale[j] * g;
                        double d = b[j] - mean;
                        bwd += d * d / scale[j];
                    }
                    /* log q(beta|beta') - log q(beta'|beta) */
                    log_alpha = (llp + lpp) - (s->ll[i] + s->lp[i]) - (bwd - fwd) / (2.0 * h * h);
                }
                uint32_t u[4];
                or_draw(s->seed, 0u, (uint32_t)i, t, ((uint32_t)OR_TAG_ACCEPT << 16) | m, u);
                if (log(or_u01_open(u[0])) < log_alpha) {
                    for (int64_t j = 0; j < p; ++j) b[j] = bp[j];
                    if (s->move_kind == 1)
                        for (int64_t j = 0; j < p; ++j) s->gl[i * p + j] = glp[j];
                    s->ll[i] = llp;
                    s->lp[i] = lpp;
                    acc[i] = 1;
                } else {
                    acc[i] = 0;
                }
            }
            free(z); free(bp); free(glp); free(eta);
        }
        for (int64_t i = 0; i < N; ++i) accepted += acc[i];
    }
    free(mu); free(var); free(scale); free(acc);
    return accepted;
}

static void or_summaries(const or_state* s, const double* W, const or_config* cfg, int64_t t, or_result* r)
{
    const int64_t p = s->p, N = s->N;
    const int nq = cfg->n_quantiles, nd = cfg->n_deltas;
#pragma omp parallel
    {
        or_pair* srt = (or_pair*)malloc(sizeof(or_pair) * (size_t)N);
#pragma omp for schedule(static)
        for (int64_t j = 0; j < p; ++j) {
            if (r->mean) {
                double m = 0.0;
                for (int64_t i = 0; i < N; ++i) m += W[i] * s->beta[i * p + j];
                r->mean[t * p + j] = m;
            }
            if (r->conc) {
                /* V(c) = 1 - Pr(beta_j in (-Delta, Delta)) (Section 5.1 (d)) */
                for (int d = 0; d < nd; ++d) {
                    double inside = 0.0;
                    for (int64_t i = 0; i < N; ++i)
                        if (fabs(s->beta[i * p + j]) < cfg->deltas[d]) inside += W[i];
                    r->conc[(t * p + j) * nd + d] = 1.0 - inside;
                }
            }
            if (r->quantile && nq > 0) {
                for (int64_t i = 0; i < N; ++i) {
                    srt[i].v = s->beta[i * p + j];
                    srt[i].i = i;
                }
                qsort(srt, (size_t)N, sizeof(or_pair), or_pair_cmp);
                or_quantiles_sorted(srt, W, N, cfg->quantiles, nq, r->quantile + (t * p + j) * nq);
            }
        }
        free(srt);
    }
}

/* Normalise log-weights in place (sum exp = 1); return the log of the sum. */
static double or_normalise(double* logw, double* W, int64_t N, double* ess)
{
    double lse;
    or_lse_ess(logw, N, &lse, ess);
    for (int64_t i = 0; i < N; ++i) {
        logw[i] -= lse;
        W[i] = exp(logw[i]);
    }
    return lse;
}

static int or_resample_state(or_state* s, double* logw, double* W, uint32_t t)
{
    const int64_t N = s->N, p = s->p;
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    double* nb = (double*)malloc(sizeof(double) * (size_t)(N * p));
    double* ng = (s->move_kind == 1) ? (double*)malloc(sizeof(double) * (size_t)(N * p)) : NULL;
    double* nll = (double*)malloc(sizeof(double) * (size_t)N);
    double* nlp = (double*)malloc(sizeof(double) * (size_t)N);
    if (!idx || !nb || !nll || !nlp || (s->move_kind == 1 && !ng)) {
        free(idx); free(nb); free(ng); free(nll); free(nlp);
        return -1;
    }
    uint32_t u[4];
    or_draw(s->seed, 0u, 0u, t, (uint32_t)OR_TAG_RESAMPLE << 16, u);
    or_resample_systematic(W, N, or_u01(u[0]), idx);
    for (int64_t k = 0; k < N; ++k) {
        int64_t a = idx[k];
        memcpy(nb + k * p, s->beta + a * p, sizeof(double) * (size_t)p);
        if (ng) memcpy(ng + k * p, s->gl + a * p, sizeof(double) * (size_t)p);
        nll[k] = s->ll[a];
        nlp[k] = s->lp[a];
    }
    memcpy(s->beta, nb, sizeof(double) * (size_t)(N * p));
    if (ng) memcpy(s->gl, ng, sizeof(double) * (size_t)(N * p));
    memcpy(s->ll, nll, sizeof(double) * (size_t)N);
    memcpy(s->lp, nlp, sizeof(double) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) {
        logw[i] = -log((double)N);
        W[i] = 1.0 / (double)N;
    }
    free(idx); free(nb); free(ng); free(nll); free(nlp);
    return 0;
}

/*
 * Run the SPA sweep: targets pi_t(beta) = p(beta | X, y, a, c_t), t = 0..T-1.
 *   t = 0: particles from the prior Gt(a, c_0) by inversion of its tail
 *          P(|beta| > x) = (1 + x/(a c))^{-a}, weighted by the likelihood
 *          (importance sampling, log Z_0 estimate = LSE(l) - log N); with
 *          init_mode 1 they are then resampled and moved for burn_in_steps blocks
 *          of M moves at c_0 (Section 4.1 starts from MCMC draws at pi_1).
 *   t >= 1: reweight by the prior ratio, estimate Z_t/Z_{t-1} = sum_i W_{t-1} w_t,
 *          normalise (eq. normalize_weights).
 *   every t: resample if ESS < ess_frac * N, then M moves at c_t (resampling
 *          before moving, Section 4), then the per-scale summaries of Section 5.
 * Returns 0, or -1 on bad input / allocation failure.
 */
int or_run(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, double a, const double* sched,
           int64_t T, int64_t N, int32_t M, uint64_t seed, const or_config* cfg, or_result* r)
{
    if (n < 1 || p < 1 || N < 1 || T < 1 || M < 0 || !(a > 0.0)) return -1;
    if (cfg->move_kind < 0 || cfg->move_kind > 2) return -1;
    for (int64_t t = 0; t < T; ++t)
        if (!(sched[t] > 0.0) || isinf(sched[t])) return -1;
#ifdef _OPENMP
    if (cfg->n_threads > 0) omp_set_num_threads(cfg->n_threads);
#endif
    double* X = or_make_x(G, n, p);
    if (!X) return -1;
    or_state s;
    s.X = X; s.y = y; s.n = n; s.p = p; s.N = N; s.a = a; s.seed = seed; s.move_kind = cfg->move_kind;
    s.beta = (double*)malloc(sizeof(double) * (size_t)(N * p));
    s.ll = (double*)malloc(sizeof(double) * (size_t)N);
    s.lp = (double*)malloc(sizeof(double) * (size_t)N);
    s.gl = (cfg->move_kind == 1) ? (double*)malloc(sizeof(double) * (size_t)(N * p)) : NULL;
    double* logw = (double*)malloc(sizeof(double) * (size_t)N);
    double* W = (double*)malloc(sizeof(double) * (size_t)N);
    if (!s.beta || !s.ll || !s.lp || !logw || !W || (cfg->move_kind == 1 && !s.gl)) {
        free(X); free(s.beta); free(s.ll); free(s.lp); free(s.gl); free(logw); free(W);
        return -1;
    }

    /* t = 0: draws from the prior Gt(a, c_0) (or the double exponential). */
    const double c0 = sched[0];
#pragma omp parallel
    {
        double* eta = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            double* b = s.beta + i * p;
            for (int64_t j = 0; j < p; ++j) b[j] = or_prior_draw(seed, (uint32_t)i, j, a, c0);
            s.ll[i] = or_loglik_x(X, y, n, p, b, eta);
            s.lp[i] = or_logprior(a, c0, b, p);
            if (s.gl) or_grad_x(X, y, n, p, eta, s.gl + i * p);
        }
        free(eta);
    }
    uint32_t m_base = 0;
    double ess;
    /* Proposal scale multiplier: fixed for the random walk; for MALA it follows the
     * acceptance rate of the previous block of moves towards 0.574. It depends only on
     * moves already made, so each step's kernel is still pi_t-invariant. */
    double lam = (cfg->move_kind == 0) ? cfg->rw_scale : cfg->mala_h;
    /* importance weights of the prior draws: the likelihood; their mean estimates Z_0 */
    for (int64_t i = 0; i < N; ++i) logw[i] = s.ll[i];
    double lse0 = or_normalise(logw, W, N, &ess);
    if (r->log_z_inc) r->log_z_inc[0] = lse0 - log((double)N);
    if (cfg->init_mode == 1) {
        /* resample-move start (Section 4.1 asks for draws from a long MCMC run at pi_1):
         * resample the weighted prior draws, then burn_in_steps blocks of M moves. */
        if (or_resample_state(&s, logw, W, 0u) != 0) {
            free(X); free(s.beta); free(s.ll); free(s.lp); free(s.gl); free(logw); free(W);
            return -1;
        }
        for (int32_t b = 0; b < cfg->burn_in_steps; ++b) {
            int64_t acc = or_moves(&s, c0, 0u, m_base, M, W, cfg, lam);
            if (cfg->move_kind == 1 && M > 0) lam *= exp((double)acc / ((double)M * (double)N) - 0.574);
            m_base += (uint32_t)M;
        }
        ess = (double)N;
    }

    int rc = 0;
    for (int64_t t = 0; t < T; ++t) {
        const double c = sched[t];
        if (t > 0) {
            const double cp = sched[t - 1];
            /* reweight: w_t = gamma_t(beta_{t-1}) / gamma_{t-1}(beta_{t-1}) */
            for (int64_t i = 0; i < N; ++i) {
                logw[i] += or_log_incr_weight(a, cp, c, s.beta + i * p, p);
                s.lp[i] = or_logprior(a, c, s.beta + i * p, p);
            }
            /* previous logw are normalised, so LSE is the log of sum_i W_{t-1} w_t */
            double lse = or_normalise(logw, W, N, &ess);
            if (r->log_z_inc) r->log_z_inc[t] = lse;
        }
        if (r->ess) r->ess[t] = ess;
        int do_res = ess < cfg->ess_frac * (double)N;
        if (r->resampled) r->resampled[t] = (uint8_t)do_res;
        if (do_res && or_resample_state(&s, logw, W, (uint32_t)t) != 0) {
            rc = -1;
            break;
        }
        int64_t acc = or_moves(&s, c, (uint32_t)t, (t == 0) ? m_base : 0u, M, W, cfg, lam);
        /* the acceptance rate per proposal: per coordinate update for the cycle kernel */
        const double props = (double)M * (double)N * (cfg->move_kind == 2 ? (double)p : 1.0);
        double rate = (M > 0) ? (double)acc / props : 0.0;
        if (r->accept_rate) r->accept_rate[t] = rate;
        if (cfg->move_kind == 1 && M > 0) lam *= exp(rate - 0.574);
        or_summaries(&s, W, cfg, t, r);
        if (r->best) {
            int64_t k = 0;
            for (int64_t i = 1; i < N; ++i)
                if (s.ll[i] + s.lp[i] > s.ll[k] + s.lp[k]) k = i;
            memcpy(r->best + t * p, s.beta + k * p, sizeof(double) * (size_t)p);
        }
    }
    if (r->final_beta) memcpy(r->final_beta, s.beta, sizeof(double) * (size_t)(N * p));
    if (r->final_logw) memcpy(r->final_logw, logw, sizeof(double) * (size_t)N);
    free(X); free(s.beta); free(s.ll); free(s.lp); free(s.gl); free(logw); free(W);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Scale-marginalised summaries (Section 4, eq. all_particles): with a uniform   */
/* prior on log b and the log-spaced schedule, the particle systems of all steps */
/* are mixed with weights Z_t / Z_1, each estimated by the running product of    */
/* the Z_t / Z_{t-1} estimates. Step t's weight is                               */
/*   w_t = exp(L_t - max L) / sum_s exp(L_s - max L),  L_t = sum_{s=1..t} inc_s   */
/* (inc_0, the t = 0 evidence, is common to every L_t and is left out). Mixture  */
/* means and concentrations are the w-weighted averages of the per-step ones;    */
/* post_c[t] = w_t is the posterior of the scale on the schedule's grid.         */
/* ------------------------------------------------------------------------- */
int or_marginal(const double* log_z_inc, const double* mean, const double* conc, int64_t T, int64_t p, int D,
                double* post_c, double* mean_out, double* conc_out)
{
    if (T < 1 || p < 1 || D < 0) return -1;
    double* L = (double*)malloc(sizeof(double) * (size_t)T);
    if (!L) return -1;
    double acc = 0.0, m = -INFINITY;
    for (int64_t t = 0; t < T; ++t) {
        if (t > 0) acc += log_z_inc[t];
        L[t] = acc;
        if (L[t] > m) m = L[t];
    }
    double s = 0.0;
    for (int64_t t = 0; t < T; ++t) s += exp(L[t] - m);
    for (int64_t t = 0; t < T; ++t) post_c[t] = exp(L[t] - m) / s;
    for (int64_t j = 0; j < p; ++j) {
        double mm = 0.0;
        for (int64_t t = 0; t < T; ++t) mm += post_c[t] * mean[t * p + j];
        mean_out[j] = mm;
        for (int d = 0; d < D; ++d) {
            double cc = 0.0;
            for (int64_t t = 0; t < T; ++t) cc += post_c[t] * conc[(t * p + j) * D + d];
            conc_out[j * D + d] = cc;
        }
    }
    free(L);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* MAP by EM (Section 2.1, eqs. beta_it and adapt_weights). The scale-mixture   */
/* representation makes each EM step a weighted-L1 logistic regression:         */
/*   w_j = (a+1) / (a c + |beta_j|)      (double exponential, a = inf: 1/c)     */
/*   beta <- argmax_beta l(beta) - sum_j w_j |beta_j|                           */
/* repeated from beta0 until the largest change is below tol (or max_em steps). */
/* The convex inner problem is solved by cyclic coordinate descent on the       */
/* quadratic majorizer of the logistic loss (its second derivative along a      */
/* standardised column is at most sum_i x_ij^2 / 4): each coordinate step       */
/*   beta_j <- S(beta_j + g_j / L_j, w_j / L_j),  S(u, k) = sign(u) max(|u|-k, 0) */
/* with g_j the gradient of l at the current point, decreases the objective, and */
/* sweeps run until no coordinate moves by more than 1e-13.                     */
/* Writes the mode to beta_out and log l(beta) + log p(beta | a, c) to logpost. */
/* ------------------------------------------------------------------------- */
int or_map(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, double a, double c, const double* beta0,
           int32_t max_em, double tol, double* beta_out, double* logpost)
{
    if (n < 1 || p < 1 || !(a > 0.0) || !(c > 0.0) || max_em < 1) return -1;
    double* X = or_make_x(G, n, p);
    if (!X) return -1;
    double* eta = (double*)malloc(sizeof(double) * (size_t)n);
    double* w = (double*)malloc(sizeof(double) * (size_t)p);
    double* L = (double*)malloc(sizeof(double) * (size_t)p);
    double* prev = (double*)malloc(sizeof(double) * (size_t)p);
    if (!eta || !w || !L || !prev) {
        free(X); free(eta); free(w); free(L); free(prev);
        return -1;
    }
    double* b = beta_out;
    for (int64_t j = 0; j < p; ++j) {
        b[j] = beta0[j];
        double s2 = 0.0;
        for (int64_t i = 0; i < n; ++i) s2 += X[i * p + j] * X[i * p + j];
        L[j] = 0.25 * s2;
    }
    for (int64_t i = 0; i < n; ++i) {
        double e = 0.0;
        for (int64_t j = 0; j < p; ++j) e += X[i * p + j] * b[j];
        eta[i] = e;
    }
    for (int32_t em = 0; em < max_em; ++em) {
        for (int64_t j = 0; j < p; ++j) {
            w[j] = isinf(a) ? 1.0 / c : (a + 1.0) / (a * c + fabs(b[j]));
            prev[j] = b[j];
        }
        for (int sweep = 0; sweep < 200000; ++sweep) {
            double moved = 0.0;
            for (int64_t j = 0; j < p; ++j) {
                double g = 0.0;
                for (int64_t i = 0; i < n; ++i) g += X[i * p + j] * ((double)y[i] - or_sigmoid(eta[i]));
                const double u = b[j] + g / L[j], k = w[j] / L[j];
                const double nb = (u > k) ? u - k : ((u < -k) ? u + k : 0.0);
                const double d = nb - b[j];
                if (d != 0.0) {
                    for (int64_t i = 0; i < n; ++i) eta[i] += X[i * p + j] * d;
                    b[j] = nb;
                }
                if (fabs(d) > moved) moved = fabs(d);
            }
            if (moved < 1e-13) break;
        }
        double change = 0.0;
        for (int64_t j = 0; j < p; ++j)
            if (fabs(b[j] - prev[j]) > change) change = fabs(b[j] - prev[j]);
        if (change < tol) break;
    }
    if (logpost) *logpost = or_loglik_x(X, y, n, p, b, NULL) + or_logprior(a, c, b, p);
    free(X); free(eta); free(w); free(L); free(prev);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The MAP path along a sweep (Section 4.1): at every step t the EM of Section   */
/* 2.1 is started from the step's particle of highest posterior density and,    */
/* for t > 0, from the previous step's MAP; the mode with the higher log        */
/* posterior is kept (on a tie, the one from the best particle). This walks the  */
/* steps in order:                                                               */
/*   A_t = EM(c_t, best_t),  S_0 = A_0,                                          */
/*   S_t = EM(c_t, S_{t-1}) if its log posterior exceeds A_t's, else A_t.        */
/* best: [T * p] starts; map_out [T * p] the kept modes, logpost [T] their       */
/* log l + log p, chained [T] (may be NULL) 1 where EM from S_{t-1} was kept.    */
/* ------------------------------------------------------------------------- */
int or_map_path(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, double a, const double* sched, int64_t T,
                const double* best, int32_t max_em, double tol, double* map_out, double* logpost, uint8_t* chained)
{
    if (T < 1) return -1;
    double* B = (double*)malloc(sizeof(double) * (size_t)p);
    if (!B) return -1;
    int rc = 0;
    for (int64_t t = 0; t < T && rc == 0; ++t) {
        double* S = map_out + t * p;
        double lpA = 0.0, lpB = 0.0;
        rc = or_map(G, y, n, p, a, sched[t], best + t * p, max_em, tol, S, &lpA);
        if (rc != 0) break;
        logpost[t] = lpA;
        if (chained) chained[t] = 0;
        if (t == 0) continue;
        rc = or_map(G, y, n, p, a, sched[t], map_out + (t - 1) * p, max_em, tol, B, &lpB);
        if (rc == 0 && lpB > lpA) {
            memcpy(S, B, sizeof(double) * (size_t)p);
            logpost[t] = lpB;
            if (chained) chained[t] = 1;
        }
    }
    free(B);
    return rc;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
