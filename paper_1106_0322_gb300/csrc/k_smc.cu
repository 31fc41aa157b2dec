// k_smc.cu -- the per-step kernels of the SMC sampler over the prior scale (Section 4).
//
// Particle state: beta [N][p] FP32 (particle-major), log-likelihood ll[N] and log prior
// lp[N] in FP64, normalised log-weights logw[N] and weights W[N] in FP64. FP64 is used
// for the weight arithmetic (log-sum-exp, ESS, log-evidence, resampling sums) and for
// row sums of FP32 terms; everything per (particle, marker) is FP32.
#include <cfloat>

#include "spa_device.cuh"
#include "spa_internal.h"

namespace spa {

namespace {

constexpr int WARPS_PER_BLOCK = 8;

__device__ __forceinline__ int64_t warp_global_id()
{
    return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

// log prior of one coordinate without the -log(2c) constant, in "row-sum units":
// Gt: log1p(|b|/(a c)) (multiplied by -(a+1) later); DE: |b| (multiplied by -1/c later).
__device__ __forceinline__ float prior_term(float b, float ac, int de)
{
    const float x = fabsf(b);
    return de ? x : log1pf(x / ac);
}
__device__ __forceinline__ double prior_from_terms(double terms, int p, double a, double c, int de)
{
    return -(double)p * log(2.0 * c) - (de ? terms / c : (a + 1.0) * terms);
}

// ------------------------------------------------------------------- init (t = 0)
__global__ void k_init_prior(float* __restrict__ beta, int64_t N, int p, PriorArgs pr, const double* __restrict__ sched,
                             int t0, const uint64_t* __restrict__ seedp)
{
    const uint64_t seed = *seedp;
    const float c = (float)sched[t0];
    const int64_t total = N * (int64_t)p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / p;
        const int j = (int)(e - i * p);
        beta[e] = prior_draw(seed, (uint32_t)i, (uint32_t)j, pr.a, c, pr.de != 0);
    }
}

// ------------------------------------------------------------ RW proposal / pack
// One warp per particle; lane l handles the 4-coordinate groups g = l, l+32, ... (one
// Philox block of four normals each).
__global__ void __launch_bounds__(256) k_propose_rw(const float* __restrict__ beta, float* __restrict__ beta_p,
                                                   __nv_bfloat16* __restrict__ A, int ldA, int Kp,
                                                   double* __restrict__ lin_p, double* __restrict__ lp_p,
                                                   const float* __restrict__ sigma, const float* __restrict__ l2e_over_s,
                                                   const float* __restrict__ mean_f, const double* __restrict__ v, int64_t N,
                                                   int p, PriorArgs pr, const double* __restrict__ sched, int t, uint32_t m,
                                                   const uint64_t* __restrict__ seedp, int noise)
{
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const uint64_t seed = noise ? *seedp : 0ull;
    const double c = sched[t];
    const float ac = (float)((double)pr.a * c);
    const float* row = beta + i * p;
    float* rowp = beta_p + i * p;
    double lin = 0.0, lterm = 0.0, off = 0.0;
    const int groups = (p + 3) >> 2;
    for (int g = lane; g < groups; g += 32) {
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (noise) {
            const float4 z4 = normals4(seed, (uint32_t)g, (uint32_t)i, (uint32_t)t, m);
            z[0] = z4.x; z[1] = z4.y; z[2] = z4.z; z[3] = z4.w;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = 4 * g + k;
            if (j < p) {
                const float b = noise ? row[j] + sigma[j] * z[k] : row[j];
                rowp[j] = b;
                lin += (double)b * v[j];
                lterm += (double)prior_term(b, ac, pr.de);
                if (A) {
                    const float bt = b * l2e_over_s[j];
                    __nv_bfloat16 hi, lo;
                    split_bf16(bt, hi, lo);
                    A[i * ldA + j] = hi;
                    A[i * ldA + Kp + j] = lo;
                    off += (double)mean_f[j] * (double)bt;
                }
            }
        }
    }
    lin = warp_sum(lin);
    lterm = warp_sum(lterm);
    off = warp_sum(off);
    if (lane == 0) {
        lin_p[i] = lin;
        lp_p[i] = prior_from_terms(lterm, p, (double)pr.a, c, pr.de);
        if (A) {
            __nv_bfloat16 hi, lo;
            split_bf16((float)(-off), hi, lo);
            A[i * ldA + p] = hi;
            A[i * ldA + Kp + p] = lo;
        }
    }
}

// ----------------------------------------------------------------- MALA proposal
// beta' = beta + (h^2/2) D grad log pi_t(beta) + h D^{1/2} xi with D = diag(D_j) and
// h = lambda p^{-1/6}; grad log pi_t = grad l (stored per particle) + the prior gradient
// -(a+1) sgn(beta)/(a c + |beta|) (double exponential: -sgn(beta)/c). Also stores
// sum_j xi_j^2, since log q(beta'|beta) = -sum_j xi_j^2 / 2 + const.
__device__ __forceinline__ float dlogprior(float b, float a1, float ac, float inv_c, int de)
{
    const float sg = (b > 0.0f) ? 1.0f : ((b < 0.0f) ? -1.0f : 0.0f);
    return de ? -sg * inv_c : -a1 * sg / (ac + fabsf(b));
}

__global__ void __launch_bounds__(256) k_propose_mala(const float* __restrict__ beta, const float* __restrict__ gl,
                                                     float* __restrict__ beta_p, __nv_bfloat16* __restrict__ A, int ldA,
                                                     int Kp, double* __restrict__ lin_p, double* __restrict__ lp_p,
                                                     double* __restrict__ xi2, const float* __restrict__ D,
                                                     const double* __restrict__ lam, const float* __restrict__ l2e_over_s,
                                                     const float* __restrict__ mean_f, const double* __restrict__ v,
                                                     int64_t N, int p, PriorArgs pr, const double* __restrict__ sched,
                                                     int t, uint32_t m, const uint64_t* __restrict__ seedp)
{
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const uint64_t seed = *seedp;
    const double c = sched[t];
    const float ac = (float)((double)pr.a * c), a1 = pr.a + 1.0f, inv_c = (float)(1.0 / c);
    const double hd = *lam * pow((double)p, -1.0 / 6.0);
    const float h = (float)hd, h2 = (float)(0.5 * hd * hd);
    const float* row = beta + i * p;
    const float* grow = gl + i * p;
    float* rowp = beta_p + i * p;
    double lin = 0.0, lterm = 0.0, off = 0.0, zz = 0.0;
    const int groups = (p + 3) >> 2;
    for (int g = lane; g < groups; g += 32) {
        const float4 z4 = normals4(seed, (uint32_t)g, (uint32_t)i, (uint32_t)t, m);
        const float z[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = 4 * g + k;
            if (j < p) {
                const float b0 = row[j];
                const float grad = grow[j] + dlogprior(b0, a1, ac, inv_c, pr.de);
                const float Dj = D[j];
                const float b = b0 + h2 * Dj * grad + h * sqrtf(Dj) * z[k];
                rowp[j] = b;
                zz += (double)z[k] * (double)z[k];
                lin += (double)b * v[j];
                lterm += (double)prior_term(b, ac, pr.de);
                if (A) {
                    const float bt = b * l2e_over_s[j];
                    __nv_bfloat16 hi, lo;
                    split_bf16(bt, hi, lo);
                    A[i * ldA + j] = hi;
                    A[i * ldA + Kp + j] = lo;
                    off += (double)mean_f[j] * (double)bt;
                }
            }
        }
    }
    lin = warp_sum(lin);
    lterm = warp_sum(lterm);
    off = warp_sum(off);
    zz = warp_sum(zz);
    if (lane == 0) {
        lin_p[i] = lin;
        lp_p[i] = prior_from_terms(lterm, p, (double)pr.a, c, pr.de);
        xi2[i] = zz;
        if (A) {
            __nv_bfloat16 hi, lo;
            split_bf16((float)(-off), hi, lo);
            A[i * ldA + p] = hi;
            A[i * ldA + Kp + p] = lo;
        }
    }
}

// MH test of a MALA proposal: log alpha = l' + lp' - l - lp + log q(beta|beta') - log q(beta'|beta),
// log q(beta|beta') = -sum_j (beta_j - beta'_j - (h^2/2) D_j g'_j)^2 / (2 h^2 D_j),
// log q(beta'|beta) = -sum_j xi_j^2 / 2. On acceptance the state and its gradient move.
__global__ void __launch_bounds__(256) k_accept_mala(AcceptArgs a, float* __restrict__ gl, const float* __restrict__ gl_p,
                                                    const double* __restrict__ xi2, const float* __restrict__ D,
                                                    const double* __restrict__ lam, int64_t N, int p, PriorArgs pr,
                                                    const double* __restrict__ sched, int t, uint32_t m,
                                                    const uint64_t* __restrict__ seedp, uint32_t* __restrict__ err)
{
    __shared__ unsigned int block_acc;
    if (threadIdx.x == 0) block_acc = 0;
    __syncthreads();
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    if (i < N) {
        const double c = sched[t];
        const float ac = (float)((double)pr.a * c), a1 = pr.a + 1.0f, inv_c = (float)(1.0 / c);
        const double hd = *lam * pow((double)p, -1.0 / 6.0);
        const float h2 = (float)(0.5 * hd * hd);
        const float* b0 = a.beta + i * p;
        const float* b1 = a.beta_p + i * p;
        const float* g1 = gl_p + i * p;
        double bwd = 0.0;
        for (int j = lane; j < p; j += 32) {
            const float gp = g1[j] + dlogprior(b1[j], a1, ac, inv_c, pr.de);
            const float d = b0[j] - b1[j] - h2 * D[j] * gp;
            bwd += (double)d * (double)d / (double)D[j];
        }
        bwd = warp_sum(bwd);
        int accept = 0;
        if (lane == 0) {
            double sp = 0.0;
            for (int s = 0; s < a.n_parts; ++s) sp += (double)a.partial[(int64_t)s * a.ld_part + i];
            const double llp = a.lin_p[i] - a.sp_scale * sp;
            if (!isfinite(llp)) atomicOr(err, DERR_NONFINITE);
            const double log_alpha =
                (llp + a.lp_p[i]) - (a.ll[i] + a.lp[i]) - bwd / (2.0 * hd * hd) + 0.5 * xi2[i];
            const uint4 u = philox4x32_10(make_uint4(0u, (uint32_t)i, (uint32_t)t, (TAG_ACCEPT << 16) | m),
                                          seed_key(*seedp));
            accept = log(u01_open_d(u.x)) < log_alpha;
            if (accept) {
                a.ll[i] = llp;
                a.lp[i] = a.lp_p[i];
            }
        }
        accept = __shfl_sync(0xffffffffu, accept, 0);
        if (accept) {
            float* dst = a.beta + i * p;
            float* gdst = gl + i * p;
            for (int j = lane; j < p; j += 32) {
                dst[j] = b1[j];
                gdst[j] = g1[j];
            }
            if (lane == 0) atomicAdd(&block_acc, 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && block_acc && a.acc_count) atomicAdd(a.acc_count, (unsigned long long)block_acc);
}

// --------------------------------------------------------------- finish / MH test
__global__ void __launch_bounds__(256) k_accept(AcceptArgs a, int64_t N, int p, int mode, int t, uint32_t m,
                                                const uint64_t* __restrict__ seedp, uint32_t* __restrict__ err)
{
    __shared__ unsigned int block_acc;
    if (threadIdx.x == 0) block_acc = 0;
    __syncthreads();
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    int accept = 0;
    if (i < N) {
        double llp = 0.0;
        if (lane == 0) {
            double sp = 0.0;
            for (int s = 0; s < a.n_parts; ++s) sp += (double)a.partial[(int64_t)s * a.ld_part + i];
            llp = a.lin_p[i] - a.sp_scale * sp;
            if (!isfinite(llp)) atomicOr(err, DERR_NONFINITE);
            if (mode == 0) {
                a.ll[i] = llp;
                if (a.lp) a.lp[i] = a.lp_p[i];
                if (a.logw) a.logw[i] = llp;
            } else {
                const double log_alpha = (llp + a.lp_p[i]) - (a.ll[i] + a.lp[i]);
                const uint4 u = philox4x32_10(make_uint4(0u, (uint32_t)i, (uint32_t)t, (TAG_ACCEPT << 16) | m),
                                              seed_key(*seedp));
                accept = log(u01_open_d(u.x)) < log_alpha;
                if (accept) {
                    a.ll[i] = llp;
                    a.lp[i] = a.lp_p[i];
                }
            }
        }
        accept = __shfl_sync(0xffffffffu, accept, 0);
        if (accept) {
            const float* src = a.beta_p + i * p;
            float* dst = a.beta + i * p;
            for (int j = lane; j < p; j += 32) dst[j] = src[j];
            if (lane == 0) atomicAdd(&block_acc, 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && block_acc && a.acc_count) atomicAdd(a.acc_count, (unsigned long long)block_acc);
}

// ------------------------------------------------------------------ reweighting
// log w_i = sum_j log p(beta_ij | c_t) - log p(beta_ij | c_{t-1}), in the form without
// cancellation: -log(c_t/c_{t-1}) - (a+1) log1p(x (c_{t-1} - c_t) / (c_t (a c_{t-1} + x))),
// x = |beta_ij| (double exponential: -log(c_t/c_{t-1}) - x (1/c_t - 1/c_{t-1})).
__global__ void __launch_bounds__(256) k_reweight(const float* __restrict__ beta, double* __restrict__ logw,
                                                  double* __restrict__ lp, int64_t N, int p, PriorArgs pr,
                                                  const double* __restrict__ sched, int t, uint32_t* __restrict__ err)
{
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const double c = sched[t], cp = sched[t - 1];
    const float k1 = (float)(cp - c), kc = (float)c, kac = (float)((double)pr.a * cp);
    const float ac = (float)((double)pr.a * c);
    double sdiff = 0.0, snew = 0.0;
    for (int j = lane; j < p; j += 32) {
        const float x = fabsf(beta[i * p + j]);
        if (pr.de) {
            sdiff += (double)x;
        } else {
            sdiff += (double)log1pf(x * k1 / (kc * (kac + x)));
        }
        snew += (double)prior_term(x, ac, pr.de);
    }
    sdiff = warp_sum(sdiff);
    snew = warp_sum(snew);
    if (lane == 0) {
        const double base = -(double)p * log(c / cp);
        const double d = pr.de ? base - sdiff * (1.0 / c - 1.0 / cp) : base - ((double)pr.a + 1.0) * sdiff;
        const double nl = logw[i] + d;
        if (!isfinite(nl)) atomicOr(err, DERR_NONFINITE);
        logw[i] = nl;
        lp[i] = prior_from_terms(snew, p, (double)pr.a, c, pr.de);
    }
}

// ---------------------------------------------------------- log-sum-exp and ESS
constexpr int LSE_THREADS = 1024;

__device__ double block_reduce_max(double v, double* sh)
{
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = LSE_THREADS / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] = fmax(sh[tid], sh[tid + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}
__device__ double block_reduce_sum(double v, double* sh)
{
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = LSE_THREADS / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] = sh[tid] + sh[tid + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(LSE_THREADS) k_lse_ess(double* __restrict__ logw, double* __restrict__ W, int64_t N,
                                                          int t, int mode, double ess_frac, double* __restrict__ ess_out,
                                                          double* __restrict__ logz_out, uint8_t* __restrict__ res_out,
                                                          int* __restrict__ flag, uint32_t* __restrict__ err)
{
    __shared__ double sh[LSE_THREADS];
    const int tid = threadIdx.x;
    double mx = -DBL_MAX;
    for (int64_t i = tid; i < N; i += LSE_THREADS) mx = fmax(mx, logw[i]);
    mx = block_reduce_max(mx, sh);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = tid; i < N; i += LSE_THREADS) {
        const double e = exp(logw[i] - mx);
        s1 += e;
        s2 += e * e;
    }
    s1 = block_reduce_sum(s1, sh);
    s2 = block_reduce_sum(s2, sh);
    const double lse = mx + log(s1);
    const double ess = (s1 * s1) / s2;
    for (int64_t i = tid; i < N; i += LSE_THREADS) {
        const double l = logw[i] - lse;
        logw[i] = l;
        W[i] = exp(l);
    }
    if (tid == 0) {
        if (!isfinite(lse) || !(ess >= 1.0 - 1e-9)) atomicOr(err, !isfinite(lse) ? DERR_NONFINITE : DERR_ESS);
        const int res = (mode == 2) ? 1 : (ess < ess_frac * (double)N);
        *flag = res;
        if (logz_out) logz_out[t] = (mode == 0) ? lse : lse - log((double)N);
        if (mode != 2) {
            if (ess_out) ess_out[t] = ess;
            if (res_out) res_out[t] = (uint8_t)res;
        }
    }
}

__global__ void k_mark_uniform(int64_t N, int t, double* ess_out, uint8_t* res_out, int* flag)
{
    if (threadIdx.x == 0) {
        *flag = 0;
        if (ess_out) ess_out[t] = (double)N;
        if (res_out) res_out[t] = 0;
    }
}

// ------------------------------------------------------------ systematic resampling
constexpr int RS_THREADS = 1024;
constexpr int RS_BLOCK = 256;  // cumulative-sum block of the specified association order

// cum must hold N + ceil(N/256) doubles: the cumulative sums, then one carry per block.
__global__ void __launch_bounds__(RS_THREADS) k_resample_index(const double* __restrict__ W, int64_t N,
                                                                double* __restrict__ cum, int32_t* __restrict__ idx,
                                                                const int* __restrict__ flag, int t,
                                                                const uint64_t* __restrict__ seedp, double u_override)
{
    if (flag && *flag == 0) return;
    __shared__ double u_sh;
    const int tid = threadIdx.x;
    const int64_t nblk = (N + RS_BLOCK - 1) / RS_BLOCK;
    double* carry = cum + N;
    // (1) running sum inside each 256-block, in index order
    for (int64_t b = tid; b < nblk; b += RS_THREADS) {
        const int64_t i0 = b * RS_BLOCK, i1 = (i0 + RS_BLOCK < N) ? i0 + RS_BLOCK : N;
        double local = 0.0;
        for (int64_t i = i0; i < i1; ++i) {
            local = __dadd_rn(local, W[i]);
            cum[i] = local;
        }
    }
    __syncthreads();
    // (2) running sum of the block totals, in block order: carry_b = sum of totals before b
    if (tid == 0) {
        double c = 0.0;
        for (int64_t b = 0; b < nblk; ++b) {
            carry[b] = c;
            const int64_t last = ((b + 1) * RS_BLOCK < N ? (b + 1) * RS_BLOCK : N) - 1;
            c = __dadd_rn(c, cum[last]);
        }
        if (seedp) {
            const uint4 u = philox4x32_10(make_uint4(0u, 0u, (uint32_t)t, TAG_RESAMPLE << 16), seed_key(*seedp));
            u_sh = u01_d(u.x);
        } else {
            u_sh = u_override;
        }
    }
    __syncthreads();
    // (3) C_i = carry_b + local_i (block 0: carry 0, exact)
    for (int64_t b = 1 + tid; b < nblk; b += RS_THREADS) {
        const int64_t i0 = b * RS_BLOCK, i1 = (i0 + RS_BLOCK < N) ? i0 + RS_BLOCK : N;
        const double cb = carry[b];
        for (int64_t i = i0; i < i1; ++i) cum[i] = __dadd_rn(cb, cum[i]);
    }
    __syncthreads();
    // (4) A_k = min{i : C_i > (k + u)/N}, clamped to N - 1 (binary search: C is non-decreasing)
    const double u = u_sh;
    for (int64_t k = tid; k < N; k += RS_THREADS) {
        const double target = __ddiv_rn(__dadd_rn((double)k, u), (double)N);
        int64_t lo = 0, hi = N;  // first index in [lo, hi) with cum > target
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cum[mid] > target)
                hi = mid;
            else
                lo = mid + 1;
        }
        idx[k] = (int32_t)(lo < N ? lo : N - 1);
    }
}

__global__ void k_gather(const int32_t* __restrict__ idx, const float* __restrict__ beta, float* __restrict__ beta_tmp,
                         const double* __restrict__ ll, const double* __restrict__ lp, double* __restrict__ ll_tmp,
                         double* __restrict__ lp_tmp, const float* __restrict__ g, float* __restrict__ g_tmp, int64_t N,
                         int p, const int* __restrict__ flag)
{
    if (*flag == 0) return;
    const int64_t total = N * (int64_t)p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / p;
        const int j = (int)(e - k * p);
        const int64_t a = idx[k];
        beta_tmp[e] = beta[a * p + j];
        if (g) g_tmp[e] = g[a * p + j];
        if (j == 0) {
            ll_tmp[k] = ll[a];
            lp_tmp[k] = lp[a];
        }
    }
}

__global__ void k_copyback(float* __restrict__ beta, const float* __restrict__ beta_tmp, double* __restrict__ ll,
                           double* __restrict__ lp, const double* __restrict__ ll_tmp, const double* __restrict__ lp_tmp,
                           float* __restrict__ g, const float* __restrict__ g_tmp, double* __restrict__ logw,
                           double* __restrict__ W, int64_t N, int p, const int* __restrict__ flag)
{
    if (*flag == 0) return;
    const int64_t total = N * (int64_t)p;
    const double lw = -log((double)N), w = 1.0 / (double)N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / p;
        const int j = (int)(e - k * p);
        beta[e] = beta_tmp[e];
        if (g) g[e] = g_tmp[e];
        if (j == 0) {
            ll[k] = ll_tmp[k];
            lp[k] = lp_tmp[k];
            logw[k] = lw;
            W[k] = w;
        }
    }
}

// -------------------------------------------------------------- column moments
constexpr int CS_ROWS = 8;

__global__ void k_colstats_partial(const float* __restrict__ beta, const double* __restrict__ W, int64_t N, int p,
                                   double* __restrict__ part)
{
    __shared__ double sh[2][CS_ROWS][32];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = blockIdx.x * 32 + tx;
    double s1 = 0.0, s2 = 0.0;
    if (j < p) {
        for (int64_t i = (int64_t)blockIdx.y * CS_ROWS + ty; i < N; i += (int64_t)CS_ROWS * gridDim.y) {
            const double w = W[i];
            const double b = (double)beta[i * p + j];
            s1 += w * b;
            s2 += w * b * b;
        }
    }
    sh[0][ty][tx] = s1;
    sh[1][ty][tx] = s2;
    __syncthreads();
    if (ty == 0 && j < p) {
        for (int r = 1; r < CS_ROWS; ++r) {
            s1 += sh[0][r][tx];
            s2 += sh[1][r][tx];
        }
        part[((int64_t)blockIdx.y * p + j) * 2 + 0] = s1;
        part[((int64_t)blockIdx.y * p + j) * 2 + 1] = s2;
    }
}

__global__ void k_colstats_finish(const double* __restrict__ part, int p, int splits, float* __restrict__ scale_out,
                                  int kind, double lam_const, const double* __restrict__ lam_dev, double sd_floor,
                                  const double* __restrict__ sched, int t)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p) return;
    double s1 = 0.0, s2 = 0.0;
    for (int s = 0; s < splits; ++s) {
        s1 += part[((int64_t)s * p + j) * 2 + 0];
        s2 += part[((int64_t)s * p + j) * 2 + 1];
    }
    const double var = fmax(s2 - s1 * s1, 0.0);
    const double fl = sd_floor * sched[t];
    const double lam = lam_dev ? *lam_dev : lam_const;
    if (kind == 0) {
        const double sd = sqrt(var);
        scale_out[j] = (float)(lam / sqrt((double)p) * fmax(sd, fl));
    } else {
        scale_out[j] = (float)fmax(var, fl * fl);
    }
}

// ------------------------------------------------------------------ summaries
// One CTA per marker j. Weighted mean and concentrations in FP64 (fixed reduction order);
// weighted quantiles Q_q = smallest value v with sum_{beta_i <= v} W_i >= q, found by
// bisection over the order-preserving 32-bit key of v, with the weights as 2^-56
// fixed-point integers so that the cumulative sums are exact and order-free.
constexpr int SUM_THREADS = 512;
constexpr int SUM_ELEMS = 32;  // particles per thread held in registers (N <= 16384)

__device__ __forceinline__ uint32_t float_key(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k)
{
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(u);
}

__device__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    for (int k = 0; k < SUM_THREADS / 32; ++k) r += sh[k];
    return r;
}

__device__ double block_sum_f64(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int k = 0; k < SUM_THREADS / 32; ++k) r += sh[k];
    return r;
}

__global__ void __launch_bounds__(SUM_THREADS, 1) k_summaries(const float* __restrict__ beta, const double* __restrict__ W,
                                                               int64_t N, int p, SummaryArgs sa, int t,
                                                               double* __restrict__ mean, double* __restrict__ quant,
                                                               double* __restrict__ conc)
{
    __shared__ unsigned long long shu[SUM_THREADS / 32];
    __shared__ double shd[SUM_THREADS / 32];
    const int j = blockIdx.x;
    const int tid = threadIdx.x;
    const double FIX = 72057594037927936.0;  // 2^56
    // mean and concentrations
    double sm = 0.0;
    double sc[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) sc[d] = 0.0;
    for (int64_t i = tid; i < N; i += SUM_THREADS) {
        const double w = W[i];
        const float b = beta[i * p + j];
        sm += w * (double)b;
#pragma unroll
        for (int d = 0; d < 8; ++d)
            if (d < sa.nd && fabs((double)b) < sa.delta[d]) sc[d] += w;
    }
    sm = block_sum_f64(sm, shd);
    if (tid == 0 && mean) mean[(int64_t)t * p + j] = sm;
    for (int d = 0; d < sa.nd; ++d) {
        const double s = block_sum_f64(sc[d], shd);
        if (tid == 0 && conc) conc[((int64_t)t * p + j) * sa.nd + d] = 1.0 - s;
    }
    if (!quant || sa.nq == 0) return;
    // quantiles
    uint32_t key[SUM_ELEMS];
    unsigned long long wf[SUM_ELEMS];
    const bool in_regs = N <= (int64_t)SUM_THREADS * SUM_ELEMS;
    uint32_t kmax = 0;
    unsigned long long tot = 0;
    if (in_regs) {
#pragma unroll
        for (int e = 0; e < SUM_ELEMS; ++e) {
            const int64_t i = tid + (int64_t)e * SUM_THREADS;
            if (i < N) {
                key[e] = float_key(beta[i * p + j]);
                wf[e] = __double2ull_rn(W[i] * FIX);
            } else {
                key[e] = 0xFFFFFFFFu;
                wf[e] = 0ull;
            }
            kmax = (wf[e] && key[e] > kmax) ? key[e] : kmax;
            tot += wf[e];
        }
    } else {
        for (int64_t i = tid; i < N; i += SUM_THREADS) {
            const uint32_t k = float_key(beta[i * p + j]);
            const unsigned long long w = __double2ull_rn(W[i] * FIX);
            kmax = (w && k > kmax) ? k : kmax;
            tot += w;
        }
    }
    tot = block_sum_u64(tot, shu);
    // block max of kmax via the u64 reduction buffer
    {
        unsigned int v = kmax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        __syncthreads();
        if ((tid & 31) == 0) shu[tid >> 5] = v;
        __syncthreads();
        unsigned int r = 0;
        for (int k = 0; k < SUM_THREADS / 32; ++k) r = max(r, (unsigned int)shu[k]);
        kmax = r;
    }
    for (int q = 0; q < sa.nq; ++q) {
        const unsigned long long target = (unsigned long long)ceil(sa.q[q] * FIX);
        uint32_t r = 0;
        if (tot < target) {
            r = kmax;  // rounding left the total below q: the largest value, as in the definition
        } else {
            for (int bit = 31; bit >= 0; --bit) {
                const uint32_t probe = r | ((1u << bit) - 1u);
                unsigned long long s = 0;
                if (in_regs) {
#pragma unroll
                    for (int e = 0; e < SUM_ELEMS; ++e) s += (key[e] <= probe) ? wf[e] : 0ull;
                } else {
                    for (int64_t i = tid; i < N; i += SUM_THREADS) {
                        const uint32_t k = float_key(beta[i * p + j]);
                        if (k <= probe) s += __double2ull_rn(W[i] * FIX);
                    }
                }
                s = block_sum_u64(s, shu);
                if (s < target) r |= (1u << bit);
            }
        }
        if (tid == 0) quant[((int64_t)t * p + j) * sa.nq + q] = (double)key_float(r);
    }
}

__global__ void k_accept_rate(const unsigned long long* acc, int T, double denom, double* rate)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) rate[t] = denom > 0.0 ? (double)acc[t] / denom : 0.0;
}

// ------------------------------------------------------------ stream-test kernels
__global__ void k_philox(const uint32_t* ctr, uint2 key, int64_t count, uint32_t* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint4 r = philox4x32_10(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]), key);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

__global__ void k_normals(uint64_t seed, uint32_t particle, uint32_t t, uint32_t m, int64_t p, float* out)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * g >= p) return;
    const float4 z = normals4(seed, (uint32_t)g, particle, t, m);
    const float zz[4] = {z.x, z.y, z.z, z.w};
    for (int k = 0; k < 4 && 4 * g + k < p; ++k) out[4 * g + k] = zz[k];
}

__global__ void k_prior_sample(uint64_t seed, PriorArgs pr, float c, int64_t N, int64_t p, float* out)
{
    const int64_t total = N * p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / p;
        out[e] = prior_draw(seed, (uint32_t)i, (uint32_t)(e - i * p), pr.a, c, pr.de != 0);
    }
}

__global__ void k_prior_logpdf(PriorArgs pr, double c, const float* beta, int64_t k, double* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    const float ac = (float)((double)pr.a * c);
    out[i] = prior_from_terms((double)prior_term(beta[i], ac, pr.de), 1, (double)pr.a, c, pr.de);
}

}  // namespace

// ======================================================================= launchers
static unsigned warps_grid(int64_t N) { return (unsigned)((N + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK); }
static unsigned elem_grid(int64_t total)
{
    int64_t b = (total + 255) / 256;
    if (b < 1) b = 1;
    return (unsigned)(b < 8192 ? b : 8192);
}

cudaError_t launch_init_prior(float* beta, int64_t N, int p, PriorArgs pr, const double* sched, int t0,
                              const uint64_t* seed, cudaStream_t st)
{
    k_init_prior<<<elem_grid(N * p), 256, 0, st>>>(beta, N, p, pr, sched, t0, seed);
    return cudaGetLastError();
}

cudaError_t launch_propose_rw(const float* beta, float* beta_p, __nv_bfloat16* A, int ldA, int Kp, double* lin_p,
                              double* lp_p, const float* sigma, const float* l2e_over_s, const float* mean_f,
                              const double* v, int64_t N, int p, PriorArgs pr, const double* sched, int t, uint32_t m,
                              const uint64_t* seed, int noise, cudaStream_t st)
{
    k_propose_rw<<<warps_grid(N), 32 * WARPS_PER_BLOCK, 0, st>>>(beta, beta_p, A, ldA, Kp, lin_p, lp_p, sigma, l2e_over_s,
                                                                  mean_f, v, N, p, pr, sched, t, m, seed, noise);
    return cudaGetLastError();
}

cudaError_t launch_propose_mala(const float* beta, const float* gl, float* beta_p, __nv_bfloat16* A, int ldA, int Kp,
                                double* lin_p, double* lp_p, double* xi2, const float* D, const double* lam,
                                const float* l2e_over_s, const float* mean_f, const double* v, int64_t N, int p,
                                PriorArgs pr, const double* sched, int t, uint32_t m, const uint64_t* seed, cudaStream_t st)
{
    k_propose_mala<<<warps_grid(N), 32 * WARPS_PER_BLOCK, 0, st>>>(beta, gl, beta_p, A, ldA, Kp, lin_p, lp_p, xi2, D, lam,
                                                                    l2e_over_s, mean_f, v, N, p, pr, sched, t, m, seed);
    return cudaGetLastError();
}

cudaError_t launch_accept_mala(const AcceptArgs& a, float* gl, const float* gl_p, const double* xi2, const float* D,
                               const double* lam, int64_t N, int p, PriorArgs pr, const double* sched, int t, uint32_t m,
                               const uint64_t* seed, uint32_t* err, cudaStream_t st)
{
    k_accept_mala<<<warps_grid(N), 32 * WARPS_PER_BLOCK, 0, st>>>(a, gl, gl_p, xi2, D, lam, N, p, pr, sched, t, m, seed,
                                                                   err);
    return cudaGetLastError();
}

cudaError_t launch_accept(const AcceptArgs& a, int64_t N, int p, int mode, int t, uint32_t m, const uint64_t* seed,
                          uint32_t* err, cudaStream_t st)
{
    k_accept<<<warps_grid(N), 32 * WARPS_PER_BLOCK, 0, st>>>(a, N, p, mode, t, m, seed, err);
    return cudaGetLastError();
}

cudaError_t launch_reweight(const float* beta, double* logw, double* lp, int64_t N, int p, PriorArgs pr,
                            const double* sched, int t, uint32_t* err, cudaStream_t st)
{
    k_reweight<<<warps_grid(N), 32 * WARPS_PER_BLOCK, 0, st>>>(beta, logw, lp, N, p, pr, sched, t, err);
    return cudaGetLastError();
}

cudaError_t launch_lse_ess(double* logw, double* W, int64_t N, int t, int mode, double ess_frac, double* ess_out,
                           double* logz_out, uint8_t* resampled_out, int* flag, uint32_t* err, cudaStream_t st)
{
    k_lse_ess<<<1, LSE_THREADS, 0, st>>>(logw, W, N, t, mode, ess_frac, ess_out, logz_out, resampled_out, flag, err);
    return cudaGetLastError();
}

cudaError_t launch_mark_uniform(int64_t N, int t, double* ess_out, uint8_t* resampled_out, int* flag, cudaStream_t st)
{
    k_mark_uniform<<<1, 32, 0, st>>>(N, t, ess_out, resampled_out, flag);
    return cudaGetLastError();
}

cudaError_t launch_resample_index(const double* W, int64_t N, double* cum, int32_t* idx, const int* flag, int t,
                                  const uint64_t* seed, double u_override, cudaStream_t st)
{
    k_resample_index<<<1, RS_THREADS, 0, st>>>(W, N, cum, idx, flag, t, seed, u_override);
    return cudaGetLastError();
}

cudaError_t launch_gather(const int32_t* idx, const float* beta, float* beta_tmp, const double* ll, const double* lp,
                          double* ll_tmp, double* lp_tmp, const float* g, float* g_tmp, int64_t N, int p,
                          const int* flag, cudaStream_t st)
{
    k_gather<<<elem_grid(N * p), 256, 0, st>>>(idx, beta, beta_tmp, ll, lp, ll_tmp, lp_tmp, g, g_tmp, N, p, flag);
    return cudaGetLastError();
}

cudaError_t launch_copyback(float* beta, const float* beta_tmp, double* ll, double* lp, const double* ll_tmp,
                            const double* lp_tmp, float* g, const float* g_tmp, double* logw, double* W, int64_t N,
                            int p, const int* flag, cudaStream_t st)
{
    k_copyback<<<elem_grid(N * p), 256, 0, st>>>(beta, beta_tmp, ll, lp, ll_tmp, lp_tmp, g, g_tmp, logw, W, N, p, flag);
    return cudaGetLastError();
}

cudaError_t launch_colstats(const float* beta, const double* W, int64_t N, int p, double* part, float* scale_out,
                            int kind, double lam_const, const double* lam_dev, double sd_floor, const double* sched,
                            int t, cudaStream_t st)
{
    dim3 block(32, CS_ROWS);
    dim3 grid((unsigned)((p + 31) / 32), COLSTAT_SPLITS);
    k_colstats_partial<<<grid, block, 0, st>>>(beta, W, N, p, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_colstats_finish<<<(unsigned)((p + 127) / 128), 128, 0, st>>>(part, p, COLSTAT_SPLITS, scale_out, kind, lam_const,
                                                                   lam_dev, sd_floor, sched, t);
    return cudaGetLastError();
}

cudaError_t launch_summaries(const float* beta, const double* W, int64_t N, int p, const SummaryArgs& s, int t,
                             double* mean, double* quant, double* conc, cudaStream_t st)
{
    k_summaries<<<(unsigned)p, SUM_THREADS, 0, st>>>(beta, W, N, p, s, t, mean, quant, conc);
    return cudaGetLastError();
}

cudaError_t launch_accept_rate(const unsigned long long* acc, int T, double denom, double* rate, cudaStream_t st)
{
    k_accept_rate<<<(T + 127) / 128, 128, 0, st>>>(acc, T, denom, rate);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint2 key, int64_t count, uint32_t* out, cudaStream_t st)
{
    k_philox<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(ctr, key, count, out);
    return cudaGetLastError();
}

cudaError_t launch_normals(uint64_t seed, uint32_t particle, uint32_t t, uint32_t m, int64_t p, float* out,
                           cudaStream_t st)
{
    const int64_t groups = (p + 3) / 4;
    k_normals<<<(unsigned)((groups + 127) / 128), 128, 0, st>>>(seed, particle, t, m, p, out);
    return cudaGetLastError();
}

cudaError_t launch_prior_sample(uint64_t seed, PriorArgs pr, double c, int64_t N, int64_t p, float* out,
                                cudaStream_t st)
{
    k_prior_sample<<<elem_grid(N * p), 256, 0, st>>>(seed, pr, (float)c, N, p, out);
    return cudaGetLastError();
}

cudaError_t launch_prior_logpdf(PriorArgs pr, double c, const float* beta, int64_t k, double* out, cudaStream_t st)
{
    k_prior_logpdf<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(pr, c, beta, k, out);
    return cudaGetLastError();
}

}  // namespace spa
