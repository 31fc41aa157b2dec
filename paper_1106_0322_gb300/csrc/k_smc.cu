// k_smc.cu -- the per-step kernels of the SMC sampler over the prior scale (Section 4).
//
// Particle state: beta [N][p] FP32 (particle-major); log-likelihood ll[N] and log prior
// lp[N] in FP64 (lp without the constant -p log(2c), which cancels in every ratio taken
// at one scale; the change of scale is handled by the incremental weight); normalised
// log-weights and weights (WeightArrays).
//
// Precision plan for GB300: the CUDA-core FP64 rate is a small fraction of FP32 and an
// FP64 warp instruction costs a full warp's issue time even with one lane active. So sums
// over markers run in FP32 with compensated (TwoSum) accumulation, and FP64 appears only
// where one thread owns one particle (weights, log-likelihoods, log-priors, MH ratios) and
// in the resampling cumulative sum, whose association order is specified.
#include <cfloat>
#include <cmath>

#include "spa_device.cuh"
#include "spa_internal.h"

namespace spa {

namespace {

constexpr int BLOCK = 256;
constexpr int WARPS = BLOCK / 32;

__device__ __forceinline__ int64_t warp_global_id()
{
    return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

// One coordinate's term of the log prior (the -log(2c) constant dropped): Gt sums
// log1p(|b|/(a c)) and multiplies by -(a+1); the double exponential sums |b| and
// multiplies by -1/c.
__device__ __forceinline__ float prior_term(float b, float ac, int de)
{
    const float x = fabsf(b);
    return de ? x : log1pf(x / ac);
}
__device__ __forceinline__ double prior_coef(PriorArgs pr, double c) { return pr.de ? -1.0 / c : -((double)pr.a + 1.0); }

__device__ __forceinline__ float dlogprior(float b, float a1, float ac, float inv_c, int de)
{
    const float sg = (b > 0.0f) ? 1.0f : ((b < 0.0f) ? -1.0f : 0.0f);
    return de ? -sg * inv_c : -a1 * sg / (ac + fabsf(b));
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

// Split-BF16 GEMM row of one coordinate: bt = b log2(e)/s_j. Returns m_j bt for the offset.
__device__ __forceinline__ float pack_coord(__nv_bfloat16* __restrict__ Arow, int Kp, int j, float b,
                                            const float* __restrict__ l2e_over_s, const float* __restrict__ mean_f)
{
    const float bt = b * l2e_over_s[j];
    __nv_bfloat16 hi, lo;
    split_bf16(bt, hi, lo);
    Arow[j] = hi;
    Arow[Kp + j] = lo;
    return mean_f[j] * bt;
}

__device__ __forceinline__ void pack_offset(__nv_bfloat16* __restrict__ Arow, int Kp, int p, float off)
{
    __nv_bfloat16 hi, lo;
    split_bf16(-off, hi, lo);
    Arow[p] = hi;
    Arow[Kp + p] = lo;
}

// ------------------------------------------------------------ RW proposal / pack
// One warp per particle; lane l handles the 4-coordinate groups g = l, l+32, ... (one
// Philox block of four normals each).
__global__ void __launch_bounds__(BLOCK) k_propose_rw(const float* __restrict__ beta, float* __restrict__ beta_p,
                                                     __nv_bfloat16* __restrict__ A, int ldA, int Kp,
                                                     float2* __restrict__ lpt_p, const float* __restrict__ sigma,
                                                     const float* __restrict__ l2e_over_s,
                                                     const float* __restrict__ mean_f, int64_t N, int p, PriorArgs pr,
                                                     const double* __restrict__ sched, int t, uint32_t m,
                                                     const uint64_t* __restrict__ seedp, int noise)
{
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const uint64_t seed = noise ? *seedp : 0ull;
    const float ac = (float)((double)pr.a * sched[t]);
    const float* row = beta + i * p;
    float* rowp = beta_p + i * p;
    __nv_bfloat16* Arow = A ? A + i * (int64_t)ldA : nullptr;
    FSum lt;
    float off = 0.0f;
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
                lt.add(prior_term(b, ac, pr.de));
                if (Arow) off += pack_coord(Arow, Kp, j, b, l2e_over_s, mean_f);
            }
        }
    }
    lt = warp_sum(lt);
    off = warp_sum(off);
    if (lane == 0) {
        lpt_p[i] = make_float2(lt.s, lt.c);
        if (Arow) pack_offset(Arow, Kp, p, off);
    }
}

// ------------------------------------------------------------ MALA proposal
// beta' = beta + (h^2/2) D grad log pi_t(beta) + h D^{1/2} xi with D = diag(D_j) and
// h = lambda p^{-1/6} (written by the column-statistics kernel); grad log pi_t = grad l
// (stored per particle) + the prior gradient -(a+1) sgn(beta)/(a c + |beta|) (double
// exponential: -sgn(beta)/c). The forward density is evaluated at the proposal as
// written (rounded to FP32): fwd = sum_j (beta'_j - beta_j - (h^2/2) D_j g_j)^2 / D_j, so
// log q(beta'|beta) = -fwd/(2h^2) + const, the same formula as the reverse term.
__global__ void __launch_bounds__(BLOCK) k_propose_mala(const float* __restrict__ beta, const float* __restrict__ gl,
                                                       float* __restrict__ beta_p, __nv_bfloat16* __restrict__ A,
                                                       int ldA, int Kp, float2* __restrict__ lpt_p,
                                                       float2* __restrict__ fwd_out, const float* __restrict__ D,
                                                       const float* __restrict__ h_dev,
                                                       const float* __restrict__ l2e_over_s,
                                                       const float* __restrict__ mean_f, int64_t N, int p, PriorArgs pr,
                                                       const double* __restrict__ sched, int t, uint32_t m,
                                                       const uint64_t* __restrict__ seedp)
{
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const uint64_t seed = *seedp;
    const double c = sched[t];
    const float ac = (float)((double)pr.a * c), a1 = pr.a + 1.0f, inv_c = (float)(1.0 / c);
    const float h = *h_dev, h2 = 0.5f * h * h;
    const float* row = beta + i * p;
    const float* grow = gl + i * p;
    float* rowp = beta_p + i * p;
    __nv_bfloat16* Arow = A ? A + i * (int64_t)ldA : nullptr;
    FSum lt, fw;
    float off = 0.0f;
    const int groups = (p + 3) >> 2;
    for (int g = lane; g < groups; g += 32) {
        const float4 z4 = normals4(seed, (uint32_t)g, (uint32_t)i, (uint32_t)t, m);
        const float z[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = 4 * g + k;
            if (j < p) {
                const float b0 = row[j];
                const float Dj = D[j];
                const float drift = h2 * Dj * (grow[j] + dlogprior(b0, a1, ac, inv_c, pr.de));
                const float b = (b0 + drift) + h * sqrtf(Dj) * z[k];
                rowp[j] = b;
                const float d = (b - b0) - drift;
                fw.add(d * d / Dj);
                lt.add(prior_term(b, ac, pr.de));
                if (Arow) off += pack_coord(Arow, Kp, j, b, l2e_over_s, mean_f);
            }
        }
    }
    lt = warp_sum(lt);
    fw = warp_sum(fw);
    off = warp_sum(off);
    if (lane == 0) {
        lpt_p[i] = make_float2(lt.s, lt.c);
        fwd_out[i] = make_float2(fw.s, fw.c);
        if (Arow) pack_offset(Arow, Kp, p, off);
    }
}

// --------------------------------------------------------------- finish / MH test
// One thread per particle for the FP64 scalars (32 particles per warp instruction), then
// the block's warps copy the accepted rows.
__device__ __forceinline__ double finish_loglik(const AcceptArgs& a, int64_t i)
{
    FSum sp;
    for (int s = 0; s < a.n_parts; ++s) sp.add(a.partial[(int64_t)s * a.ld_part + i]);
    return a.sp_scale * sp.value();
}

constexpr int ACC_PER_BLOCK = 32;

// Copy the accepted rows of the block's 32 particles: every thread moves 4-element chunks
// of all rows at once, so the loads are in flight together.
__device__ __forceinline__ void copy_accepted_rows(const unsigned char* flag, int64_t i0, int64_t N, int p,
                                                   const float* __restrict__ src, float* __restrict__ dst,
                                                   const float* __restrict__ src2, float* __restrict__ dst2)
{
    const int64_t total = (int64_t)ACC_PER_BLOCK * p;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int q = (int)(e / p);
        if (!flag[q] || i0 + q >= N) continue;
        const int64_t off = i0 * p + e;
        dst[off] = src[off];
        if (src2) dst2[off] = src2[off];
    }
}

__global__ void __launch_bounds__(BLOCK) k_accept(AcceptArgs a, int64_t N, int p, PriorArgs pr,
                                                 const double* __restrict__ sched, int mode, int t, uint32_t m,
                                                 const uint64_t* __restrict__ seedp, uint32_t* __restrict__ err)
{
    __shared__ unsigned char flag[ACC_PER_BLOCK];
    __shared__ int nacc;
    const int64_t i0 = (int64_t)blockIdx.x * ACC_PER_BLOCK;
    if (threadIdx.x < 32) {
        const int64_t i = i0 + threadIdx.x;
        int accept = 0;
        if (i < N) {
            const double llp = finish_loglik(a, i);
            const float2 q = a.lpt_p[i];
            const double lpp = prior_coef(pr, sched[t]) * ((double)q.x + (double)q.y);
            if (!isfinite(llp)) atomicOr(err, DERR_NONFINITE);
            if (mode == 0) {
                a.ll[i] = llp;
                if (a.lp) a.lp[i] = lpp;
                if (a.logw) a.logw[i] = llp;
            } else {
                const double log_alpha = (llp - a.ll[i]) + (lpp - a.lp[i]);
                const uint4 u = philox4x32_10(make_uint4(0u, (uint32_t)i, (uint32_t)t, (TAG_ACCEPT << 16) | m),
                                              seed_key(*seedp));
                accept = (double)logf(u01_open_f(u.x)) < log_alpha;
                if (accept) {
                    a.ll[i] = llp;
                    a.lp[i] = lpp;
                }
            }
        }
        flag[threadIdx.x] = (unsigned char)accept;
        const int cnt = __popc(__ballot_sync(0xffffffffu, accept));
        if (threadIdx.x == 0) {
            nacc = cnt;
            if (cnt && a.acc_count) atomicAdd(a.acc_count, (unsigned long long)cnt);
        }
    }
    __syncthreads();
    if (nacc == 0) return;
    copy_accepted_rows(flag, i0, N, p, a.beta_p, a.beta, nullptr, nullptr);
}

// MH test of a MALA proposal: log alpha = l' + lp' - l - lp + log q(beta|beta') - log q(beta'|beta),
// log q(x|z) = -sum_j (x_j - z_j - (h^2/2) D_j g_j(z))^2 / (2 h^2 D_j) + const. Accepted rows
// move beta and its gradient.
__global__ void __launch_bounds__(BLOCK) k_accept_mala(AcceptArgs a, float* __restrict__ gl,
                                                      const float* __restrict__ gl_p, const float2* __restrict__ fwd,
                                                      const float* __restrict__ D, const float* __restrict__ h_dev,
                                                      int64_t N, int p, PriorArgs pr, const double* __restrict__ sched,
                                                      int t, uint32_t m, const uint64_t* __restrict__ seedp,
                                                      uint32_t* __restrict__ err)
{
    __shared__ unsigned char flag[ACC_PER_BLOCK];
    __shared__ float2 bwd_sh[ACC_PER_BLOCK];
    __shared__ int nacc;
    const int64_t i0 = (int64_t)blockIdx.x * ACC_PER_BLOCK;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double c = sched[t];
    const float ac = (float)((double)pr.a * c), a1 = pr.a + 1.0f, inv_c = (float)(1.0 / c);
    const float h = *h_dev, h2 = 0.5f * h * h;
    // reverse-move residuals, one warp per particle
    for (int q = w; q < ACC_PER_BLOCK; q += WARPS) {
        const int64_t k = i0 + q;
        FSum bwd;
        if (k < N) {
            const float* b0 = a.beta + k * p;
            const float* b1 = a.beta_p + k * p;
            const float* g1 = gl_p + k * p;
            for (int j = lane; j < p; j += 32) {
                const float Dj = D[j];
                const float drift = h2 * Dj * (g1[j] + dlogprior(b1[j], a1, ac, inv_c, pr.de));
                const float d = (b0[j] - b1[j]) - drift;
                bwd.add(d * d / Dj);
            }
        }
        bwd = warp_sum(bwd);
        if (lane == 0) bwd_sh[q] = make_float2(bwd.s, bwd.c);
    }
    __syncthreads();
    if (w == 0) {
        const int64_t i = i0 + lane;
        int accept = 0;
        if (i < N) {
            const double llp = finish_loglik(a, i);
            const float2 q = a.lpt_p[i];
            const double lpp = prior_coef(pr, c) * ((double)q.x + (double)q.y);
            if (!isfinite(llp)) atomicOr(err, DERR_NONFINITE);
            const float2 bw = bwd_sh[lane];
            const float2 fw = fwd[i];
            const double hh2 = 2.0 * (double)h * (double)h;
            const double log_alpha = (llp - a.ll[i]) + (lpp - a.lp[i]) -
                                     (((double)bw.x + (double)bw.y) - ((double)fw.x + (double)fw.y)) / hh2;
            const uint4 u = philox4x32_10(make_uint4(0u, (uint32_t)i, (uint32_t)t, (TAG_ACCEPT << 16) | m),
                                          seed_key(*seedp));
            accept = (double)logf(u01_open_f(u.x)) < log_alpha;
            if (accept) {
                a.ll[i] = llp;
                a.lp[i] = lpp;
            }
        }
        flag[lane] = (unsigned char)accept;
        const int cnt = __popc(__ballot_sync(0xffffffffu, accept));
        if (lane == 0) {
            nacc = cnt;
            if (cnt && a.acc_count) atomicAdd(a.acc_count, (unsigned long long)cnt);
        }
    }
    __syncthreads();
    if (nacc == 0) return;
    copy_accepted_rows(flag, i0, N, p, a.beta_p, a.beta, gl_p, gl);
}

// ------------------------------------------------------------------ reweighting
// log w_i = sum_j log p(beta_ij | c_t) - log p(beta_ij | c_{t-1}) in the form without
// cancellation: -log(c_t/c_{t-1}) - (a+1) log1p(x (c_{t-1} - c_t) / (c_t (a c_{t-1} + x))),
// x = |beta_ij| (double exponential: -log(c_t/c_{t-1}) - x (1/c_t - 1/c_{t-1})).
// A block handles 32 particles: its warps form the FP32 row sums, then warp 0 finishes one
// particle per lane in FP64.
constexpr int RW_PER_BLOCK = 32;
constexpr int RW_THREADS = 32 * RW_PER_BLOCK;

__global__ void __launch_bounds__(RW_THREADS) k_reweight(const float* __restrict__ beta, double* __restrict__ logw,
                                                   double* __restrict__ lp, int64_t N, int p, PriorArgs pr,
                                                   const double* __restrict__ sched, int t, uint32_t* __restrict__ err)
{
    __shared__ float4 sums[RW_PER_BLOCK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * RW_PER_BLOCK;
    const double c = sched[t], cp = sched[t - 1];
    const float k1 = (float)(cp - c), kc = (float)c, kac = (float)((double)pr.a * cp);
    const float ac = (float)((double)pr.a * c);
    {
        const int q = w;
        const int64_t i = base + q;
        FSum sdiff, snew;
        if (i < N) {
            for (int j = lane; j < p; j += 32) {
                const float x = fabsf(beta[i * p + j]);
                sdiff.add(pr.de ? x : log1pf(x * k1 / (kc * (kac + x))));
                snew.add(prior_term(x, ac, pr.de));
            }
        }
        sdiff = warp_sum(sdiff);
        snew = warp_sum(snew);
        if (lane == 0) sums[q] = make_float4(sdiff.s, sdiff.c, snew.s, snew.c);
    }
    __syncthreads();
    if (w == 0) {
        const int64_t i = base + lane;
        if (i < N) {
            const float4 s = sums[lane];
            const double sd = (double)s.x + (double)s.y, sn = (double)s.z + (double)s.w;
            const double lbase = -(double)p * log(c / cp);
            const double d = pr.de ? lbase - sd * (1.0 / c - 1.0 / cp) : lbase - ((double)pr.a + 1.0) * sd;
            const double nl = logw[i] + d;
            if (!isfinite(nl)) atomicOr(err, DERR_NONFINITE);
            logw[i] = nl;
            lp[i] = prior_coef(pr, c) * sn;
        }
    }
}

// ---------------------------------------------------------- log-sum-exp and ESS
__device__ double block_max_f64(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = sh[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, sh[k]);
    return r;
}
__device__ double block_sum_f64(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = sh[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    return r;
}

// Each block: (m_b, sum e^{x - m_b}, sum e^{2(x - m_b)}) over its elements. The last block
// to finish combines the blocks in block order and publishes LSE, ESS, log Z and the flag.
__global__ void __launch_bounds__(BLOCK) k_lse_partial(const double* __restrict__ logw, int64_t N,
                                                      double* __restrict__ scratch, unsigned int* __restrict__ counter,
                                                      int t, int mode, double ess_frac, double* __restrict__ ess_out,
                                                      double* __restrict__ logz_out, uint8_t* __restrict__ res_out,
                                                      int* __restrict__ flag, uint32_t* __restrict__ err)
{
    __shared__ double sh[BLOCK / 32];
    __shared__ bool last;
    const int64_t stride = (int64_t)gridDim.x * BLOCK;
    double mx = -DBL_MAX;
    for (int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x; i < N; i += stride) mx = fmax(mx, logw[i]);
    const double mb = block_max_f64(mx, sh);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x; i < N; i += stride) {
        const double e = exp(logw[i] - mb);
        s1 += e;
        s2 += e * e;
    }
    s1 = block_sum_f64(s1, sh);
    s2 = block_sum_f64(s2, sh);
    const int B = gridDim.x;
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = mb;
        scratch[B + blockIdx.x] = s1;
        scratch[2 * B + blockIdx.x] = s2;
        __threadfence();
        last = (atomicAdd(counter, 1u) == (unsigned)(B - 1));
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    // combine the block partials: lane l takes blocks l, l+32, ... (fixed order), then a
    // fixed-order warp tree
    const int lane = threadIdx.x;
    double m = -DBL_MAX;
    for (int b = lane; b < B; b += 32) m = fmax(m, scratch[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    double S1 = 0.0, S2 = 0.0;
    for (int b = lane; b < B; b += 32) {
        const double f = (scratch[B + b] > 0.0) ? exp(scratch[b] - m) : 0.0;
        S1 += scratch[B + b] * f;
        S2 += scratch[2 * B + b] * f * f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        S1 += __shfl_xor_sync(0xffffffffu, S1, o);
        S2 += __shfl_xor_sync(0xffffffffu, S2, o);
    }
    if (lane != 0) return;
    const double lse = m + log(S1);
    const double ess = (S1 * S1) / S2;
    scratch[3 * B] = lse;
    *counter = 0u;
    if (!isfinite(lse) || !(ess >= 1.0 - 1e-9)) atomicOr(err, !isfinite(lse) ? DERR_NONFINITE : DERR_ESS);
    const int res = (mode == 2) ? 1 : (ess < ess_frac * (double)N);
    *flag = res;
    if (logz_out) logz_out[t] = (mode == 0) ? lse : lse - log((double)N);
    if (mode != 2) {
        if (ess_out) ess_out[t] = ess;
        if (res_out) res_out[t] = (uint8_t)res;
    }
}

__device__ __forceinline__ uint32_t weight_fix(double W) { return (uint32_t)__double2ull_rn(W * 2147483648.0); }

__global__ void k_normalise(WeightArrays w, int64_t N, const double* __restrict__ lse_ptr)
{
    const double lse = *lse_ptr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double l = w.logw[i] - lse;
        const double W = exp(l);
        w.logw[i] = l;
        w.W[i] = W;
        w.Wf[i] = (float)W;
        w.wfix[i] = weight_fix(W);
    }
}

__global__ void k_weight_forms(const double* __restrict__ W, int64_t N, float* __restrict__ Wf,
                               uint32_t* __restrict__ wfix)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        Wf[i] = (float)W[i];
        wfix[i] = weight_fix(W[i]);
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

// The cumulative sum C of W in the specified order: a running sum inside each 256-block
// in index order, a running sum of the block totals, C_i = carry(block) + local_i.
// cum holds N + ceil(N/256) + 1 doubles: C, then one carry per block, then u.
__global__ void __launch_bounds__(RS_THREADS) k_resample_scan(const double* __restrict__ W, int64_t N,
                                                               double* __restrict__ cum, const int* __restrict__ flag,
                                                               int t, const uint64_t* __restrict__ seedp,
                                                               double u_override)
{
    if (flag && *flag == 0) return;
    const int tid = threadIdx.x;
    const int64_t nblk = (N + RS_BLOCK - 1) / RS_BLOCK;
    double* carry = cum + N;
    for (int64_t b = tid; b < nblk; b += RS_THREADS) {
        const int64_t i0 = b * RS_BLOCK, i1 = (i0 + RS_BLOCK < N) ? i0 + RS_BLOCK : N;
        double local = 0.0;
        for (int64_t i = i0; i < i1; ++i) {
            local = __dadd_rn(local, W[i]);
            cum[i] = local;
        }
    }
    __syncthreads();
    if (tid == 0) {
        double c = 0.0;
        for (int64_t b = 0; b < nblk; ++b) {
            carry[b] = c;
            const int64_t last = ((b + 1) * RS_BLOCK < N ? (b + 1) * RS_BLOCK : N) - 1;
            c = __dadd_rn(c, cum[last]);
        }
        if (seedp) {
            const uint4 u = philox4x32_10(make_uint4(0u, 0u, (uint32_t)t, TAG_RESAMPLE << 16), seed_key(*seedp));
            carry[nblk] = u01_d(u.x);
        } else {
            carry[nblk] = u_override;
        }
    }
    __syncthreads();
    for (int64_t b = 1 + tid; b < nblk; b += RS_THREADS) {
        const int64_t i0 = b * RS_BLOCK, i1 = (i0 + RS_BLOCK < N) ? i0 + RS_BLOCK : N;
        const double cb = carry[b];
        for (int64_t i = i0; i < i1; ++i) cum[i] = __dadd_rn(cb, cum[i]);
    }
}

// A_k = min{i : C_i > (k + u)/N}, clamped to N - 1. C is non-negative and non-decreasing,
// and for non-negative doubles the order of the bit patterns as signed integers is the
// numeric order, so the search compares integers.
__global__ void k_resample_search(const double* __restrict__ cum, int64_t N, int32_t* __restrict__ idx,
                                  const int* __restrict__ flag)
{
    if (flag && *flag == 0) return;
    const int64_t nblk = (N + RS_BLOCK - 1) / RS_BLOCK;
    const double u = cum[N + nblk];
    const long long* ci = reinterpret_cast<const long long*>(cum);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const long long target = __double_as_longlong(__ddiv_rn(__dadd_rn((double)k, u), (double)N));
        int64_t lo = 0, hi = N;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (ci[mid] > target)
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
                           float* __restrict__ g, const float* __restrict__ g_tmp, WeightArrays w, int64_t N, int p,
                           const int* __restrict__ flag, double lw, double wi, uint32_t wf)
{
    if (*flag == 0) return;
    const int64_t total = N * (int64_t)p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / p;
        const int j = (int)(e - k * p);
        beta[e] = beta_tmp[e];
        if (g) g[e] = g_tmp[e];
        if (j == 0) {
            ll[k] = ll_tmp[k];
            lp[k] = lp_tmp[k];
            w.logw[k] = lw;
            w.W[k] = wi;
            w.Wf[k] = (float)wi;
            w.wfix[k] = wf;
        }
    }
}

// -------------------------------------------------------------- column moments
constexpr int CS_ROWS = 8;

__global__ void k_colstats_partial(const float* __restrict__ beta, const float* __restrict__ Wf, int64_t N, int p,
                                   float4* __restrict__ part)
{
    __shared__ float4 sh[CS_ROWS][32];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = blockIdx.x * 32 + tx;
    FSum s1, s2;
    if (j < p) {
        const int64_t step = (int64_t)CS_ROWS * gridDim.y;
        int64_t i = (int64_t)blockIdx.y * CS_ROWS + ty;
        for (; i + 3 * step < N; i += 4 * step) {  // four rows in flight
            float b[4], wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                b[u] = beta[(i + u * step) * p + j];
                wv[u] = Wf[i + u * step];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float wb = wv[u] * b[u];
                s1.add(wb);
                s2.add(wb * b[u]);
            }
        }
        for (; i < N; i += step) {
            const float b = beta[i * p + j];
            const float wb = Wf[i] * b;
            s1.add(wb);
            s2.add(wb * b);
        }
    }
    sh[ty][tx] = make_float4(s1.s, s1.c, s2.s, s2.c);
    __syncthreads();
    if (ty == 0 && j < p) {
        for (int r = 1; r < CS_ROWS; ++r) {
            const float4 o = sh[r][tx];
            s1.add(o.x);
            s1.c += o.y;
            s2.add(o.z);
            s2.c += o.w;
        }
        part[(int64_t)blockIdx.y * p + j] = make_float4(s1.s, s1.c, s2.s, s2.c);
    }
}

// One warp per coordinate: lane s takes split s (fixed order), then a warp tree.
__global__ void k_colstats_finish(const float4* __restrict__ part, int p, int splits, float* __restrict__ scale_out,
                                  int kind, double lam_const, const double* __restrict__ lam_dev, double sd_floor,
                                  const double* __restrict__ sched, int t, float* __restrict__ h_out, double p_pow)
{
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= p) return;
    double s1 = 0.0, s2 = 0.0;
    for (int s = lane; s < splits; s += 32) {
        const float4 q = part[(int64_t)s * p + j];
        s1 += (double)q.x + (double)q.y;
        s2 += (double)q.z + (double)q.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane != 0) return;
    const double lam = lam_dev ? *lam_dev : lam_const;
    if (j == 0 && h_out) *h_out = (float)(lam * p_pow);
    const double var = fmax(s2 - s1 * s1, 0.0);
    const double fl = sd_floor * sched[t];
    if (kind == 0) {
        scale_out[j] = (float)(lam / sqrt((double)p) * fmax(sqrt(var), fl));
    } else {
        scale_out[j] = (float)fmax(var, fl * fl);
    }
}

// ------------------------------------------------------------------ summaries
// One CTA per marker j. Weighted mean (FP32 weights, compensated sum) and concentrations
// 1 - sum_{|beta| < Delta} W (Delta passed as the smallest float >= Delta, which makes the
// float comparison equal to the exact one). Weighted quantiles Q_q = the smallest value v
// with sum_{beta_i <= v} W_i >= q, by a three-pass radix select (11, 11, 10 bits) over the
// order-preserving 32-bit key of v. Weights enter the histograms as the integers
// round(W 2^31), so every cumulative sum is exact and independent of the order of the
// atomic additions.
constexpr int SUM_THREADS = 512;
constexpr size_t SUM_STAGED_MAX = 200 * 1024;  // dynamic shared memory of the staged variant

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

// First bin of hist[0..nbins) (weights) at which *below + the cumulative weight reaches
// target; one warp. Adds the weight of the bins before it to *below. Returns -1 if no bin
// reaches the target.
__device__ int warp_find_bin(const uint32_t* hist, int nbins, unsigned long long target, unsigned long long* below)
{
    const int lane = threadIdx.x & 31;
    const int per = nbins / 32;
    unsigned long long mine = 0;
    for (int k = 0; k < per; ++k) mine += hist[lane * per + k];
    unsigned long long incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned long long base = *below;
    const unsigned int hit = __ballot_sync(0xffffffffu, base + incl >= target);
    if (hit == 0u) return -1;
    const int L = __ffs(hit) - 1;
    int bin = -1;
    unsigned long long add = 0;
    if (lane == L) {
        unsigned long long cum = base + incl - mine;
        for (int k = 0; k < per; ++k) {
            const unsigned long long h = hist[L * per + k];
            if (cum + h >= target) {
                bin = L * per + k;
                break;
            }
            cum += h;
        }
        add = cum - base;
    }
    bin = __shfl_sync(0xffffffffu, bin, L);
    add = __shfl_sync(0xffffffffu, add, L);
    if (bin >= 0) *below = base + add;
    return bin;
}

__device__ void block_fsum_store(FSum v, float* shs, float* shc, double* out)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) {
        shs[w] = v.s;
        shc[w] = v.c;
    }
    __syncthreads();
    if (threadIdx.x == 0 && out) {
        FSum r;
        for (int k = 0; k < SUM_THREADS / 32; ++k) {
            r.add(shs[k]);
            r.c += shc[k];
        }
        *out = r.value();
    }
}

__global__ void __launch_bounds__(SUM_THREADS, 1) k_summaries(const float* __restrict__ beta, const float* __restrict__ Wf,
                                                               const uint32_t* __restrict__ wfix, int64_t N, int p,
                                                               SummaryArgs sa, int t, double* __restrict__ mean,
                                                               double* __restrict__ quant, double* __restrict__ conc,
                                                               int staged)
{
    extern __shared__ uint32_t sm[];
    __shared__ float shs[SUM_THREADS / 32], shc[SUM_THREADS / 32];
    __shared__ unsigned long long shu[SUM_THREADS / 32];
    __shared__ uint32_t shk[SUM_THREADS / 32];
    __shared__ int bins[8][3];
    __shared__ unsigned long long below[8];
    __shared__ double conc_sh[8];
    const int j = blockIdx.x;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int nq = sa.nq, nd = sa.nd;
    uint32_t* keys = sm;
    uint32_t* wts = sm + (staged ? N : 0);
    uint32_t* hist = sm + (staged ? 2 * N : 0);  // (nq or 1) * 2048 words
    float dthr[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        float f = (float)sa.delta[d];
        if ((double)f < sa.delta[d]) f = nextafterf(f, INFINITY);
        dthr[d] = f;
    }
    // ---- pass 0: stage keys and weights; mean, concentrations, maximum key, total weight
    FSum msum;
    FSum cs[8];
    uint32_t kmax = 0;
    unsigned long long tot = 0;
    for (int64_t i = tid; i < N; i += SUM_THREADS) {
        const float b = beta[i * p + j];
        const uint32_t k = float_key(b);
        const uint32_t wv = wfix[i];
        const float wf = Wf[i];
        if (staged) {
            keys[i] = k;
            wts[i] = wv;
        }
        msum.add(wf * b);
#pragma unroll
        for (int d = 0; d < 8; ++d)
            if (d < nd && fabsf(b) < dthr[d]) cs[d].add(wf);
        kmax = k > kmax ? k : kmax;
        tot += wv;
    }
    double mval = 0.0;
    block_fsum_store(msum, shs, shc, &mval);
    if (tid == 0 && mean) mean[(int64_t)t * p + j] = mval;
    for (int d = 0; d < nd; ++d) {
        block_fsum_store(cs[d], shs, shc, &conc_sh[d]);
        if (tid == 0 && conc) conc[((int64_t)t * p + j) * nd + d] = 1.0 - conc_sh[d];
    }
    if (!quant || nq == 0) return;
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        uint32_t v = kmax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        __syncthreads();
        if (lane == 0) {
            shu[w] = tot;
            shk[w] = v;
        }
        __syncthreads();
        tot = 0;
        uint32_t r = 0;
        for (int k = 0; k < SUM_THREADS / 32; ++k) {
            tot += shu[k];
            r = max(r, shk[k]);
        }
        kmax = r;
    }
    if (tid < 8) below[tid] = 0ull;
    // ---- radix passes: (shift, bits) = (21, 11), (10, 11), (0, 10)
    for (int pass = 0; pass < 3; ++pass) {
        const int bits = (pass == 2) ? 10 : 11;
        const int shift = (pass == 0) ? 21 : ((pass == 1) ? 10 : 0);
        const int nb = 1 << bits;
        const int nh = (pass == 0) ? 1 : nq;  // the first histogram is shared by every level
        for (int e = tid; e < nh * nb; e += SUM_THREADS) hist[e] = 0u;
        __syncthreads();
        for (int64_t i = tid; i < N; i += SUM_THREADS) {
            const uint32_t k = staged ? keys[i] : float_key(beta[i * p + j]);
            const uint32_t wv = staged ? wts[i] : wfix[i];
            if (wv == 0u) continue;
            const uint32_t dig = (k >> shift) & (uint32_t)(nb - 1);
            if (pass == 0) {
                atomicAdd(&hist[dig], wv);
            } else {
                const uint32_t pre = k >> (shift + bits);
                for (int q = 0; q < nq; ++q) {
                    if (bins[q][0] < 0) continue;
                    const uint32_t want =
                        (pass == 1) ? (uint32_t)bins[q][0] : (((uint32_t)bins[q][0] << 11) | (uint32_t)bins[q][1]);
                    if (pre == want) atomicAdd(&hist[q * nb + dig], wv);
                }
            }
        }
        __syncthreads();
        if (w < nq) {
            const int q = w;
            const unsigned long long target = (unsigned long long)ceil(sa.q[q] * 2147483648.0);
            int b = -1;
            if (tot >= target && (pass == 0 || bins[q][0] >= 0)) {
                unsigned long long bl = below[q];
                b = warp_find_bin(hist + (pass == 0 ? 0 : q * nb), nb, target, &bl);
                if (lane == 0) below[q] = bl;
            }
            if (lane == 0) {
                if (pass == 0)
                    bins[q][0] = b;
                else if (bins[q][0] >= 0)
                    bins[q][pass] = b;
            }
        }
        __syncthreads();
    }
    if (tid < nq) {
        const int q = tid;
        uint32_t key;
        if (bins[q][0] < 0 || bins[q][1] < 0 || bins[q][2] < 0)
            key = kmax;  // rounding left the total below q: the largest value, as in the definition
        else
            key = ((uint32_t)bins[q][0] << 21) | ((uint32_t)bins[q][1] << 10) | (uint32_t)bins[q][2];
        quant[((int64_t)t * p + j) * nq + q] = (double)key_float(key);
    }
}

__global__ void k_accept_rate(const unsigned long long* acc, int T, double denom, double* rate)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) rate[t] = denom > 0.0 ? (double)acc[t] / denom : 0.0;
}

__global__ void k_adapt_lambda(double* lam, const unsigned long long* acc, double denom)
{
    if (threadIdx.x == 0 && denom > 0.0) *lam *= exp((double)*acc / denom - 0.574);
}

__global__ void k_set_f64(double* ptr, double v)
{
    if (threadIdx.x == 0) *ptr = v;
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

// The full log density, -log(2c) included.
__global__ void k_prior_logpdf(PriorArgs pr, double c, const float* beta, int64_t k, double* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    const float ac = (float)((double)pr.a * c);
    out[i] = -log(2.0 * c) + prior_coef(pr, c) * (double)prior_term(beta[i], ac, pr.de);
}

}  // namespace

// ======================================================================= launchers
static unsigned warps_grid(int64_t N) { return (unsigned)((N + WARPS - 1) / WARPS); }
static unsigned elem_grid(int64_t total)
{
    int64_t b = (total + 255) / 256;
    if (b < 1) b = 1;
    return (unsigned)(b < 8192 ? b : 8192);
}

cudaError_t smc_init_attributes()
{
    return cudaFuncSetAttribute(k_summaries, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SUM_STAGED_MAX);
}

cudaError_t launch_init_prior(float* beta, int64_t N, int p, PriorArgs pr, const double* sched, int t0,
                              const uint64_t* seed, cudaStream_t st)
{
    k_init_prior<<<elem_grid(N * p), 256, 0, st>>>(beta, N, p, pr, sched, t0, seed);
    return cudaGetLastError();
}

cudaError_t launch_propose_rw(const float* beta, float* beta_p, __nv_bfloat16* A, int ldA, int Kp, float2* lpt_p,
                              const float* sigma, const float* l2e_over_s, const float* mean_f, int64_t N, int p,
                              PriorArgs pr, const double* sched, int t, uint32_t m, const uint64_t* seed, int noise,
                              cudaStream_t st)
{
    k_propose_rw<<<warps_grid(N), BLOCK, 0, st>>>(beta, beta_p, A, ldA, Kp, lpt_p, sigma, l2e_over_s, mean_f, N, p, pr,
                                                  sched, t, m, seed, noise);
    return cudaGetLastError();
}

cudaError_t launch_propose_mala(const float* beta, const float* gl, float* beta_p, __nv_bfloat16* A, int ldA, int Kp,
                                float2* lpt_p, float2* fwd, const float* D, const float* h, const float* l2e_over_s,
                                const float* mean_f, int64_t N, int p, PriorArgs pr, const double* sched, int t,
                                uint32_t m, const uint64_t* seed, cudaStream_t st)
{
    k_propose_mala<<<warps_grid(N), BLOCK, 0, st>>>(beta, gl, beta_p, A, ldA, Kp, lpt_p, fwd, D, h, l2e_over_s, mean_f,
                                                    N, p, pr, sched, t, m, seed);
    return cudaGetLastError();
}

cudaError_t launch_accept(const AcceptArgs& a, int64_t N, int p, PriorArgs pr, const double* sched, int mode, int t,
                          uint32_t m, const uint64_t* seed, uint32_t* err, cudaStream_t st)
{
    k_accept<<<(unsigned)((N + ACC_PER_BLOCK - 1) / ACC_PER_BLOCK), BLOCK, 0, st>>>(a, N, p, pr, sched, mode, t, m, seed,
                                                                                     err);
    return cudaGetLastError();
}

cudaError_t launch_accept_mala(const AcceptArgs& a, float* gl, const float* gl_p, const float2* fwd, const float* D,
                               const float* h, int64_t N, int p, PriorArgs pr, const double* sched, int t, uint32_t m,
                               const uint64_t* seed, uint32_t* err, cudaStream_t st)
{
    k_accept_mala<<<(unsigned)((N + ACC_PER_BLOCK - 1) / ACC_PER_BLOCK), BLOCK, 0, st>>>(a, gl, gl_p, fwd, D, h, N, p, pr,
                                                                                          sched, t, m, seed, err);
    return cudaGetLastError();
}

cudaError_t launch_reweight(const float* beta, double* logw, double* lp, int64_t N, int p, PriorArgs pr,
                            const double* sched, int t, uint32_t* err, cudaStream_t st)
{
    k_reweight<<<(unsigned)((N + RW_PER_BLOCK - 1) / RW_PER_BLOCK), RW_THREADS, 0, st>>>(beta, logw, lp, N, p, pr, sched,
                                                                                         t, err);
    return cudaGetLastError();
}

cudaError_t launch_lse_ess(const WeightArrays& w, int64_t N, double* scratch, unsigned int* counter, int t, int mode,
                           double ess_frac, double* ess_out, double* logz_out, uint8_t* resampled_out, int* flag,
                           uint32_t* err, cudaStream_t st)
{
    int64_t blocks = (N + BLOCK - 1) / BLOCK;
    if (blocks > LSE_BLOCKS) blocks = LSE_BLOCKS;
    k_lse_partial<<<(unsigned)blocks, BLOCK, 0, st>>>(w.logw, N, scratch, counter, t, mode, ess_frac, ess_out, logz_out,
                                                      resampled_out, flag, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_normalise<<<elem_grid(N), 256, 0, st>>>(w, N, scratch + 3 * blocks);
    return cudaGetLastError();
}

cudaError_t launch_weight_forms(const double* W, int64_t N, float* Wf, uint32_t* wfix, cudaStream_t st)
{
    k_weight_forms<<<elem_grid(N), 256, 0, st>>>(W, N, Wf, wfix);
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
    k_resample_scan<<<1, RS_THREADS, 0, st>>>(W, N, cum, flag, t, seed, u_override);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_resample_search<<<elem_grid(N), 256, 0, st>>>(cum, N, idx, flag);
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
                            const double* lp_tmp, float* g, const float* g_tmp, const WeightArrays& w, int64_t N,
                            int p, const int* flag, cudaStream_t st)
{
    // uniform weights after resampling: log(1/N), 1/N and round(2^31 / N), formed on the host
    const double wi = 1.0 / (double)N;
    const uint32_t wf = (uint32_t)std::llrint(wi * 2147483648.0);
    k_copyback<<<elem_grid(N * p), 256, 0, st>>>(beta, beta_tmp, ll, lp, ll_tmp, lp_tmp, g, g_tmp, w, N, p, flag,
                                                 -std::log((double)N), wi, wf);
    return cudaGetLastError();
}

cudaError_t launch_colstats(const float* beta, const float* Wf, int64_t N, int p, float4* part, float* scale_out,
                            int kind, double lam_const, const double* lam_dev, double sd_floor, const double* sched,
                            int t, float* h_out, cudaStream_t st)
{
    dim3 block(32, CS_ROWS);
    dim3 grid((unsigned)((p + 31) / 32), COLSTAT_SPLITS);
    k_colstats_partial<<<grid, block, 0, st>>>(beta, Wf, N, p, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_colstats_finish<<<(unsigned)((p + 7) / 8), 256, 0, st>>>(part, p, COLSTAT_SPLITS, scale_out, kind, lam_const,
                                                               lam_dev, sd_floor, sched, t, h_out,
                                                               std::pow((double)p, -1.0 / 6.0));
    return cudaGetLastError();
}

cudaError_t launch_summaries(const float* beta, const float* Wf, const uint32_t* wfix, int64_t N, int p,
                             const SummaryArgs& s, int t, double* mean, double* quant, double* conc, cudaStream_t st)
{
    const int nh = s.nq > 1 ? s.nq : 1;
    const size_t hist_bytes = (size_t)nh * 2048 * sizeof(uint32_t);
    const size_t staged_bytes = (size_t)N * 2 * sizeof(uint32_t) + hist_bytes;
    const int staged = staged_bytes <= SUM_STAGED_MAX ? 1 : 0;
    const size_t bytes = staged ? staged_bytes : hist_bytes;
    k_summaries<<<(unsigned)p, SUM_THREADS, bytes, st>>>(beta, Wf, wfix, N, p, s, t, mean, quant, conc, staged);
    return cudaGetLastError();
}

cudaError_t launch_accept_rate(const unsigned long long* acc, int T, double denom, double* rate, cudaStream_t st)
{
    k_accept_rate<<<(T + 127) / 128, 128, 0, st>>>(acc, T, denom, rate);
    return cudaGetLastError();
}

cudaError_t launch_adapt_lambda(double* lam, const unsigned long long* acc, double denom, cudaStream_t st)
{
    k_adapt_lambda<<<1, 32, 0, st>>>(lam, acc, denom);
    return cudaGetLastError();
}

cudaError_t launch_set_f64(double* ptr, double v, cudaStream_t st)
{
    k_set_f64<<<1, 32, 0, st>>>(ptr, v);
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
