// k_map.cu -- MAP estimates along the scale path by EM (Section 2.1; Section 4.1 for their
// use at every scale).
//
// The scale-mixture representation of the generalized t prior turns each EM step into a
// weighted-L1 logistic regression (eqs. beta_it and adapt_weights):
//   w_j = (a+1) / (a c + |beta_j|)   (double exponential: 1/c)
//   beta <- argmax_beta l(beta) - sum_j w_j |beta_j|.
// One thread block runs one EM solve. The inner convex problem is solved by proximal
// gradient steps beta <- S(z + grad l(z) / L, w / L) with L = ||X||_2^2 / 4 (the logistic
// loss's curvature bound), Nesterov momentum, and the gradient-based restart of
// O'Donoghue and Candes (2015): momentum is dropped whenever (z - beta') . (beta' - beta) > 0.
// Each step is two FP32 matrix-vector products with the standardised X, both from X^T
// log2(e) in [p][n] layout (coalesced columns for X z, coalesced rows for X^T r).
//
// Along a sweep (Section 4.1): at step t the EM starts from the particle with the highest
// posterior density and from the previous step's MAP, and keeps the mode with the higher
// log posterior l(beta) + log p(beta | a, c_t). With A_t the mode from the best particle this
// is the recurrence S_0 = A_0, S_t = better(A_t, EM(c_t, S_{t-1})), solved here in parallel
// over t by Jacobi rounds: round 0 solves every A_t at once; round k re-solves
// EM(c_t, S_{t-1}) only for the steps whose predecessor changed in round k - 1. After round
// k the first k + 1 entries are final, and a round that changes nothing has reached the
// recurrence's unique solution. One EM solve is a deterministic function of its start and
// c, so the result is bit-identical to walking the steps in order.
#include <cfloat>
#include <cmath>

#include "spa_device.cuh"
#include "spa_internal.h"

namespace spa {

namespace {

constexpr int MAP_THREADS = 512;
constexpr int MAP_MAX_INNER = 4000;  // proximal-gradient steps per EM step

__device__ __forceinline__ float block_sum_f(float v, float* red)
{
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += red[k];
    return r;
}

__device__ __forceinline__ float block_max_f(float v, float* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = fmaxf(r, red[k]);
    return r;
}

__device__ __forceinline__ double block_sum_d(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += red[k];
    return r;
}

// eta = X z, one thread per individual: it walks column j of X^T log2(e) (consecutive
// threads read consecutive individuals, so every load is coalesced; a row of X would put
// each thread on its own cache line), z from shared memory, scaled back by ln 2
__device__ void gemv_x(const MapData& d, const float* z, float* eta)
{
    for (int64_t i = threadIdx.x; i < d.n; i += blockDim.x) {
        const float* col = d.XT2 + i;
        float a0 = 0.0f, a1 = 0.0f;
        int j = 0;
        for (; j + 1 < d.p; j += 2) {
            a0 = fmaf(col[(int64_t)j * d.n], z[j], a0);
            a1 = fmaf(col[(int64_t)(j + 1) * d.n], z[j + 1], a1);
        }
        if (j < d.p) a0 = fmaf(col[(int64_t)j * d.n], z[j], a0);
        eta[i] = (a0 + a1) * 0.69314718f;
    }
}

// g = X^T r: warp w takes markers j = w, w + W, ...; its lanes split the individuals (rows of
// X^T log2(e), scaled back by ln 2)
__device__ void gemv_xt(const MapData& d, const float* r, float* g)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, W = blockDim.x >> 5;
    for (int j = w; j < d.p; j += W) {
        const float* xr = d.XT2 + (int64_t)j * d.n;
        float acc = 0.0f;
        for (int64_t i = lane; i < d.n; i += 32) acc = fmaf(xr[i], r[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) g[j] = acc * 0.69314718f;
    }
}

__device__ __forceinline__ float sigmoid_f(float x)
{
    const float e = __expf(-fabsf(x));
    return x >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e);
}

// log p(b | a, c) of one coordinate, FP64 (the constant -log 2c included)
__device__ __forceinline__ double logprior1_d(PriorArgs pr, double c, float b)
{
    const double x = fabs((double)b);
    return pr.de ? -log(2.0 * c) - x / c : -log(2.0 * c) - ((double)pr.a + 1.0) * log1p(x / ((double)pr.a * c));
}

// Shared-memory plan of one solve: beta, z, prev, w, g (p each), eta / residual (n),
// reduction scratch.
struct MapSmem {
    float *beta, *z, *prev, *w, *g, *eta;
    float* red;
    double* redd;
};

__device__ MapSmem map_smem(float* base, int64_t n, int p)
{
    MapSmem m;
    m.beta = base;
    m.z = m.beta + p;
    m.prev = m.z + p;
    m.w = m.prev + p;
    m.g = m.w + p;
    m.eta = m.g + p;
    m.red = m.eta + n;
    uintptr_t a = reinterpret_cast<uintptr_t>(m.red + 64);
    m.redd = reinterpret_cast<double*>((a + 7) & ~(uintptr_t)7);
    return m;
}

// One EM solve by the whole block from the point already in m.beta; returns the log
// posterior l(beta) + log p(beta | a, c) at the mode (FP64 sums).
__device__ double map_em_block(const MapData& d, double c, int max_em, float tol, const MapSmem& m)
{
    const int p = d.p;
    const float L = *d.lip, invL = 1.0f / L;
    const float ac = (float)((double)d.pr.a * c), a1 = d.pr.a + 1.0f, invc = (float)(1.0 / c);
    const float tol_in = 0.1f * tol;
    for (int em = 0; em < max_em; ++em) {
        for (int j = threadIdx.x; j < p; j += blockDim.x) {
            m.w[j] = d.pr.de ? invc : a1 / (ac + fabsf(m.beta[j]));
            m.prev[j] = m.beta[j];
            m.z[j] = m.beta[j];
        }
        __syncthreads();
        float tk = 1.0f;
        for (int it = 0; it < MAP_MAX_INNER; ++it) {
            gemv_x(d, m.z, m.eta);
            __syncthreads();
            for (int64_t i = threadIdx.x; i < d.n; i += blockDim.x)
                m.eta[i] = (d.y[i] ? 1.0f : 0.0f) - sigmoid_f(m.eta[i]);
            __syncthreads();
            gemv_xt(d, m.eta, m.g);
            __syncthreads();
            float dot = 0.0f, diff = 0.0f;
            for (int j = threadIdx.x; j < p; j += blockDim.x) {
                const float u = fmaf(m.g[j], invL, m.z[j]), k = m.w[j] * invL;
                const float bn = u > k ? u - k : (u < -k ? u + k : 0.0f);
                dot += (m.z[j] - bn) * (bn - m.beta[j]);
                diff = fmaxf(diff, fabsf(bn - m.beta[j]));
                m.g[j] = bn;  // the new point
            }
            dot = block_sum_f(dot, m.red);
            diff = block_max_f(diff, m.red);
            const bool restart = dot > 0.0f;
            const float tn = restart ? 1.0f : 0.5f * (1.0f + sqrtf(fmaf(4.0f * tk, tk, 1.0f)));
            const float mom = restart ? 0.0f : (tk - 1.0f) / tn;
            for (int j = threadIdx.x; j < p; j += blockDim.x) {
                const float bn = m.g[j];
                m.z[j] = fmaf(mom, bn - m.beta[j], bn);
                m.beta[j] = bn;
            }
            tk = tn;
            __syncthreads();
            if (diff < tol_in) break;
        }
        float ch = 0.0f;
        for (int j = threadIdx.x; j < p; j += blockDim.x) ch = fmaxf(ch, fabsf(m.beta[j] - m.prev[j]));
        ch = block_max_f(ch, m.red);
        if (ch < tol) break;
    }
    gemv_x(d, m.beta, m.eta);
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < d.n; i += blockDim.x) {
        const double e = (double)m.eta[i];
        acc += (d.y[i] ? e : 0.0) - (fmax(e, 0.0) + log1p(exp(-fabs(e))));
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) acc += logprior1_d(d.pr, c, m.beta[j]);
    return block_sum_d(acc, m.redd);
}

// S independent solves (one block each) from beta0[s].
__global__ void __launch_bounds__(MAP_THREADS) k_map(MapData d, const float* __restrict__ beta0, double c, int max_em,
                                                    float tol, float* __restrict__ beta_out, double* __restrict__ lp_out)
{
    extern __shared__ float map_sm[];
    const MapSmem m = map_smem(map_sm, d.n, d.p);
    const int s = blockIdx.x;
    for (int j = threadIdx.x; j < d.p; j += blockDim.x) m.beta[j] = beta0[(int64_t)s * d.p + j];
    __syncthreads();
    const double lp = map_em_block(d, c, max_em, tol, m);
    for (int j = threadIdx.x; j < d.p; j += blockDim.x) beta_out[(int64_t)s * d.p + j] = m.beta[j];
    if (threadIdx.x == 0) lp_out[s] = lp;
}

// One Jacobi round of the MAP path recurrence, block t = step t. Round 0 solves from the
// step's best particle into A / lpA and seeds S = A with every step marked changed. Round
// k >= 1 reads the previous round's S_r / lpS_r / chg_r and writes S_w / lpS_w / chg_w: a
// step whose predecessor did not change copies its entry; the others solve
// EM(c_t, S_r[t-1]), keep it if its log posterior is above lpA[t] (ties keep A_t), and
// count themselves in *n_changed when the kept mode differs from S_r[t].
__global__ void __launch_bounds__(MAP_THREADS) k_map_round(MapData d, const float* __restrict__ best,
                                                          const double* __restrict__ sched, int round, int max_em,
                                                          float tol, float* __restrict__ A, double* __restrict__ lpA,
                                                          const float* __restrict__ S_r, const double* __restrict__ lpS_r,
                                                          const int* __restrict__ chg_r, float* __restrict__ S_w,
                                                          double* __restrict__ lpS_w, int* __restrict__ chg_w,
                                                          int* __restrict__ n_changed)
{
    extern __shared__ float map_sm[];
    const MapSmem m = map_smem(map_sm, d.n, d.p);
    const int p = d.p, t = blockIdx.x;
    const int64_t o = (int64_t)t * p;
    const double c = sched[t];
    if (round == 0) {
        for (int j = threadIdx.x; j < p; j += blockDim.x) m.beta[j] = best[o + j];
        __syncthreads();
        const double lp = map_em_block(d, c, max_em, tol, m);
        for (int j = threadIdx.x; j < p; j += blockDim.x) {
            A[o + j] = m.beta[j];
            S_w[o + j] = m.beta[j];
        }
        if (threadIdx.x == 0) {
            lpA[t] = lp;
            lpS_w[t] = lp;
            chg_w[t] = 1;
        }
        return;
    }
    if (t == 0 || chg_r[t - 1] == 0) {
        for (int j = threadIdx.x; j < p; j += blockDim.x) S_w[o + j] = S_r[o + j];
        if (threadIdx.x == 0) {
            lpS_w[t] = lpS_r[t];
            chg_w[t] = 0;
        }
        return;
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) m.beta[j] = S_r[o - p + j];
    __syncthreads();
    const double lp2 = map_em_block(d, c, max_em, tol, m);
    const bool chain = lp2 > lpA[t];
    float ndiff = 0.0f;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        const float v = chain ? m.beta[j] : A[o + j];
        S_w[o + j] = v;
        if (__float_as_uint(v) != __float_as_uint(S_r[o + j])) ndiff = 1.0f;
    }
    ndiff = block_max_f(ndiff, m.red);
    if (threadIdx.x == 0) {
        const double lpn = chain ? lp2 : lpA[t];
        const bool changed = ndiff > 0.0f || lpn != lpS_r[t];
        lpS_w[t] = lpn;
        chg_w[t] = changed ? 1 : 0;
        if (changed) atomicAdd(n_changed, 1);
    }
}

// The particle of highest posterior density at step t: sp (l pair) + coef (log-prior pair)
// (the constant -p log 2c is common to all particles); ties go to the lowest index. One block.
__global__ void __launch_bounds__(1024) k_best_particle(MhState s, const float* __restrict__ beta, int64_t N, int p,
                                                       PriorArgs pr, const double* __restrict__ sched, int t,
                                                       float* __restrict__ best)
{
    __shared__ float bv[32];
    __shared__ long long bi[32];
    const float coef = pr.de ? (float)(-1.0 / sched[t]) : -(pr.a + 1.0f);
    float v = -FLT_MAX;
    long long idx = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const float2 L = s.llq[i], Q = s.lpq[i];
        const float lpv = s.sp_scale * (L.x + L.y) + coef * (Q.x + Q.y);
        if (lpv > v) {
            v = lpv;
            idx = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const long long i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (v2 > v || (v2 == v && i2 < idx)) {
            v = v2;
            idx = i2;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        bv[threadIdx.x >> 5] = v;
        bi[threadIdx.x >> 5] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float bb = bv[0];
        long long ii = bi[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
            if (bv[k] > bb || (bv[k] == bb && bi[k] < ii)) {
                bb = bv[k];
                ii = bi[k];
            }
        bi[0] = ii;
    }
    __syncthreads();
    const long long w = bi[0];
    for (int j = threadIdx.x; j < p; j += blockDim.x) best[(int64_t)t * p + j] = beta[w * p + j];
}

// ||X||_2^2 / 4 by power iteration on X^T X (200 steps from the all-ones vector), with a 2%
// margin so the step 1/L stays below the inverse curvature bound. One block.
__global__ void __launch_bounds__(MAP_THREADS) k_map_lipschitz(MapData d, float* __restrict__ lip_out)
{
    extern __shared__ float map_sm[];
    const MapSmem m = map_smem(map_sm, d.n, d.p);
    for (int j = threadIdx.x; j < d.p; j += blockDim.x) m.z[j] = 1.0f;
    __syncthreads();
    float lam = 0.0f;
    for (int it = 0; it < 200; ++it) {
        gemv_x(d, m.z, m.eta);
        __syncthreads();
        gemv_xt(d, m.eta, m.g);
        __syncthreads();
        float s2 = 0.0f;
        for (int j = threadIdx.x; j < d.p; j += blockDim.x) s2 += m.g[j] * m.g[j];
        const float nrm = sqrtf(block_sum_f(s2, m.red));
        float z2 = 0.0f;
        for (int j = threadIdx.x; j < d.p; j += blockDim.x) z2 += m.z[j] * m.z[j];
        lam = nrm / sqrtf(block_sum_f(z2, m.red));  // ||X^T X z|| / ||z||
        for (int j = threadIdx.x; j < d.p; j += blockDim.x) m.z[j] = m.g[j] / nrm;
        __syncthreads();
    }
    if (threadIdx.x == 0) *lip_out = 0.25f * lam * 1.02f;
}

size_t map_smem_bytes(int64_t n, int p) { return sizeof(float) * (size_t)(5 * p + n + 64) + sizeof(double) * 33; }

}  // namespace

bool map_fits(int64_t n, int p) { return map_smem_bytes(n, p) <= MAP_SMEM_MAX; }

cudaError_t map_init_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_map, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MAP_SMEM_MAX);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_map_round, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MAP_SMEM_MAX);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_map_lipschitz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MAP_SMEM_MAX);
    return e;
}

cudaError_t launch_map_lipschitz(const MapData& d, float* lip, cudaStream_t st)
{
    k_map_lipschitz<<<1, MAP_THREADS, map_smem_bytes(d.n, d.p), st>>>(d, lip);
    return cudaGetLastError();
}

cudaError_t launch_map(const MapData& d, const float* beta0, int S, double c, int max_em, float tol, float* beta_out,
                       double* lp_out, cudaStream_t st)
{
    k_map<<<S, MAP_THREADS, map_smem_bytes(d.n, d.p), st>>>(d, beta0, c, max_em, tol, beta_out, lp_out);
    return cudaGetLastError();
}

cudaError_t launch_map_round(const MapData& d, const float* best, const double* sched, int T, int round, int max_em,
                             float tol, const MapRoundBufs& b, cudaStream_t st)
{
    const int r = (round + 1) & 1, w = round & 1;
    const int64_t tp = (int64_t)T * d.p;
    k_map_round<<<T, MAP_THREADS, map_smem_bytes(d.n, d.p), st>>>(
        d, best, sched, round, max_em, tol, b.A, b.lpA, b.S + r * tp, b.lpS + r * T, b.chg + r * T, b.S + w * tp,
        b.lpS + w * T, b.chg + w * T, b.n_changed);
    return cudaGetLastError();
}

cudaError_t launch_best_particle(const MhState& s, const float* beta, int64_t N, int p, PriorArgs pr,
                                 const double* sched, int t, float* best, cudaStream_t st)
{
    k_best_particle<<<1, 1024, 0, st>>>(s, beta, N, p, pr, sched, t, best);
    return cudaGetLastError();
}

}  // namespace spa
