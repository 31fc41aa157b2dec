// k_smc.cu -- the per-step kernels of the SMC sampler over the prior scale (Section 4).
//
// Particle state: beta [N][p] FP32 (particle-major); the log-likelihood and the log-prior
// term sum as compensated FP32 pairs (llq, lpq; the log-prior without the constant
// -p log(2c), which cancels in every ratio taken at one scale; the change of scale is
// handled by the incremental weight in FP64); normalised log-weights and weights
// (WeightArrays).
//
// Precision plan for GB300: the CUDA-core FP64 rate is a small fraction of FP32 and an
// FP64 warp instruction costs a full warp's issue time even with one lane active. So sums
// over markers run in FP32 with compensated (TwoSum) accumulation, the Metropolis-Hastings
// ratios are formed in FP32 from compensated pairs, and FP64 appears only in the weights
// (incremental weight, log-sum-exp, ESS, log-evidence; one thread per particle) and in the
// resampling cumulative sum, whose association order is specified.
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
__device__ __forceinline__ float prior_term(float b, float inv_ac, int de)
{
    const float x = fabsf(b);
    return de ? x : log1pf(x * inv_ac);
}
__device__ __forceinline__ double prior_coef(PriorArgs pr, double c) { return pr.de ? -1.0 / c : -((double)pr.a + 1.0); }

// The Gt terms of four coordinates at once: log1p(x0) + ... + log1p(x3) with x = |b|/(a c),
// as the logarithm of the product of the factors 1 + x_k (one logarithm instead of four).
// Each factor and product carries a relative rounding of 2^-24, so the sum is accurate to
// a few 1e-7 in absolute terms, about the same as four rounded log1p terms of moderate size.
// Products beyond FP32 range (factors near 1e9) take the four logarithms instead. Every
// kernel that forms a state's log-prior sum for the MH test (the moves, and the reweighting's
// sum at the new scale) uses this grouping when p % 4 == 0, so that the test compares one
// function of the state.
__device__ __forceinline__ float prior_terms4(float4 b, float inv_ac)
{
    const float f0 = fmaf(fabsf(b.x), inv_ac, 1.0f), f1 = fmaf(fabsf(b.y), inv_ac, 1.0f);
    const float f2 = fmaf(fabsf(b.z), inv_ac, 1.0f), f3 = fmaf(fabsf(b.w), inv_ac, 1.0f);
    const float q = (f0 * f1) * (f2 * f3);
    if (q <= FLT_MAX) return logf(q);
    return log1pf(fabsf(b.x) * inv_ac) + log1pf(fabsf(b.y) * inv_ac) + log1pf(fabsf(b.z) * inv_ac) +
           log1pf(fabsf(b.w) * inv_ac);
}

// The prior's gradient in MALA's drift. The drift can be any fixed function of the state:
// the MH test evaluates the forward and reverse proposal densities with this same function,
// so the fast quotient (within 2 ulp) keeps each step's kernel exactly pi_t-invariant.
__device__ __forceinline__ float dlogprior(float b, float a1, float ac, float inv_c, int de)
{
    const float sg = (b > 0.0f) ? 1.0f : ((b < 0.0f) ? -1.0f : 0.0f);
    return de ? -sg * inv_c : __fdividef(-a1 * sg, ac + fabsf(b));
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

// Four consecutive coordinates j..j+3 (j a multiple of 4): two 8-byte stores per half.
__device__ __forceinline__ float pack_coord4(__nv_bfloat16* __restrict__ Arow, int Kp, int j, float4 b, float4 l2e,
                                             float4 mf)
{
    const float bt[4] = {b.x * l2e.x, b.y * l2e.y, b.z * l2e.z, b.w * l2e.w};
    __align__(8) __nv_bfloat16 hi[4];
    __align__(8) __nv_bfloat16 lo[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) split_bf16(bt[k], hi[k], lo[k]);
    *reinterpret_cast<uint2*>(Arow + j) = *reinterpret_cast<const uint2*>(hi);
    *reinterpret_cast<uint2*>(Arow + Kp + j) = *reinterpret_cast<const uint2*>(lo);
    return mf.x * bt[0] + mf.y * bt[1] + mf.z * bt[2] + mf.w * bt[3];
}

__device__ __forceinline__ void pack_offset(__nv_bfloat16* __restrict__ Arow, int Kp, int p, float off)
{
    __nv_bfloat16 hi, lo;
    split_bf16(-off, hi, lo);
    Arow[p] = hi;
    Arow[Kp + p] = lo;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
// read-only path: per-coordinate constants no thread writes while the kernel runs
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float comp(const float4& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }

// ------------------------------------------------------------ Metropolis-Hastings test
// The log-likelihood of particle i is sp_scale * (sum of the GEMM partials + ydq[i]), kept
// as a compensated FP32 pair (s, c) in partial units; the log-prior is coef(c_t) * (sum of
// log1p(|b|/(a c_t)) or |b|), kept as the pair of that sum. At one scale both differences
// of the MH ratio are between nearby values, so they are formed in FP32 from the pairs:
// s' - s is exact when the two are within a factor of two, and the c parts carry the rest.

// The block's proposals' softplus partials, gathered for the MH tests (one warp per particle,
// WARPS particles per block): thread t adds the chunks q = t / WARPS, t / WARPS + 32, ... of
// particle WARPS blockIdx.x + t % WARPS, so the WARPS threads of a group read one 32-byte
// sector per chunk, where a warp per particle touches one sector per lane. Slice s of a
// particle is exactly the compensated partial sum that lane s of a warp-per-particle loop
// over q = s, s + 32, ... forms, so the warp's tree over the slices gives the same bits.
struct PartSlices {
    float2 v[32][WARPS];
};
__device__ __forceinline__ void gather_partials(const MhState& s, int64_t N, PartSlices& sh)
{
    const int k = threadIdx.x % WARPS, slice = threadIdx.x / WARPS;
    const int64_t i = (int64_t)blockIdx.x * WARPS + k;
    FSum L;
    if (i < N)
        for (int q = slice; q < s.n_parts; q += 32) L.add(s.partial[(int64_t)q * s.ld_part + i]);
    sh.v[slice][k] = make_float2(L.s, L.c);
}

// The proposal's log-likelihood pair: the warp sums the slices, then adds y . eta.
__device__ __forceinline__ FSum proposal_loglik(const MhState& s, const PartSlices& sh, int64_t i, int lane)
{
    FSum L;
    const float2 v = sh.v[lane][threadIdx.x >> 5];
    L.s = v.x;
    L.c = v.y;
    L = warp_sum(L);
    const float2 yd = s.ydq[i];
    L.add(yd.x);
    L.add(yd.y);
    return L;
}

// log U of the MH test of move m for the block's particles (one warp per particle, so
// blockDim.x / 32 of them), by the kernel that proposes move m: lanes 0.. of warp 0 draw
// them side by side instead of lane 0 of every warp one at a time in the test.
__device__ __forceinline__ void draw_accept_logu(const MhState& s, int64_t N, int t, uint32_t m, uint64_t seed)
{
    const int lane = threadIdx.x & 31;
    if (!s.lu || threadIdx.x >= 32 || lane >= (int)(blockDim.x >> 5)) return;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + lane;
    if (i >= N) return;
    const uint4 u = philox4x32_10(make_uint4(0u, (uint32_t)i, (uint32_t)t, (TAG_ACCEPT << 16) | m), seed_key(seed));
    s.lu[(int64_t)(m & 1u) * s.ld_lu + i] = logf(u01_open_f(u.x));
}

// Warp-cooperative MH test of particle i's pending proposal; `extra` is the MALA
// q-correction. Lane 0 decides with the accept uniform of move m_prev (drawn by the kernel
// that proposed it) and, on acceptance, moves the proposal's log-likelihood and log-prior
// into the current state. Returns the decision on every lane.
__device__ __forceinline__ bool mh_decide(const MhState& s, const PartSlices& sh, int64_t i, int lane, float coef,
                                          float extra, uint32_t m_prev, uint32_t* err)
{
    const FSum L = proposal_loglik(s, sh, i, lane);
    int accept = 0;
    if (lane == 0) {
        const float2 L0 = s.llq[i];
        const float2 Q1 = s.lpt_p[i], Q0 = s.lpq[i];
        // written two launches back, by the kernel that proposed (read from L2)
        const float lu = __ldcg(s.lu + (int64_t)(m_prev & 1u) * s.ld_lu + i);
        const float dL = (L.s - L0.x) + (L.c - L0.y);
        const float dQ = (Q1.x - Q0.x) + (Q1.y - Q0.y);
        // rounded as written (no contraction), so that the decision does not depend on
        // how the compiler schedules the surrounding code
        const float log_alpha = __fadd_rn(__fadd_rn(__fmul_rn(s.sp_scale, dL), __fmul_rn(coef, dQ)), extra);
        if (!isfinite(L.s)) atomicOr(err, DERR_NONFINITE);
        accept = lu < log_alpha;
        if (accept) {
            s.llq[i] = make_float2(L.s, L.c);
            s.lpq[i] = Q1;
        }
    }
    return __shfl_sync(0xffffffffu, accept, 0) != 0;
}


// ------------------------------------------------------------ RW move kernel
// One warp per particle. With DECIDE, the warp first runs the MH test of the proposal
// left by the previous move (its log-likelihood partials are complete, the GEMM having run
// in between) and, on acceptance, writes that proposal back as the particle's state while
// reading it. Then it draws the next random-walk proposal beta' = beta + sigma xi from the
// (possibly just accepted) state: beta' to beta_p, the compensated log-prior term sum to
// lpt_p, y . eta' = beta' . v to ydq and (A != NULL) the split-BF16 GEMM row
// [hi(bt) | lo(bt)] with bt_j = beta'_j log2(e)/s_j and the offset o = -sum_j m_j bt_j in
// column p. noise = 0 packs beta unchanged (log-likelihood entry points, t = 0).
// Lane l handles the 4-coordinate groups g = l, l+32, ... (one Philox block of normals).

// One 4-coordinate group of a random-walk proposal (VEC: p % 4 == 0, float4 access).
// `live` masks the memory traffic of a lane whose group lies beyond p.
template <bool VEC>
__device__ __forceinline__ void rw_group(const MoveArgs& a, int p, int g, bool live, bool acc, int noise, float4 z,
                                         float inv_ac, int de, const float* src, float* dst, float* cur,
                                         __nv_bfloat16* Arow, FSum& lt, float& yd, float& off)
{
    const int j0 = 4 * g;
    if (VEC) {
        if (!live) return;
        const float4 b0 = ld4(src + j0);
        if (acc) st4(cur + j0, b0);
        const float4 sg = ld4(a.sigma + j0);
        const float4 b = noise ? make_float4(fmaf(sg.x, z.x, b0.x), fmaf(sg.y, z.y, b0.y), fmaf(sg.z, z.z, b0.z),
                                             fmaf(sg.w, z.w, b0.w))
                               : b0;
        st4(dst + j0, b);
        const float4 v = ld4(a.vy + j0);
        if (de) {
#pragma unroll
            for (int k = 0; k < 4; ++k) lt.add(fabsf(comp(b, k)));
        } else {
            lt.add(prior_terms4(b, inv_ac));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) yd = fmaf(comp(b, k), comp(v, k), yd);
        if (Arow) off += pack_coord4(Arow, a.Kp, j0, b, ld4(a.l2e_over_s + j0), ld4(a.mean_f + j0));
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = j0 + k;
            if (live && j < p) {
                const float b0 = src[j];
                if (acc) cur[j] = b0;
                const float b = noise ? fmaf(a.sigma[j], comp(z, k), b0) : b0;
                dst[j] = b;
                lt.add(prior_term(b, inv_ac, de));
                yd = fmaf(b, a.vy[j], yd);
                if (Arow) off += pack_coord(Arow, a.Kp, j, b, a.l2e_over_s, a.mean_f);
            }
        }
    }
}

// The scale constants of every step of a schedule, formed once per sweep, so that the move
// kernels read their step's float4 instead of redoing FP64 arithmetic in every block:
// x = a c_t (FP64 product), y = the log-prior coefficient (-(a+1), or -1/c_t for the double
// exponential), z = 1/c_t, w = 1/(a c_t) (FP64 quotient).
__global__ void k_step_constants(PriorArgs pr, const double* __restrict__ sched, int T, int p, float4* __restrict__ out,
                                 ReweightK* __restrict__ rk)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const double c = sched[t];
    float4 k;
    k.x = (float)((double)pr.a * c);
    k.z = 1.0f / (float)c;
    k.y = pr.de ? -k.z : -(pr.a + 1.0f);
    k.w = (float)(1.0 / ((double)pr.a * c));
    out[t] = k;
    if (rk) {
        ReweightK r{};
        if (t > 0) {
            const double cp = sched[t - 1];
            r.k1 = (float)(cp - c);
            r.kc = (float)c;
            r.kac = (float)((double)pr.a * cp);
            r.inv_ac = (float)(1.0 / ((double)pr.a * c));
            r.lbase = -(double)p * log(c / cp);
            r.dinv = 1.0 / c - 1.0 / cp;
        }
        rk[t] = r;
    }
}

// Accepted-proposal count of a block: one slot per warp, written by its lane 0 whatever the
// outcome; thread 0 sums them and makes one global atomic.
__device__ __forceinline__ void count_warps(unsigned long long* acc_count, const int* accw)
{
    __syncthreads();
    if (threadIdx.x == 0 && acc_count) {
        int s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += accw[k];
        if (s) atomicAdd(acc_count, (unsigned long long)s);
    }
}

template <bool DECIDE, bool VEC>
__global__ void __launch_bounds__(BLOCK, 5) k_move_rw(MoveArgs a, int64_t N, int p, PriorArgs pr,
                                                  const float4* __restrict__ stepk, int t, uint32_t m, uint32_t m_prev,
                                                  const uint64_t* __restrict__ seedp, int noise, uint32_t* err)
{
    __shared__ int accw[BLOCK / 32];
    __shared__ PartSlices parts;
    grid_dependency_wait();  // the previous kernel (the likelihood GEMM) has finished
    grid_launch_dependents();
    if (DECIDE) {
        gather_partials(a.mh, N, parts);
        __syncthreads();
    }
    const float4 sk = stepk[t];
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    bool acc = false;
    if (i < N) {
        const uint64_t seed = (noise || DECIDE) ? *seedp : 0ull;
        if (DECIDE) acc = mh_decide(a.mh, parts, i, lane, sk.y, 0.0f, m_prev, err);
        const float* src = (acc ? a.beta_p : a.beta) + i * p;
        float* dst = a.beta_p + i * p;
        float* cur = a.beta + i * p;
        __nv_bfloat16* Arow = a.A ? a.A + i * (int64_t)a.ldA : nullptr;
        FSum lt;
        float yd = 0.0f, off = 0.0f;
        const int groups = (p + 3) >> 2;
        for (int g = lane; g < groups; g += 32) {
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (noise) z = normals4(seed, (uint32_t)g, (uint32_t)i, (uint32_t)t, m);
            rw_group<VEC>(a, p, g, true, acc, noise, z, sk.w, pr.de, src, dst, cur, Arow, lt, yd, off);
        }
        lt = warp_sum(lt);
        yd = warp_sum(yd);
        off = warp_sum(off);
        if (lane == 0) {
            a.lpt_p[i] = make_float2(lt.s, lt.c);
            a.ydq[i] = make_float2(yd, 0.0f);
            if (Arow) pack_offset(Arow, a.Kp, p, off);
        }
    }
    if (noise) draw_accept_logu(a.mh, N, t, m, *seedp);
    if (DECIDE) {
        if (lane == 0) accw[threadIdx.x >> 5] = acc ? 1 : 0;
        count_warps(a.mh.acc_count, accw);
    }
}

// ------------------------------------------------------------ MALA move kernel
// The reverse move's residual sum of particle i's pending proposal (lane partial, before the
// warp sum): sum_j (beta_j - beta'_j - (h^2/2) D_j g'_j)^2 / D_j, g' = grad l' + the prior
// gradient at beta'. VEC (p % 4 == 0): lane l takes the 4-coordinate groups l, l + 32, ...
// with float4 loads; else coordinates l, l + 32, ...
template <bool VEC>
__device__ __forceinline__ FSum mala_reverse(const MoveArgs& a, int64_t i, int p, int lane, float h2, float a1, float ac,
                                             float inv_c, int de)
{
    FSum bwd;
    const float* b0 = a.beta + i * p;
    const float* b1 = a.beta_p + i * p;
    const float* g1 = a.gl_p + i * p;
    if (VEC) {
        for (int j0 = 4 * lane; j0 < p; j0 += 128) {
            const float4 x0 = ld4(b0 + j0), x1 = ld4(b1 + j0), gg = ld4(g1 + j0);
            const float4 Dv = ldg4(a.sigma + j0), iD = ldg4(a.inv_D + j0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float drift = h2 * comp(Dv, k) * (comp(gg, k) + dlogprior(comp(x1, k), a1, ac, inv_c, de));
                const float d = (comp(x0, k) - comp(x1, k)) - drift;
                bwd.add(d * d * comp(iD, k));
            }
        }
    } else {
        for (int j = lane; j < p; j += 32) {
            const float drift = h2 * a.sigma[j] * (g1[j] + dlogprior(b1[j], a1, ac, inv_c, de));
            const float d = (b0[j] - b1[j]) - drift;
            bwd.add(d * d * a.inv_D[j]);
        }
    }
    return bwd;
}

// beta' = beta + (h^2/2) D grad log pi_t(beta) + h D^{1/2} xi with D = diag(D_j) and
// h = lambda p^{-1/6} (written by the column-statistics kernel); grad log pi_t = grad l
// (stored per particle) + the prior gradient -(a+1) sgn(beta)/(a c + |beta|) (double
// exponential: -sgn(beta)/c). The forward density is evaluated at the proposal as
// written (rounded to FP32): fwd = sum_j (beta'_j - beta_j - (h^2/2) D_j g_j)^2 / D_j, so
// log q(beta'|beta) = -fwd/(2h^2) + const, the same formula as the reverse term. With
// DECIDE the warp first forms the reverse term of the pending proposal,
// bwd = sum_j (beta_j - beta'_j - (h^2/2) D_j g'_j)^2 / D_j, and runs its MH test with
// log alpha = l' + lp' - l - lp - (bwd - fwd)/(2h^2); an accepted proposal and its gradient
// are written back as the state while being read. At most 64 registers, so that 4 blocks
// fit an SM (1.68 waves of 8192 particle warps; the test variant would take 74 and 3 blocks).
template <bool DECIDE, bool VEC>
__global__ void __launch_bounds__(BLOCK, 4) k_move_mala(MoveArgs a, int64_t N, int p, PriorArgs pr,
                                                    const float4* __restrict__ stepk, int t, uint32_t m,
                                                    uint32_t m_prev, const uint64_t* __restrict__ seedp, uint32_t* err)
{
    __shared__ int accw[BLOCK / 32];
    __shared__ PartSlices parts;
    grid_dependency_wait();  // the previous kernel (the gradient finish, or the step's proposal scales) has finished
    grid_launch_dependents();
    if (DECIDE) {
        gather_partials(a.mh, N, parts);
        __syncthreads();
    }
    const float4 sk = stepk[t];
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    bool acc = false;
    if (i < N) {
        const uint64_t seed = *seedp;
        const float ac = sk.x, a1 = pr.a + 1.0f, inv_c = sk.z;
        const float h = *a.h, h2 = 0.5f * h * h;
        const float* D = a.sigma;
        if (DECIDE) {
            const FSum bwd = warp_sum(mala_reverse<VEC>(a, i, p, lane, h2, a1, ac, inv_c, pr.de));
            const float2 fw = a.fwd[i];
            const float extra = -((bwd.s - fw.x) + (bwd.c - fw.y)) / (2.0f * h * h);
            acc = mh_decide(a.mh, parts, i, lane, sk.y, extra, m_prev, err);
        }
        const float* src = (acc ? a.beta_p : a.beta) + i * p;
        const float* gsrc = (acc ? a.gl_p : a.gl) + i * p;
        float* cur = a.beta + i * p;
        float* gcur = a.gl + i * p;
        float* dst = a.beta_p + i * p;
        __nv_bfloat16* Arow = a.A ? a.A + i * (int64_t)a.ldA : nullptr;
        FSum lt, fw;
        float yd = 0.0f, off = 0.0f;
        const int groups = (p + 3) >> 2;
        const bool grouped = (p & 3) == 0 && !pr.de;  // the four-coordinate prior term
        if (VEC) {
            // p % 4 == 0: the same per-coordinate arithmetic on float4 groups, the state's and
            // the gradient's rows read and written 16 bytes at a time, the GEMM row 8
            for (int g = lane; g < groups; g += 32) {
                const float4 z4 = normals4(seed, (uint32_t)g, (uint32_t)i, (uint32_t)t, m);
                const int j0 = 4 * g;
                const float4 x0 = ld4(src + j0), g0 = ld4(gsrc + j0);
                if (acc) {
                    st4(cur + j0, x0);
                    st4(gcur + j0, g0);
                }
                const float4 Dv = ldg4(D + j0), sD = ldg4(a.sqrt_D + j0), iD = ldg4(a.inv_D + j0);
                const float4 v = ldg4(a.vy + j0);
                float bq[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float b0 = comp(x0, k);
                    const float drift = h2 * comp(Dv, k) * (comp(g0, k) + dlogprior(b0, a1, ac, inv_c, pr.de));
                    const float b = (b0 + drift) + h * comp(sD, k) * comp(z4, k);
                    const float d = (b - b0) - drift;
                    fw.add(d * d * comp(iD, k));
                    bq[k] = b;
                    yd = fmaf(b, comp(v, k), yd);
                }
                const float4 b4 = make_float4(bq[0], bq[1], bq[2], bq[3]);
                st4(dst + j0, b4);
                if (grouped) {
                    lt.add(prior_terms4(b4, sk.w));
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) lt.add(prior_term(bq[k], sk.w, pr.de));
                }
                if (Arow) off += pack_coord4(Arow, a.Kp, j0, b4, ldg4(a.l2e_over_s + j0), ldg4(a.mean_f + j0));
            }
        }
        for (int g = VEC ? groups : lane; g < groups; g += 32) {
            const float4 z4 = normals4(seed, (uint32_t)g, (uint32_t)i, (uint32_t)t, m);
            float bq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = 4 * g + k;
                if (j < p) {
                    const float b0 = src[j];
                    const float g0 = gsrc[j];
                    if (acc) {
                        cur[j] = b0;
                        gcur[j] = g0;
                    }
                    const float drift = h2 * D[j] * (g0 + dlogprior(b0, a1, ac, inv_c, pr.de));
                    const float b = (b0 + drift) + h * a.sqrt_D[j] * comp(z4, k);
                    dst[j] = b;
                    const float d = (b - b0) - drift;
                    fw.add(d * d * a.inv_D[j]);
                    bq[k] = b;
                    if (!grouped) lt.add(prior_term(b, sk.w, pr.de));
                    yd = fmaf(b, a.vy[j], yd);
                    if (Arow) off += pack_coord(Arow, a.Kp, j, b, a.l2e_over_s, a.mean_f);
                }
            }
            if (grouped) lt.add(prior_terms4(make_float4(bq[0], bq[1], bq[2], bq[3]), sk.w));
        }
        lt = warp_sum(lt);
        fw = warp_sum(fw);
        yd = warp_sum(yd);
        off = warp_sum(off);
        if (lane == 0) {
            a.lpt_p[i] = make_float2(lt.s, lt.c);
            a.fwd[i] = make_float2(fw.s, fw.c);
            a.ydq[i] = make_float2(yd, 0.0f);
            if (Arow) pack_offset(Arow, a.Kp, p, off);
        }
    }
    draw_accept_logu(a.mh, N, t, m, *seedp);
    if (DECIDE) {
        if (lane == 0) accw[threadIdx.x >> 5] = acc ? 1 : 0;
        count_warps(a.mh.acc_count, accw);
    }
}

// ------------------------------------------------- single-coordinate update cycle
// The paper's own kernel (Section 4.1, "Further details"): a cycle of single-coordinate
// random-walk Metropolis updates, j = 0..p-1 in order, each proposing beta_j' = beta_j +
// sd * xi, repeated M times per step. One warp per particle, one launch per step.
// eta2 = log2(e) X beta lives in shared memory (computed from X^T at the start of the step)
// and changes by x_.j delta when an update is accepted, so an update costs O(n):
//   delta l = delta v_j - ln 2 * sum_i [softplus2(eta2_i + x2_ij delta) - softplus2(eta2_i)]
// with the linear half from v = X^T y. softplus2 = max(eta2, 0) + log2(1 + 2^-|eta2|); the
// max parts are summed as differences, the log parts as the base-2 logarithm of the
// product of their factors (each in [1, 2], SITE_CHUNK per product), and each lane keeps
// that log for its individuals at the current state, so a trial needs one ex2 per
// individual. The normal is Box-Muller's cosine branch on words 0 and 1 of the Philox
// block (j, particle, t, TAG_SITE << 16 | m), word 2 the update's uniform.
constexpr int SITE_CHUNK = 64;

// Per-lane: sum over the lane's individuals r = lane + 32k of max(eta2', 0) - max(eta2, 0)
// (dm) and log2 of the product of (1 + 2^-|eta2'|) (returned), eta2' = eta2 + x2 delta.
__device__ __forceinline__ float site_trial(const float* __restrict__ eta, const float* __restrict__ xr, int n,
                                            int lane, float delta, float& dm)
{
    float lq = 0.0f, d = 0.0f;
    for (int k0 = 0; 32 * k0 < n; k0 += SITE_CHUNK) {
        float prod = 1.0f;
        const int r1 = min(n, 32 * (k0 + SITE_CHUNK));
        for (int r = lane + 32 * k0; r < r1; r += 32) {
            const float e0 = eta[r];
            const float e1 = fmaf(xr[r], delta, e0);
            d += fmaxf(e1, 0.0f) - fmaxf(e0, 0.0f);
            prod = fmaf(prod, ex2_approx(-fabsf(e1)), prod);
        }
        lq += lg2_approx(prod);
    }
    dm = d;
    return lq;
}

__global__ void k_move_site(SiteArgs a, int64_t N, int p, int n, PriorArgs pr, const float4* __restrict__ stepk, int t,
                            uint32_t m0, int M, const uint64_t* __restrict__ seedp)
{
    extern __shared__ float site_sm[];
    __shared__ int blk;
    const int wpc = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) blk = 0;
    __syncthreads();
    const float4 sk = stepk[t];
    float* eta = site_sm + (size_t)w * (size_t)(n + p);
    float* brow = eta + n;
    const int64_t i = (int64_t)blockIdx.x * wpc + w;
    if (i < N) {
        const uint64_t seed = *seedp;
        const float coef = sk.y, inv_ac = sk.w;
        float* bg = a.beta + i * p;
        for (int j = lane; j < p; j += 32) brow[j] = bg[j];
        for (int r = lane; r < n; r += 32) eta[r] = 0.0f;
        __syncwarp();
        for (int j = 0; j < p; ++j) {  // eta2 = X2 beta, marker by marker (coalesced rows of X^T)
            const float bj = brow[j];
            const float* xr = a.XT2 + (size_t)j * n;
            for (int r = lane; r < n; r += 32) eta[r] = fmaf(xr[r], bj, eta[r]);
        }
        float dm;
        float lq = site_trial(eta, a.XT2, n, lane, 0.0f, dm);  // delta = 0: the current state
        int nacc = 0;
        for (int mm = 0; mm < M; ++mm) {
            const uint32_t m = m0 + (uint32_t)mm;
            for (int j = 0; j < p; ++j) {
                const uint4 u = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)i, (uint32_t)t, (TAG_SITE << 16) | m),
                                              seed_key(seed));
                float sn, cs;
                sincospif(2.0f * u01_open_f(u.y), &sn, &cs);
                const float delta = a.sd * (sqrtf(-2.0f * logf(u01_open_f(u.x))) * cs);
                const float* xr = a.XT2 + (size_t)j * n;
                const float lq1 = site_trial(eta, xr, n, lane, delta, dm);
                const float dsp = warp_sum(dm + (lq1 - lq));
                const float b0 = brow[j], b1 = b0 + delta;
                const float dlp = coef * (prior_term(b1, inv_ac, pr.de) - prior_term(b0, inv_ac, pr.de));
                const float dl = fmaf(delta, a.vy[j], -0.69314718f * dsp);
                int acc = logf(u01_open_f(u.z)) < dl + dlp;
                acc = __shfl_sync(0xffffffffu, acc, 0);
                if (acc) {
                    for (int r = lane; r < n; r += 32) eta[r] = fmaf(xr[r], delta, eta[r]);
                    lq = lq1;
                    if (lane == 0) brow[j] = b1;
                    ++nacc;
                }
                __syncwarp();
            }
        }
        for (int j = lane; j < p; j += 32) bg[j] = brow[j];
        if (lane == 0 && nacc) atomicAdd(&blk, nacc);
        // the MH state at the end of the step, in the units the move kernels keep it:
        // l = beta . v - ln 2 (sum_i max(eta2_i, 0) + sum of the lanes' log products), and the
        // log-prior term sum
        if (a.llq) {
            float mx = 0.0f, yd = 0.0f;
            FSum lt;
            for (int r = lane; r < n; r += 32) mx += fmaxf(eta[r], 0.0f);
            for (int j = lane; j < p; j += 32) {
                yd = fmaf(brow[j], a.vy[j], yd);
                lt.add(prior_term(brow[j], inv_ac, pr.de));
            }
            const float sp2 = warp_sum(mx + lq);
            yd = warp_sum(yd);
            lt = warp_sum(lt);
            if (lane == 0) {
                a.llq[i] = make_float2((yd - 0.69314718f * sp2) * a.inv_sp_scale, 0.0f);
                a.lpq[i] = make_float2(lt.s, lt.c);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk && a.acc_count) atomicAdd(a.acc_count, (unsigned long long)blk);
}

// ------------------------------------------------------------ last move of a step
// MH test of the pending proposals (RW, or MALA with the reverse term), then accepted
// proposals (and their gradients) are copied into the state rows, so that between steps
// beta and gl hold the particles.
template <bool MALA, bool VEC>
__global__ void __launch_bounds__(BLOCK) k_move_commit(MoveArgs a, int64_t N, int p, PriorArgs pr,
                                                      const float4* __restrict__ stepk, int t, uint32_t m_prev,
                                                      const uint64_t* __restrict__ seedp, uint32_t* err)
{
    __shared__ int accw[BLOCK / 32];
    __shared__ PartSlices parts;
    grid_dependency_wait();
    gather_partials(a.mh, N, parts);
    __syncthreads();
    const float4 sk = stepk[t];
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    bool acc = false;
    if (i < N) {
        float extra = 0.0f;
        if (MALA) {
            const float ac = sk.x, a1 = pr.a + 1.0f, inv_c = sk.z;
            const float h = *a.h, h2 = 0.5f * h * h;
            const FSum bwd = warp_sum(mala_reverse<VEC>(a, i, p, lane, h2, a1, ac, inv_c, pr.de));
            const float2 fw = a.fwd[i];
            extra = -((bwd.s - fw.x) + (bwd.c - fw.y)) / (2.0f * h * h);
        }
        acc = mh_decide(a.mh, parts, i, lane, sk.y, extra, m_prev, err);
        if (acc) {
            const float* src = a.beta_p + i * p;
            float* dst = a.beta + i * p;
            if (VEC) {
                for (int j = 4 * lane; j < p; j += 128) st4(dst + j, ld4(src + j));
                if (MALA)
                    for (int j = 4 * lane; j < p; j += 128) st4(a.gl + i * p + j, ld4(a.gl_p + i * p + j));
            } else {
                for (int j = lane; j < p; j += 32) dst[j] = src[j];
                if (MALA)
                    for (int j = lane; j < p; j += 32) a.gl[i * p + j] = a.gl_p[i * p + j];
            }
        }
    }
    if (lane == 0) accw[threadIdx.x >> 5] = acc ? 1 : 0;
    count_warps(a.mh.acc_count, accw);
}

// ------------------------------------------------------------ log-likelihood finish
// The packed particles' log-likelihood as the state: llq (pair), lpq = lpt_p, and in FP64
// l = sp_scale (s + c) to logw (prior-IS weights at t = 0) and/or ll_out.
__global__ void __launch_bounds__(BLOCK) k_finish_loglik(MhState s, int64_t N, double* __restrict__ logw,
                                                        double* __restrict__ ll_out, uint32_t* __restrict__ err)
{
    __shared__ PartSlices parts;
    gather_partials(s, N, parts);
    __syncthreads();
    const int64_t i = warp_global_id();
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const FSum L = proposal_loglik(s, parts, i, lane);
    if (lane != 0) return;
    if (!isfinite(L.s)) atomicOr(err, DERR_NONFINITE);
    s.llq[i] = make_float2(L.s, L.c);
    s.lpq[i] = s.lpt_p[i];
    const double l = s.sp_scale_d * ((double)L.s + (double)L.c);
    if (logw) logw[i] = l;
    if (ll_out) ll_out[i] = l;
}

// ------------------------------------------------------------------ reweighting
// log w_i = sum_j log p(beta_ij | c_t) - log p(beta_ij | c_{t-1}) in the form without
// cancellation: -log(c_t/c_{t-1}) - (a+1) log1p(x (c_{t-1} - c_t) / (c_t (a c_{t-1} + x))),
// x = |beta_ij| (double exponential: -log(c_t/c_{t-1}) - x (1/c_t - 1/c_{t-1})).
// A block handles 32 particles: its warps form the FP32 row sums, then warp 0 finishes one
// particle per lane in FP64. The step's constants come from the per-sweep table.
constexpr int RW_PER_BLOCK = 8;
constexpr int RW_THREADS = 32 * RW_PER_BLOCK;

__global__ void __launch_bounds__(RW_THREADS) k_reweight(const float* __restrict__ beta, double* __restrict__ logw,
                                                   float2* __restrict__ lpq, int64_t N, int p, PriorArgs pr,
                                                   const ReweightK* __restrict__ rkp, int t, uint32_t* __restrict__ err)
{
    grid_dependency_wait();
    __shared__ float4 sums[RW_PER_BLOCK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * RW_PER_BLOCK;
    const ReweightK rk = rkp[t];
    const float k1 = rk.k1, kc = rk.kc, kac = rk.kac, inv_ac = rk.inv_ac;
    {
        const int q = w;
        const int64_t i = base + q;
        FSum sdiff, snew;
        if (i < N) {
            const bool grouped = (p & 3) == 0 && !pr.de;  // the moves' four-coordinate prior term
            for (int j = lane; j < p; j += 32) {
                const float x = fabsf(beta[i * p + j]);
                sdiff.add(pr.de ? x : log1pf(x * k1 / (kc * (kac + x))));
                if (!grouped) snew.add(prior_term(x, inv_ac, pr.de));
            }
            if (grouped)
                for (int g = lane; 4 * g < p; g += 32)
                    snew.add(prior_terms4(*reinterpret_cast<const float4*>(beta + i * p + 4 * g), inv_ac));
        }
        sdiff = warp_sum(sdiff);
        snew = warp_sum(snew);
        if (lane == 0) sums[q] = make_float4(sdiff.s, sdiff.c, snew.s, snew.c);
    }
    __syncthreads();
    if (w == 0 && lane < RW_PER_BLOCK) {
        const int64_t i = base + lane;
        if (i < N) {
            const float4 s = sums[lane];
            const double sd = (double)s.x + (double)s.y;
            const double d = pr.de ? rk.lbase - sd * rk.dinv : rk.lbase - ((double)pr.a + 1.0) * sd;
            const double nl = logw[i] + d;
            if (!isfinite(nl)) atomicOr(err, DERR_NONFINITE);
            logw[i] = nl;
            lpq[i] = make_float2(s.z, s.w);
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
constexpr int LSE_THREADS = 128;  // one weight per thread up to 128 x LSE_BLOCKS particles

__global__ void __launch_bounds__(LSE_THREADS) k_lse_partial(const double* __restrict__ logw, int64_t N,
                                                      double* __restrict__ scratch, unsigned int* __restrict__ counter,
                                                      int t, int mode, double ess_frac, double* __restrict__ ess_out,
                                                      double* __restrict__ logz_out, uint8_t* __restrict__ res_out,
                                                      int* __restrict__ flag, uint32_t* __restrict__ err)
{
    grid_dependency_wait();
    __shared__ double sh[BLOCK / 32];
    __shared__ bool last;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double mx = -DBL_MAX;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) mx = fmax(mx, logw[i]);
    const double mb = block_max_f64(mx, sh);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
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
    grid_dependency_wait();
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
// The cumulative sum C of W in the specified order: a running sum inside each 256-block
// in index order, a running sum of the block totals, C_i = carry(block) + local_i. cum holds
// N + ceil(N/256) + 1 doubles: the block-local running sums, then one carry per block, then u.
// Three kernels spread it over the SMs: the local sums (16 blocks of 256 per CTA, staged in
// shared memory with coalesced loads and stores; lane l of warp 0 runs block l's additions),
// the carries (one thread, in block order), and the search, which forms C_i = carry + local_i
// as it reads it. The association order, and so every bit of C, is that of the definition.
constexpr int RS_BLOCK = 256;         // cumulative-sum block of the specified association order
constexpr int RS_CHUNKS = 16;         // 256-blocks per CTA of the local pass (33 KB of shared memory)
constexpr int RS_PAD = RS_BLOCK + 1;  // shared-memory row of one 256-block (odd stride: no bank conflicts)
constexpr int RS_LOCAL_THREADS = 256;
constexpr size_t RS_LOCAL_SMEM = sizeof(double) * RS_CHUNKS * RS_PAD;
constexpr int RS_CARRY_THREADS = 1024;
constexpr int RS_TOT = 4096;  // block totals staged per pass of the carry kernel

__global__ void __launch_bounds__(RS_LOCAL_THREADS) k_resample_local(const double* __restrict__ W, int64_t N,
                                                                     double* __restrict__ cum,
                                                                     const int* __restrict__ flag)
{
    grid_dependency_wait();
    if (flag && *flag == 0) return;
    extern __shared__ double rs_sm[];
    const int64_t i0 = (int64_t)blockIdx.x * RS_CHUNKS * RS_BLOCK;
    const int64_t len = (N - i0 < (int64_t)RS_CHUNKS * RS_BLOCK) ? N - i0 : (int64_t)RS_CHUNKS * RS_BLOCK;
    for (int64_t e = threadIdx.x; e < len; e += RS_LOCAL_THREADS)
        rs_sm[(e / RS_BLOCK) * RS_PAD + (e % RS_BLOCK)] = W[i0 + e];
    __syncthreads();
    if (threadIdx.x < RS_CHUNKS) {
        const int c = threadIdx.x;
        const int64_t c0 = (int64_t)c * RS_BLOCK;
        if (c0 < len) {
            const int cl = (len - c0 < RS_BLOCK) ? (int)(len - c0) : RS_BLOCK;
            double* row = rs_sm + c * RS_PAD;
            double local = 0.0;
            for (int k = 0; k < cl; ++k) {
                local = __dadd_rn(local, row[k]);
                row[k] = local;
            }
            // the block total, turned into the block's carry by k_resample_carry
            cum[N + (i0 / RS_BLOCK) + c] = local;
        }
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < len; e += RS_LOCAL_THREADS) cum[i0 + e] = rs_sm[(e / RS_BLOCK) * RS_PAD + (e % RS_BLOCK)];
}

// carry[b] = total_0 + ... + total_{b-1} in block order (the totals are read from the carry
// slots and replaced), then the resampling uniform after the carries.
__global__ void __launch_bounds__(RS_CARRY_THREADS) k_resample_carry(int64_t N, double* __restrict__ cum,
                                                                     const int* __restrict__ flag, int t,
                                                                     const uint64_t* __restrict__ seedp,
                                                                     double u_override)
{
    grid_dependency_wait();
    if (flag && *flag == 0) return;
    __shared__ double tot[RS_TOT];
    const int tid = threadIdx.x;
    const int64_t nblk = (N + RS_BLOCK - 1) / RS_BLOCK;
    double* carry = cum + N;
    double run = 0.0;  // thread 0's running sum of block totals
    for (int64_t b0 = 0; b0 < nblk; b0 += RS_TOT) {
        const int64_t b1 = (b0 + RS_TOT < nblk) ? b0 + RS_TOT : nblk;
        for (int64_t b = b0 + tid; b < b1; b += RS_CARRY_THREADS) tot[b - b0] = carry[b];
        __syncthreads();
        if (tid == 0)
            for (int64_t b = b0; b < b1; ++b) {
                carry[b] = run;
                run = __dadd_rn(run, tot[b - b0]);
            }
        __syncthreads();
    }
    if (tid == 0) {
        if (seedp) {
            const uint4 u = philox4x32_10(make_uint4(0u, 0u, (uint32_t)t, TAG_RESAMPLE << 16), seed_key(*seedp));
            carry[nblk] = u01_d(u.x);
        } else {
            carry[nblk] = u_override;
        }
    }
}

// A_k = min{i : C_i > (k + u)/N}, clamped to N - 1, with C_i = carry(i / 256) + local_i (the
// first block's carry is 0 and its C_i is local_i, as in the definition). C is non-negative
// and non-decreasing, and for non-negative doubles the order of the bit patterns as signed
// integers is the numeric order, so the search compares integers.
__device__ __forceinline__ long long resample_c_bits(const double* __restrict__ cum, int64_t N, int64_t i)
{
    const double c = (i < RS_BLOCK) ? cum[i] : __dadd_rn(cum[N + i / RS_BLOCK], cum[i]);
    return __double_as_longlong(c);
}

__global__ void k_resample_search(const double* __restrict__ cum, int64_t N, int32_t* __restrict__ idx,
                                  const int* __restrict__ flag)
{
    grid_dependency_wait();
    if (flag && *flag == 0) return;
    const int64_t nblk = (N + RS_BLOCK - 1) / RS_BLOCK;
    const double u = cum[N + nblk];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const long long target = __double_as_longlong(__ddiv_rn(__dadd_rn((double)k, u), (double)N));
        int64_t lo = 0, hi = N;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (resample_c_bits(cum, N, mid) > target)
                hi = mid;
            else
                lo = mid + 1;
        }
        idx[k] = (int32_t)(lo < N ? lo : N - 1);
    }
}

// Ancestor rows into the scratch buffers, one warp per new particle k: beta_tmp[k] =
// beta[idx[k]] (and the gradient rows for MALA), with the log-likelihood and log-prior pairs.
template <bool VEC>
__global__ void __launch_bounds__(BLOCK) k_gather(const int32_t* __restrict__ idx, const float* __restrict__ beta,
                                                 float* __restrict__ beta_tmp, const float2* __restrict__ llq,
                                                 const float2* __restrict__ lpq, float2* __restrict__ llq_tmp,
                                                 float2* __restrict__ lpq_tmp, const float* __restrict__ g,
                                                 float* __restrict__ g_tmp, int64_t N, int p, const int* __restrict__ flag)
{
    grid_dependency_wait();
    if (*flag == 0) return;
    const int64_t k = warp_global_id();
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    const int64_t a = idx[k];
    const float* src = beta + a * p;
    float* dst = beta_tmp + k * p;
    if (VEC) {
        for (int j = 4 * lane; j < p; j += 128) st4(dst + j, ld4(src + j));
        if (g)
            for (int j = 4 * lane; j < p; j += 128) st4(g_tmp + k * p + j, ld4(g + a * p + j));
    } else {
        for (int j = lane; j < p; j += 32) dst[j] = src[j];
        if (g)
            for (int j = lane; j < p; j += 32) g_tmp[k * p + j] = g[a * p + j];
    }
    if (lane == 0) {
        llq_tmp[k] = llq[a];
        lpq_tmp[k] = lpq[a];
    }
}

// The resampled particles back into the state, with uniform weights (log(1/N), 1/N and
// round(2^31/N), formed on the host).
template <bool VEC>
__global__ void __launch_bounds__(BLOCK) k_copyback(float* __restrict__ beta, const float* __restrict__ beta_tmp,
                                                   float2* __restrict__ llq, float2* __restrict__ lpq,
                                                   const float2* __restrict__ llq_tmp, const float2* __restrict__ lpq_tmp,
                                                   float* __restrict__ g, const float* __restrict__ g_tmp, WeightArrays w,
                                                   int64_t N, int p, const int* __restrict__ flag, double lw, double wi,
                                                   uint32_t wf)
{
    grid_dependency_wait();
    if (*flag == 0) return;
    const int64_t k = warp_global_id();
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    const int64_t o = k * p;
    if (VEC) {
        for (int j = 4 * lane; j < p; j += 128) st4(beta + o + j, ld4(beta_tmp + o + j));
        if (g)
            for (int j = 4 * lane; j < p; j += 128) st4(g + o + j, ld4(g_tmp + o + j));
    } else {
        for (int j = lane; j < p; j += 32) beta[o + j] = beta_tmp[o + j];
        if (g)
            for (int j = lane; j < p; j += 32) g[o + j] = g_tmp[o + j];
    }
    if (lane == 0) {
        llq[k] = llq_tmp[k];
        lpq[k] = lpq_tmp[k];
        w.logw[k] = lw;
        w.W[k] = wi;
        w.Wf[k] = (float)wi;
        w.wfix[k] = wf;
    }
}

// -------------------------------------------------------------- column moments
constexpr int CS_ROWS = 8;

__global__ void k_colstats_partial(const float* __restrict__ beta, const float* __restrict__ Wf, int64_t N, int p,
                                   float4* __restrict__ part)
{
    grid_dependency_wait();
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
    grid_dependency_wait();
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
        // MALA's D_j, and beside it sqrt(D_j) and 1/D_j for the proposal and its densities
        const double D = fmax(var, fl * fl);
        scale_out[j] = (float)D;
        scale_out[p + j] = (float)sqrt(D);
        scale_out[2 * p + j] = (float)(1.0 / D);
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
// reaches the target. Lane l owns bins l*per .. l*per+per-1 and sums them starting at a
// lane-dependent offset, so the 32 lanes hit 32 different shared-memory banks.
__device__ int warp_find_bin(const uint32_t* hist, int nbins, unsigned long long target, unsigned long long* below)
{
    const int lane = threadIdx.x & 31;
    const int per = nbins / 32;
    const uint32_t* mine_p = hist + lane * per;
    unsigned long long mine = 0;
    for (int k = 0; k < per; ++k) mine += mine_p[(k + lane) & (per - 1)];
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
    // inside lane L's range: the whole warp scans its `per` bins, `per / 32` per lane
    const unsigned long long start = __shfl_sync(0xffffffffu, base + incl - mine, L);
    const int sub = per / 32;  // bins per lane (per is a multiple of 32)
    const uint32_t* rng = hist + L * per + lane * sub;
    unsigned long long part = 0;
    for (int k = 0; k < sub; ++k) part += rng[k];
    unsigned long long inc2 = part;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, inc2, o);
        if (lane >= o) inc2 += v;
    }
    const unsigned int hit2 = __ballot_sync(0xffffffffu, start + inc2 >= target);
    const int L2 = __ffs(hit2) - 1;  // lane L's total reaches the target, so some lane does
    int bin = -1;
    unsigned long long cum = 0;
    if (lane == L2) {
        cum = start + inc2 - part;
        for (int k = 0; k < sub; ++k) {
            const unsigned long long h = rng[k];
            if (cum + h >= target) {
                bin = L * per + L2 * sub + k;
                break;
            }
            cum += h;
        }
    }
    bin = __shfl_sync(0xffffffffu, bin, L2);
    cum = __shfl_sync(0xffffffffu, cum, L2);
    if (bin >= 0) *below = cum;
    return bin;
}

// keysT[j][i] = float_key(beta[i][j]): the particles' values marker-major as
// order-preserving integer keys, so each summaries CTA streams its marker's column with
// coalesced loads. 32 x 32 tiles through shared memory. With WfS != NULL the weights (Wf,
// wfix) are copied beside them, so that the summaries read nothing the next step rewrites.
__global__ void k_keys_transpose(const float* __restrict__ beta, int64_t N, int p, uint32_t* __restrict__ keysT,
                                 const float* __restrict__ Wf, const uint32_t* __restrict__ wfix,
                                 float* __restrict__ WfS, uint32_t* __restrict__ wfixS)
{
    grid_dependency_wait();
    __shared__ uint32_t tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
    if (WfS && blockIdx.y == 0 && threadIdx.y == 0) {
        const int64_t i = i0 + threadIdx.x;
        if (i < N) {
            WfS[i] = Wf[i];
            wfixS[i] = wfix[i];
        }
    }
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r;
        const int j = j0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < N && j < p) ? float_key(beta[i * p + j]) : 0u;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r;
        const int64_t i = i0 + threadIdx.x;
        if (i < N && j < p) keysT[(int64_t)j * N + i] = tile[threadIdx.x][r];
    }
}

constexpr int SUM_SUB = 4;     // sub-histograms of the first radix digit (by warp % 4)
constexpr int SUM_BINS = 2048;  // bins of an 11-bit digit

// Per coordinate j (one CTA): the weighted mean and the concentrations (compensated FP32
// sums), and the weighted quantiles by an exact radix select on the fixed-point weights
// round(W 2^31) over the order-preserving integer keys of the values: digits of 11, 11 and
// 10 bits from the top. The first digit's histogram is built while the values are loaded,
// in SUM_SUB copies that are merged before the search (particles cluster in a few
// top-digit bins, and one copy per warp group spreads their atomics).
__global__ void __launch_bounds__(SUM_THREADS, 2) k_summaries(const uint32_t* __restrict__ keysT, const float* __restrict__ Wf,
                                                               const uint32_t* __restrict__ wfix, int64_t N, int p,
                                                               SummaryArgs sa, int t, double* __restrict__ mean,
                                                               double* __restrict__ quant, double* __restrict__ conc,
                                                               int staged)
{
    grid_dependency_wait();
    extern __shared__ uint32_t sm[];
    __shared__ float red_s[SUM_THREADS / 32][9], red_c[SUM_THREADS / 32][9];
    __shared__ unsigned long long shu[SUM_THREADS / 32];
    __shared__ uint32_t shk[SUM_THREADS / 32];
    __shared__ int bins[8][3];
    __shared__ unsigned long long below[8];
    const int j = blockIdx.x;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int nq = (quant && sa.nq > 0) ? sa.nq : 0, nd = sa.nd;
    uint32_t* keys = sm;
    uint32_t* wts = sm + (staged ? N : 0);
    uint32_t* hist = sm + (staged ? 2 * N : 0);  // max(SUM_SUB, nq) * SUM_BINS words
    if (nq > 0) {
        for (int e = tid; e < SUM_SUB * SUM_BINS; e += SUM_THREADS) hist[e] = 0u;
        if (tid < 8) below[tid] = 0ull;
        __syncthreads();
    }
    uint32_t* hsub = hist + (w & (SUM_SUB - 1)) * SUM_BINS;
    // ---- load: stage keys and weights; mean, concentrations, top-digit histogram
    FSum msum;
    FSum cs[8];
    uint32_t kmax = 0;
    unsigned long long tot = 0;
    const uint32_t* kcol = keysT + (int64_t)j * N;
    for (int64_t i = tid; i < N; i += SUM_THREADS) {
        const uint32_t k = kcol[i];
        const float b = key_float(k);
        const uint32_t wv = wfix[i];
        const float wf = Wf[i];
        if (staged) {
            keys[i] = k;
            wts[i] = wv;
        }
        msum.add(wf * b);
#pragma unroll
        for (int d = 0; d < 8; ++d)
            if (d < nd && fabsf(b) < sa.dthr[d]) cs[d].add(wf);
        kmax = k > kmax ? k : kmax;
        tot += wv;
        if (nq > 0 && wv != 0u) atomicAdd(&hsub[k >> 21], wv);
    }
    // ---- one block reduction for every scalar
    msum = warp_sum(msum);
#pragma unroll
    for (int d = 0; d < 8; ++d)
        if (d < nd) cs[d] = warp_sum(cs[d]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if (lane == 0) {
        red_s[w][0] = msum.s;
        red_c[w][0] = msum.c;
#pragma unroll
        for (int d = 0; d < 8; ++d)
            if (d < nd) {
                red_s[w][1 + d] = cs[d].s;
                red_c[w][1 + d] = cs[d].c;
            }
        shu[w] = tot;
        shk[w] = kmax;
    }
    __syncthreads();
    if (w == 0) {
        // lane v < 1 + nd finishes scalar v: the mean (v = 0) or concentration v - 1
        if (lane < 1 + nd) {
            FSum r;
            for (int k = 0; k < SUM_THREADS / 32; ++k) {
                r.add(red_s[k][lane]);
                r.c += red_c[k][lane];
            }
            const double val = (double)r.s + (double)r.c;
            if (lane == 0) {
                if (mean) mean[(int64_t)t * p + j] = val;
            } else if (conc) {
                conc[((int64_t)t * p + j) * nd + (lane - 1)] = 1.0 - val;
            }
        }
    }
    if (nq == 0) return;
    tot = 0;
    kmax = 0;
    for (int k = 0; k < SUM_THREADS / 32; ++k) {
        tot += shu[k];
        kmax = max(kmax, shk[k]);
    }
    // merge the top-digit copies into copy 0
    for (int b = tid; b < SUM_BINS; b += SUM_THREADS) {
        uint32_t v = hist[b];
#pragma unroll
        for (int s2 = 1; s2 < SUM_SUB; ++s2) v += hist[s2 * SUM_BINS + b];
        hist[b] = v;
    }
    __syncthreads();
    // ---- digit searches: the top digit on the merged histogram, then bits 10..20 and 0..9
    // of the keys that share the selected prefix, one histogram per quantile level
    for (int pass = 0; pass < 3; ++pass) {
        const int bits = (pass == 2) ? 10 : 11;
        const int shift = (pass == 0) ? 21 : ((pass == 1) ? 10 : 0);
        const int nb = 1 << bits;
        if (pass > 0) {
            uint32_t want[8];
            bool on[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                on[q] = q < nq && bins[q][0] >= 0;
                want[q] = on[q] ? ((pass == 1) ? (uint32_t)bins[q][0] : (((uint32_t)bins[q][0] << 11) | (uint32_t)bins[q][1]))
                                : 0u;
            }
            for (int e = tid; e < nq * nb; e += SUM_THREADS) hist[e] = 0u;
            __syncthreads();
            for (int64_t i = tid; i < N; i += SUM_THREADS) {
                const uint32_t k = staged ? keys[i] : kcol[i];
                const uint32_t wv = staged ? wts[i] : wfix[i];
                if (wv == 0u) continue;
                const uint32_t dig = (k >> shift) & (uint32_t)(nb - 1);
                const uint32_t pre = k >> (shift + bits);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (on[q] && pre == want[q]) atomicAdd(&hist[q * nb + dig], wv);
            }
            __syncthreads();
        }
        if (w < nq) {
            const int q = w;
            const unsigned long long target = sa.target[q];
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

// ------------------------------------------------ scale-marginalised summaries
// Section 4, eq. all_particles: with a uniform prior on log b over the log-spaced
// schedule, the particle systems of all steps mix with weights Z_t / Z_1, each the running
// product of the Z_t / Z_{t-1} estimates: w_t = exp(L_t - max L) / sum_s exp(L_s - max L),
// L_t = sum_{s=1..t} inc_s (the t = 0 evidence is common to every L_t). One thread, in
// step order (T is a few hundred).
__global__ void k_marginal_weights(const double* __restrict__ log_z_inc, int64_t T, double* __restrict__ post_c)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double acc = 0.0, m = -DBL_MAX;
    for (int64_t t = 0; t < T; ++t) {
        if (t > 0) acc += log_z_inc[t];
        post_c[t] = acc;
        m = fmax(m, acc);
    }
    double s = 0.0;
    for (int64_t t = 0; t < T; ++t) s += exp(post_c[t] - m);
    for (int64_t t = 0; t < T; ++t) post_c[t] = exp(post_c[t] - m) / s;
}

// Mixture of the per-step summaries: thread (j, v) sums w_t * mean[t][j] (v = 0) or
// w_t * conc[t][j][v - 1] over t in order.
__global__ void k_marginal_apply(const double* __restrict__ post_c, const double* __restrict__ mean,
                                 const double* __restrict__ conc, int64_t T, int64_t p, int D,
                                 double* __restrict__ mean_out, double* __restrict__ conc_out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p * (1 + D)) return;
    const int64_t j = e / (1 + D);
    const int v = (int)(e - j * (1 + D));
    double acc = 0.0;
    if (v == 0) {
        for (int64_t t = 0; t < T; ++t) acc += post_c[t] * mean[t * p + j];
        mean_out[j] = acc;
    } else {
        for (int64_t t = 0; t < T; ++t) acc += post_c[t] * conc[(t * p + j) * D + (v - 1)];
        conc_out[j * D + (v - 1)] = acc;
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
    const float inv_ac = (float)(1.0 / ((double)pr.a * c));
    out[i] = -log(2.0 * c) + prior_coef(pr, c) * (double)prior_term(beta[i], inv_ac, pr.de);
}

}  // namespace

// ======================================================================= launchers
// Launch configuration with programmatic stream serialization (programmatic dependent
// launch): the kernel may be scheduled while its predecessor drains and waits for it with
// grid_dependency_wait before reading anything the predecessor wrote.
static cudaLaunchConfig_t pdl_config(unsigned grid, unsigned block, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    return cfg;
}
static void pdl_attr(cudaLaunchConfig_t& cfg, cudaLaunchAttribute (&attr)[1])
{
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

// A launch with programmatic stream serialization: the kernels of the sweep's chain begin
// with grid_dependency_wait, so each may be scheduled while its predecessor drains.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

static unsigned warps_grid(int64_t N) { return (unsigned)((N + WARPS - 1) / WARPS); }
static unsigned elem_grid(int64_t total)
{
    int64_t b = (total + 255) / 256;
    if (b < 1) b = 1;
    return (unsigned)(b < 8192 ? b : 8192);
}

cudaError_t smc_init_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_summaries, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SUM_STAGED_MAX);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_move_site, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SITE_SMEM_MAX);
    return e;
}

cudaError_t launch_init_prior(float* beta, int64_t N, int p, PriorArgs pr, const double* sched, int t0,
                              const uint64_t* seed, cudaStream_t st)
{
    k_init_prior<<<elem_grid(N * p), 256, 0, st>>>(beta, N, p, pr, sched, t0, seed);
    return cudaGetLastError();
}

cudaError_t launch_step_constants(PriorArgs pr, const double* sched, int T, int p, float4* out, ReweightK* rk,
                                  cudaStream_t st)
{
    k_step_constants<<<(T + 127) / 128, 128, 0, st>>>(pr, sched, T, p, out, rk);
    return cudaGetLastError();
}

cudaError_t launch_move_rw(const MoveArgs& a, bool decide, int64_t N, int p, PriorArgs pr, const float4* stepk, int t,
                           uint32_t m, uint32_t m_prev, const uint64_t* seed, int noise, uint32_t* err, cudaStream_t st)
{
    const bool vec = (p & 3) == 0;
    const unsigned grid = warps_grid(N);
    if (decide) {  // follows the likelihood GEMM: programmatic dependent launch
        cudaLaunchConfig_t cfg = pdl_config(grid, BLOCK, st);
        cudaLaunchAttribute attr[1];
        pdl_attr(cfg, attr);
        if (vec)
            return cudaLaunchKernelEx(&cfg, k_move_rw<true, true>, a, N, p, pr, stepk, t, m, m_prev, seed, noise, err);
        return cudaLaunchKernelEx(&cfg, k_move_rw<true, false>, a, N, p, pr, stepk, t, m, m_prev, seed, noise, err);
    } else {
        if (vec)
            { const cudaError_t e_ = launch_pdl(k_move_rw<false, true>, dim3(grid), dim3(BLOCK), (size_t)(0), st, a, N, p, pr, stepk, t, m, m_prev, seed, noise, err); if (e_ != cudaSuccess) return e_; }
        else
            { const cudaError_t e_ = launch_pdl(k_move_rw<false, false>, dim3(grid), dim3(BLOCK), (size_t)(0), st, a, N, p, pr, stepk, t, m, m_prev, seed, noise, err); if (e_ != cudaSuccess) return e_; }
    }
    return cudaGetLastError();
}

cudaError_t launch_move_mala(const MoveArgs& a, bool decide, int64_t N, int p, PriorArgs pr, const float4* stepk, int t,
                             uint32_t m, uint32_t m_prev, const uint64_t* seed, uint32_t* err, cudaStream_t st)
{
    const bool vec = (p & 3) == 0;
    cudaLaunchConfig_t cfg = pdl_config(warps_grid(N), BLOCK, st);  // follows the gradient finish or the scales
    cudaLaunchAttribute attr[1];
    pdl_attr(cfg, attr);
    if (decide) {
        if (vec) return cudaLaunchKernelEx(&cfg, k_move_mala<true, true>, a, N, p, pr, stepk, t, m, m_prev, seed, err);
        return cudaLaunchKernelEx(&cfg, k_move_mala<true, false>, a, N, p, pr, stepk, t, m, m_prev, seed, err);
    }
    if (vec) return cudaLaunchKernelEx(&cfg, k_move_mala<false, true>, a, N, p, pr, stepk, t, m, m_prev, seed, err);
    return cudaLaunchKernelEx(&cfg, k_move_mala<false, false>, a, N, p, pr, stepk, t, m, m_prev, seed, err);
}

cudaError_t launch_move_commit(const MoveArgs& a, bool mala, int64_t N, int p, PriorArgs pr, const float4* stepk, int t,
                               uint32_t m_prev, const uint64_t* seed, uint32_t* err, cudaStream_t st)
{
    const bool vec = (p & 3) == 0;
    cudaLaunchConfig_t cfg = pdl_config(warps_grid(N), BLOCK, st);  // follows the likelihood GEMM
    cudaLaunchAttribute attr[1];
    pdl_attr(cfg, attr);
    if (mala) {
        if (vec) return cudaLaunchKernelEx(&cfg, k_move_commit<true, true>, a, N, p, pr, stepk, t, m_prev, seed, err);
        return cudaLaunchKernelEx(&cfg, k_move_commit<true, false>, a, N, p, pr, stepk, t, m_prev, seed, err);
    }
    if (vec) return cudaLaunchKernelEx(&cfg, k_move_commit<false, true>, a, N, p, pr, stepk, t, m_prev, seed, err);
    return cudaLaunchKernelEx(&cfg, k_move_commit<false, false>, a, N, p, pr, stepk, t, m_prev, seed, err);
}

int site_warps_per_block(int64_t n, int p)
{
    const int64_t per = (n + p) * (int64_t)sizeof(float);
    int64_t w = (int64_t)SITE_SMEM_MAX / (per > 0 ? per : 1);
    if (w > 8) w = 8;
    return (int)w;
}

cudaError_t launch_move_site(const SiteArgs& a, int64_t N, int p, int64_t n, PriorArgs pr, const float4* stepk, int t,
                             uint32_t m0, int M, const uint64_t* seed, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    const int wpc = site_warps_per_block(n, p);
    if (wpc < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)wpc * (size_t)(n + p) * sizeof(float);
    k_move_site<<<(unsigned)((N + wpc - 1) / wpc), 32 * wpc, smem, st>>>(a, N, p, (int)n, pr, stepk, t, m0, M, seed);
    return cudaGetLastError();
}

cudaError_t launch_finish_loglik(const MhState& s, int64_t N, double* logw, double* ll_out, uint32_t* err,
                                 cudaStream_t st)
{
    k_finish_loglik<<<warps_grid(N), BLOCK, 0, st>>>(s, N, logw, ll_out, err);
    return cudaGetLastError();
}

cudaError_t launch_reweight(const float* beta, double* logw, float2* lpq, int64_t N, int p, PriorArgs pr,
                            const ReweightK* rk, int t, uint32_t* err, cudaStream_t st)
{
    { const cudaError_t e_ = launch_pdl(k_reweight, dim3((unsigned)((N + RW_PER_BLOCK - 1) / RW_PER_BLOCK)), dim3(RW_THREADS), (size_t)(0), st, beta, logw, lpq, N, p, pr, rk,
                                                                                         t, err); if (e_ != cudaSuccess) return e_; }
    return cudaGetLastError();
}

cudaError_t launch_lse_ess(const WeightArrays& w, int64_t N, double* scratch, unsigned int* counter, int t, int mode,
                           double ess_frac, double* ess_out, double* logz_out, uint8_t* resampled_out, int* flag,
                           uint32_t* err, cudaStream_t st, bool pdl)
{
    int64_t blocks = (N + LSE_THREADS - 1) / LSE_THREADS;
    if (blocks > LSE_BLOCKS) blocks = LSE_BLOCKS;
    if (pdl) {
        const cudaError_t e_ = launch_pdl(k_lse_partial, dim3((unsigned)blocks), dim3(LSE_THREADS), (size_t)(0), st,
                                          w.logw, N, scratch, counter, t, mode, ess_frac, ess_out, logz_out,
                                          resampled_out, flag, err);
        if (e_ != cudaSuccess) return e_;
    } else {  // after a wait on another stream's event
        k_lse_partial<<<(unsigned)blocks, LSE_THREADS, 0, st>>>(w.logw, N, scratch, counter, t, mode, ess_frac, ess_out,
                                                               logz_out, resampled_out, flag, err);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one FP64 exp per weight: blocks of 64 spread them over the SMs' FP64 units
    const unsigned nb = (unsigned)std::min<int64_t>((N + 63) / 64, 8192);
    { const cudaError_t e_ = launch_pdl(k_normalise, dim3(nb), dim3(64), (size_t)(0), st, w, N, scratch + 3 * blocks); if (e_ != cudaSuccess) return e_; }
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
    const int64_t chunks = (N + RS_BLOCK - 1) / RS_BLOCK;
    const unsigned local_grid = (unsigned)((chunks + RS_CHUNKS - 1) / RS_CHUNKS);
    cudaError_t e = launch_pdl(k_resample_local, dim3(local_grid), dim3(RS_LOCAL_THREADS), RS_LOCAL_SMEM, st, W, N, cum,
                               flag);
    if (e == cudaSuccess)
        e = launch_pdl(k_resample_carry, dim3(1), dim3(RS_CARRY_THREADS), (size_t)0, st, N, cum, flag, t, seed,
                       u_override);
    if (e == cudaSuccess)
        e = launch_pdl(k_resample_search, dim3(elem_grid(N)), dim3(256), (size_t)0, st, cum, N, idx, flag);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_gather(const int32_t* idx, const float* beta, float* beta_tmp, const float2* llq, const float2* lpq,
                          float2* llq_tmp, float2* lpq_tmp, const float* g, float* g_tmp, int64_t N, int p,
                          const int* flag, cudaStream_t st)
{
    if ((p & 3) == 0)
        { const cudaError_t e_ = launch_pdl(k_gather<true>, dim3(warps_grid(N)), dim3(BLOCK), (size_t)(0), st, idx, beta, beta_tmp, llq, lpq, llq_tmp, lpq_tmp, g, g_tmp, N, p,
                                                        flag); if (e_ != cudaSuccess) return e_; }
    else
        { const cudaError_t e_ = launch_pdl(k_gather<false>, dim3(warps_grid(N)), dim3(BLOCK), (size_t)(0), st, idx, beta, beta_tmp, llq, lpq, llq_tmp, lpq_tmp, g, g_tmp, N, p,
                                                         flag); if (e_ != cudaSuccess) return e_; }
    return cudaGetLastError();
}

cudaError_t launch_copyback(float* beta, const float* beta_tmp, float2* llq, float2* lpq, const float2* llq_tmp,
                            const float2* lpq_tmp, float* g, const float* g_tmp, const WeightArrays& w, int64_t N, int p,
                            const int* flag, cudaStream_t st)
{
    // uniform weights after resampling: log(1/N), 1/N and round(2^31 / N), formed on the host
    const double wi = 1.0 / (double)N;
    const uint32_t wf = (uint32_t)std::llrint(wi * 2147483648.0);
    const double lw = -std::log((double)N);
    if ((p & 3) == 0)
        { const cudaError_t e_ = launch_pdl(k_copyback<true>, dim3(warps_grid(N)), dim3(BLOCK), (size_t)(0), st, beta, beta_tmp, llq, lpq, llq_tmp, lpq_tmp, g, g_tmp, w, N, p,
                                                          flag, lw, wi, wf); if (e_ != cudaSuccess) return e_; }
    else
        { const cudaError_t e_ = launch_pdl(k_copyback<false>, dim3(warps_grid(N)), dim3(BLOCK), (size_t)(0), st, beta, beta_tmp, llq, lpq, llq_tmp, lpq_tmp, g, g_tmp, w, N, p,
                                                           flag, lw, wi, wf); if (e_ != cudaSuccess) return e_; }
    return cudaGetLastError();
}

cudaError_t launch_colstats(const float* beta, const float* Wf, int64_t N, int p, float4* part, float* scale_out,
                            int kind, double lam_const, const double* lam_dev, double sd_floor, const double* sched,
                            int t, float* h_out, cudaStream_t st)
{
    dim3 block(32, CS_ROWS);
    dim3 grid((unsigned)((p + 31) / 32), COLSTAT_SPLITS);
    { const cudaError_t e_ = launch_pdl(k_colstats_partial, dim3(grid), dim3(block), (size_t)(0), st, beta, Wf, N, p, part); if (e_ != cudaSuccess) return e_; }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one warp (and block) per coordinate: its FP64 sums and square roots on their own SM
    { const cudaError_t e_ = launch_pdl(k_colstats_finish, dim3((unsigned)p), dim3(32), (size_t)(0), st, part, p, COLSTAT_SPLITS, scale_out, kind, lam_const,
                                                               lam_dev, sd_floor, sched, t, h_out,
                                                               std::pow((double)p, -1.0 / 6.0)); if (e_ != cudaSuccess) return e_; }
    return cudaGetLastError();
}

cudaError_t launch_keys(const float* beta, const float* Wf, const uint32_t* wfix, int64_t N, int p, uint32_t* keysT,
                        float* WfS, uint32_t* wfixS, bool pdl, cudaStream_t st)
{
    const dim3 grid((unsigned)((N + 31) / 32), (unsigned)((p + 31) / 32)), block(32, 8);
    if (pdl) return launch_pdl(k_keys_transpose, grid, block, (size_t)0, st, beta, N, p, keysT, Wf, wfix, WfS, wfixS);
    k_keys_transpose<<<grid, block, 0, st>>>(beta, N, p, keysT, Wf, wfix, WfS, wfixS);
    return cudaGetLastError();
}

cudaError_t launch_summaries_keys(const uint32_t* keysT, const float* Wf, const uint32_t* wfix, int64_t N, int p,
                                  const SummaryArgs& s, int t, double* mean, double* quant, double* conc, bool pdl,
                                  cudaStream_t st)
{
    SummaryArgs a = s;
    // host-side constants: the smallest float >= Delta (the open interval |b| < Delta tested
    // in FP32) and the fixed-point quantile targets ceil(q 2^31)
    for (int d = 0; d < 8; ++d) {
        float f = (float)a.delta[d];
        if ((double)f < a.delta[d]) f = std::nextafter(f, INFINITY);
        a.dthr[d] = f;
    }
    for (int q = 0; q < 8; ++q) a.target[q] = (unsigned long long)std::ceil(a.q[q] * 2147483648.0);
    const int nh = (quant && s.nq > 0) ? (s.nq > SUM_SUB ? s.nq : SUM_SUB) : 0;
    const size_t hist_bytes = (size_t)nh * SUM_BINS * sizeof(uint32_t);
    const size_t staged_bytes = (size_t)N * 2 * sizeof(uint32_t) + hist_bytes;
    const int staged = staged_bytes <= SUM_STAGED_MAX ? 1 : 0;
    const size_t bytes = staged ? staged_bytes : hist_bytes;
    if (pdl)
        return launch_pdl(k_summaries, dim3((unsigned)p), dim3(SUM_THREADS), bytes, st, keysT, Wf, wfix, N, p, a, t, mean,
                          quant, conc, staged);
    k_summaries<<<(unsigned)p, SUM_THREADS, bytes, st>>>(keysT, Wf, wfix, N, p, a, t, mean, quant, conc, staged);
    return cudaGetLastError();
}

cudaError_t launch_summaries(const float* beta, const float* Wf, const uint32_t* wfix, int64_t N, int p,
                             const SummaryArgs& s, int t, double* mean, double* quant, double* conc, uint32_t* keysT,
                             cudaStream_t st)
{
    const cudaError_t e = launch_keys(beta, Wf, wfix, N, p, keysT, nullptr, nullptr, true, st);
    if (e != cudaSuccess) return e;
    return launch_summaries_keys(keysT, Wf, wfix, N, p, s, t, mean, quant, conc, true, st);
}

cudaError_t launch_marginal(const double* log_z_inc, const double* mean, const double* conc, int64_t T, int64_t p,
                            int D, double* post_c, double* mean_out, double* conc_out, cudaStream_t st)
{
    k_marginal_weights<<<1, 32, 0, st>>>(log_z_inc, T, post_c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t work = p * (1 + D);
    k_marginal_apply<<<(unsigned)((work + 127) / 128), 128, 0, st>>>(post_c, mean, conc, T, p, D, mean_out, conc_out);
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
