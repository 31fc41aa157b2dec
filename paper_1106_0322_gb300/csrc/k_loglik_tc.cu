// k_loglik_tc.cu -- the particle log-likelihood on the 5th-generation tensor cores.
//
// Section 2's log-likelihood of particle k is l_k = sum_i [y_i eta_ki - softplus(eta_ki)],
// eta = X beta_k. This kernel computes it for N particles at once as a contraction
// followed by a row reduction that never leaves the chip:
//
//   eta2[k, i] = sum_j A[k, j] * Gb[i, j]      (tcgen05.mma, BF16 x BF16 -> FP32 in TMEM)
//   partial[k] += sum_i y_i eta2 - log2(1 + 2^eta2[k, i])  (epilogue warps, ex2/lg2 on the SFU)
//
// with A[k] = [hi(bt_k) | lo(bt_k)] the split-BF16 copy of bt_kj = beta_kj log2(e)/s_j
// (plus the offset -sum_j m_j bt_kj in the ones column), and Gb = [G, 1] the exact BF16
// genotypes. Both halves of A multiply the same G tile, so each pipeline stage carries
// A_hi, A_lo and G for one 64-wide k-block; eta2 = eta log2(e), so l = ln(2) * sum of
// [y eta2 - log2(1 + 2^eta2)]. y is read as a bitmask, one 32-bit word per 32 individuals.
//
// Tile: 128 particles (M, TMEM lanes) x BN individuals (N, TMEM columns). A persistent
// grid walks the (particle-tile, individual-tile) units in order; each unit's row sums go
// to their own slot of `partial`, so the final sum (in the accept kernel) has a fixed
// order. Warp roles: warp 0 issues TMA loads, warp 1 (one thread) issues the MMAs and owns
// TMEM, warps 2..9 drain the double-buffered accumulator (warp w reads TMEM lanes
// 32 (w % 4) .. +31, half (w - 2) / 4 of the columns). Every wait is bounded.
#include "spa_device.cuh"
#include "spa_internal.h"

namespace spa {

namespace {

constexpr int BM = 128;
constexpr int BK = 64;  // BF16 per 128-byte swizzle row
constexpr int EPI_WARPS = 8;
constexpr int TC_THREADS = 64 + 32 * EPI_WARPS;
constexpr int ADJ_BN_SMALL = 208;  // p + padding <= 208 covers the p = 200 workloads in one N tile

template <int BN, int STAGES>
struct TcCfg {
    static constexpr int A_TILE = BM * BK * 2;
    static constexpr int B_TILE = BN * BK * 2;
    static constexpr int STAGE = 2 * A_TILE + B_TILE;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int NBARS = 2 * STAGES + 5;  // full[S], empty[S], acc_full[2], acc_empty[2], drain
    static constexpr int SLOT_OFF = BAR_OFF + NBARS * 8;
    static constexpr int BYTES = SLOT_OFF + 16;
    static constexpr int SMEM = BYTES + 1024;  // slack for the 1024-byte alignment of the tiles
    static constexpr uint32_t TMEM_COLS = 2 * BN;
    static_assert(STAGE % 1024 == 0, "tiles must stay 1024-byte aligned");
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(TMEM_COLS == 256 || TMEM_COLS == 512, "TMEM allocation must be a power of two");
};

// Sum over 32 columns of the base-2 log-likelihood terms y eta2 - log2(1 + 2^eta2); bit k of
// ybits is y of column k.
__device__ __forceinline__ float sum_ll2_32(const float (&v)[32], int valid, uint32_t ybits)
{
    float t[32];
    if (valid >= 32) {
#pragma unroll
        for (int k = 0; k < 32; ++k) t[k] = (((ybits >> k) & 1u) ? v[k] : 0.0f) - softplus2(v[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) t[k] = (k < valid) ? (((ybits >> k) & 1u) ? v[k] : 0.0f) - softplus2(v[k]) : 0.0f;
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)
#pragma unroll
        for (int k = 0; k < w; ++k) t[k] += t[k + w];
    return t[0];
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Residual mode: besides the log-likelihood sum, r = y - logit^{-1}(eta) for the 32 columns
// of this chunk is stored as BF16 hi (row of R) and lo (row + n_r) and summed into *rsum.
// eta2 = eta log2(e): with e = 2^-|eta2|, softplus2 = max(eta2, 0) + log2(1 + e) and
// logit^{-1}(eta) = 1/(1 + e) for eta >= 0, e/(1 + e) otherwise (one ex2 shared).
__device__ __forceinline__ float resid_chunk(const float (&v)[32], int valid, uint32_t ybits,
                                             __nv_bfloat16* __restrict__ rrow, int64_t n_r, float& rsum)
{
    float sp[32];
    __align__(16) __nv_bfloat16 hi[32];
    __align__(16) __nv_bfloat16 lo[32];
    float rs[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float x = v[k];
        const float e = ex2_approx(-fabsf(x));
        const float onepe = 1.0f + e;
        const float inv = rcp_approx(onepe);
        const float sig = (x >= 0.0f) ? inv : e * inv;
        const bool ok = k < valid;
        const bool yk = (ybits >> k) & 1u;
        sp[k] = ok ? (yk ? x : 0.0f) - (fmaxf(x, 0.0f) + lg2_approx(onepe)) : 0.0f;
        const float r = ok ? (yk ? 1.0f : 0.0f) - sig : 0.0f;
        rs[k] = r;
        split_bf16(r, hi[k], lo[k]);
    }
    // 16-byte stores of the 32 hi and 32 lo values (rrow is 64-byte aligned)
    uint4* dh = reinterpret_cast<uint4*>(rrow);
    uint4* dl = reinterpret_cast<uint4*>(rrow + n_r);
    const uint4* sh = reinterpret_cast<const uint4*>(hi);
    const uint4* sl = reinterpret_cast<const uint4*>(lo);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        dh[q] = sh[q];
        dl[q] = sl[q];
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)
#pragma unroll
        for (int k = 0; k < w; ++k) {
            sp[k] += sp[k + w];
            rs[k] += rs[k + w];
        }
    rsum += rs[0];
    return sp[0];
}

template <int BN, int STAGES, bool RESID>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_loglik_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int n_tiles,
                int m_tiles, int kblocks, int ksteps, int Kp, int n, float* __restrict__ partial, int64_t N_pad,
                uint32_t* __restrict__ err, const uint32_t* __restrict__ ybits, __nv_bfloat16* __restrict__ R,
                int64_t n_r, float* __restrict__ rsum_part)
{
    using C = TcCfg<BN, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = sbase + C::BAR_OFF;
    const uint32_t drain_bar = bar0 + 8 * (2 * STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::SLOT_OFF);
#define FULL_BAR(s) (bar0 + 8u * (uint32_t)(s))
#define EMPTY_BAR(s) (bar0 + 8u * (uint32_t)(STAGES + (s)))
#define ACCF_BAR(b) (bar0 + 8u * (uint32_t)(2 * STAGES + (b)))
#define ACCE_BAR(b) (bar0 + 8u * (uint32_t)(2 * STAGES + 2 + (b)))

    const int64_t U = (int64_t)m_tiles * n_tiles;
    const int64_t u_begin = U * blockIdx.x / gridDim.x;
    const int64_t u_end = U * (blockIdx.x + 1) / gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(FULL_BAR(s), 1);
            mbar_init(EMPTY_BAR(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(ACCF_BAR(b), 1);
            mbar_init(ACCE_BAR(b), EPI_WARPS);
        }
        mbar_init(drain_bar, 1);
        mbar_fence_init();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int64_t u = u_begin; u < u_end && ok; ++u) {
                const int mt = (int)(u / n_tiles), nt = (int)(u % n_tiles);
                for (int kb = 0; kb < kblocks; ++kb) {
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded(EMPTY_BAR(s), ph ^ 1u, err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + s * C::STAGE;
                    mbar_arrive_expect_tx(FULL_BAR(s), (uint32_t)C::STAGE);
                    tma_load_2d(st, &mapA, FULL_BAR(s), kb * BK, mt * BM);
                    tma_load_2d(st + C::A_TILE, &mapA, FULL_BAR(s), Kp + kb * BK, mt * BM);
                    tma_load_2d(st + 2 * C::A_TILE, &mapB, FULL_BAR(s), kb * BK, nt * BN);
                    ++it;
                }
            }
            // Never leave with a copy in flight: the most recent use of each stage must have landed.
            const uint32_t last = it < (uint32_t)STAGES ? it : (uint32_t)STAGES;
            for (uint32_t k = 1; k <= last; ++k) {
                const uint32_t i2 = it - k;
                mbar_wait_bounded(FULL_BAR(i2 % STAGES), (i2 / STAGES) & 1u, err, 100000000ull);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16_f32(BM, BN);
            uint32_t it = 0;
            int lt = 0;
            bool ok = true;
            for (int64_t u = u_begin; u < u_end && ok; ++u, ++lt) {
                const uint32_t b = (uint32_t)(lt & 1), aph = (uint32_t)((lt >> 1) & 1);
                if (!mbar_wait_bounded(ACCE_BAR(b), aph ^ 1u, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + b * (uint32_t)BN;
                for (int kb = 0; kb < kblocks; ++kb) {
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded(FULL_BAR(s), ph, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * C::STAGE;
                    const uint64_t ahi = sdesc_sw128(st);
                    const uint64_t alo = sdesc_sw128(st + C::A_TILE);
                    const uint64_t bg = sdesc_sw128(st + 2 * C::A_TILE);
                    const int nks = (ksteps - 4 * kb) < 4 ? (ksteps - 4 * kb) : 4;
                    for (int ks = 0; ks < nks; ++ks)  // +32 bytes per K = 16 step inside the swizzle row
                        umma_bf16(d, ahi + 2u * ks, bg + 2u * ks, IDESC, (kb | ks) != 0 ? 1u : 0u);
                    for (int ks = 0; ks < nks; ++ks) umma_bf16(d, alo + 2u * ks, bg + 2u * ks, IDESC, 1u);
                    umma_commit(EMPTY_BAR(s));
                    ++it;
                }
                if (!ok) break;
                umma_commit(ACCF_BAR(b));
            }
            // Wait for every MMA this thread issued before TMEM can be released.
            umma_commit(drain_bar);
            mbar_wait_bounded(drain_bar, 0u, err, 100000000ull);
        }
    } else {
        // --------------------------------------------------------------- epilogue
        const int quad = warp & 3;         // TMEM lane quadrant this warp may access
        const int half = (warp - 2) >> 2;  // which half of the BN columns
        const int row = quad * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        int lt = 0;
        for (int64_t u = u_begin; u < u_end; ++u, ++lt) {
            const int mt = (int)(u / n_tiles), nt = (int)(u % n_tiles);
            const uint32_t b = (uint32_t)(lt & 1), aph = (uint32_t)((lt >> 1) & 1);
            if (!mbar_wait_bounded(ACCF_BAR(b), aph, err)) break;
            tc_fence_after();
            const int col0 = half * (BN / 2);
            const int valid = n - nt * BN - col0;
            float acc = 0.0f, rsum = 0.0f;
            // software pipeline over the 32-column chunks: the TMEM load of chunk k+1 is in
            // flight while chunk k is reduced
            constexpr int NCH = (BN / 2) / 32;
            const uint32_t tbase = tmem_base + lane_addr + b * (uint32_t)BN + (uint32_t)col0;
            uint32_t ra[32], rb[32];
            if (valid > 0) {
                tmem_ld32_async(tbase, ra);
                tmem_wait_ld(ra);
            }
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) {
                const int c = ch * 32;
                if (valid - c <= 0) break;
                uint32_t(&cur)[32] = (ch & 1) ? rb : ra;
                uint32_t(&nxt)[32] = (ch & 1) ? ra : rb;
                const bool more = (ch + 1 < NCH) && (valid - c - 32 > 0);
                if (more) tmem_ld32_async(tbase + (uint32_t)(c + 32), nxt);
                float v[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(cur[k]);
                const int64_t i0 = (int64_t)nt * BN + col0 + c;
                const uint32_t yb = __ldg(ybits + (i0 >> 5));
                if (RESID) {
                    acc += resid_chunk(v, valid - c, yb, R + ((int64_t)mt * BM + row) * 2 * n_r + i0, n_r, rsum);
                } else {
                    acc += sum_ll2_32(v, valid - c, yb);
                }
                if (more) tmem_wait_ld(nxt);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(ACCE_BAR(b));
            partial[((int64_t)nt * 2 + half) * N_pad + (int64_t)mt * BM + row] = acc;
            if (RESID) rsum_part[((int64_t)nt * 2 + half) * N_pad + (int64_t)mt * BM + row] = rsum;
        }
    }
#undef FULL_BAR
#undef EMPTY_BAR
#undef ACCF_BAR
#undef ACCE_BAR
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

// ----------------------------------------------------------------------- adjoint
// C[k, j] = sum_i r_ki g_ij for 128 particles x BN2 markers, contracting over the
// individuals of this CTA's k-range: A = [R_hi | R_lo] (N_pad x 2 n_r), B = G^T
// (markers x n_r, exact BF16), both K-major with the 128-byte swizzle. One output tile per
// CTA; warps 2..5 copy the FP32 accumulator to gpart[ks][particle][marker]. The final
// gradient (C - m_j sum_i r_ki) / s_j is formed by k_grad_finish.
constexpr int ADJ_THREADS = 64 + 32 * 4;

template <int BN2, int STAGES>
struct AdjCfg {
    static constexpr int A_TILE = BM * BK * 2;
    static constexpr int B_TILE = BN2 * BK * 2;
    static constexpr int STAGE = 2 * A_TILE + B_TILE;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int NBARS = 2 * STAGES + 2;  // full, empty, acc_full, drain
    static constexpr int SLOT_OFF = BAR_OFF + NBARS * 8;
    static constexpr int SMEM = SLOT_OFF + 16 + 1024;
    static constexpr uint32_t TMEM_COLS = 256;
    static_assert(STAGE % 1024 == 0, "tiles must stay 1024-byte aligned");
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(BN2 % 16 == 0 && BN2 <= 256, "MMA N");
};

template <int BN2, int STAGES>
__global__ void __launch_bounds__(ADJ_THREADS, 1)
    k_adjoint_tc(const __grid_constant__ CUtensorMap mapR, const __grid_constant__ CUtensorMap mapGT, int m_tiles,
                 int p_tiles, int kblocks, int ksplit, int n_r, int p, float* __restrict__ gpart, int64_t N_pad,
                 uint32_t* __restrict__ err)
{
    using C = AdjCfg<BN2, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = sbase + C::BAR_OFF;
    const uint32_t accf_bar = bar0 + 8u * (uint32_t)(2 * STAGES);
    const uint32_t drain_bar = accf_bar + 8u;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::SLOT_OFF);
#define FULL_BAR(s) (bar0 + 8u * (uint32_t)(s))
#define EMPTY_BAR(s) (bar0 + 8u * (uint32_t)(STAGES + (s)))
    // unit = (mt, pt, ks)
    const int u = blockIdx.x;
    const int ks = u % ksplit;
    const int pt = (u / ksplit) % p_tiles;
    const int mt = u / (ksplit * p_tiles);
    const int kb0 = (int)((int64_t)kblocks * ks / ksplit), kb1 = (int)((int64_t)kblocks * (ks + 1) / ksplit);

    if (threadIdx.x == 0) {
        for (int q = 0; q < STAGES; ++q) {
            mbar_init(FULL_BAR(q), 1);
            mbar_init(EMPTY_BAR(q), 1);
        }
        mbar_init(accf_bar, 1);
        mbar_init(drain_bar, 1);
        mbar_fence_init();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&mapR);
        tma_prefetch_desc(&mapGT);
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int kb = kb0; kb < kb1; ++kb) {
                const uint32_t q = it % STAGES, ph = (it / STAGES) & 1u;
                if (!mbar_wait_bounded(EMPTY_BAR(q), ph ^ 1u, err)) break;
                const uint32_t st = sbase + q * C::STAGE;
                mbar_arrive_expect_tx(FULL_BAR(q), (uint32_t)C::STAGE);
                tma_load_2d(st, &mapR, FULL_BAR(q), kb * BK, mt * BM);
                tma_load_2d(st + C::A_TILE, &mapR, FULL_BAR(q), n_r + kb * BK, mt * BM);
                tma_load_2d(st + 2 * C::A_TILE, &mapGT, FULL_BAR(q), kb * BK, pt * BN2);
                ++it;
            }
            const uint32_t last = it < (uint32_t)STAGES ? it : (uint32_t)STAGES;
            for (uint32_t k = 1; k <= last; ++k) {
                const uint32_t i2 = it - k;
                mbar_wait_bounded(FULL_BAR(i2 % STAGES), (i2 / STAGES) & 1u, err, 100000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16_f32(BM, BN2);
            uint32_t it = 0;
            bool ok = true;
            for (int kb = kb0; kb < kb1; ++kb) {
                const uint32_t q = it % STAGES, ph = (it / STAGES) & 1u;
                if (!mbar_wait_bounded(FULL_BAR(q), ph, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t st = sbase + q * C::STAGE;
                const uint64_t ahi = sdesc_sw128(st), alo = sdesc_sw128(st + C::A_TILE);
                const uint64_t bg = sdesc_sw128(st + 2 * C::A_TILE);
#pragma unroll
                for (int k = 0; k < 4; ++k) umma_bf16(tmem_base, ahi + 2u * k, bg + 2u * k, IDESC, (kb > kb0 || k) ? 1u : 0u);
#pragma unroll
                for (int k = 0; k < 4; ++k) umma_bf16(tmem_base, alo + 2u * k, bg + 2u * k, IDESC, 1u);
                umma_commit(EMPTY_BAR(q));
                ++it;
            }
            if (ok) umma_commit(accf_bar);
            umma_commit(drain_bar);
            mbar_wait_bounded(drain_bar, 0u, err, 100000000ull);
        }
    } else {
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const int cols = (p - pt * BN2) < BN2 ? (p - pt * BN2) : BN2;
        if (kb1 > kb0 && mbar_wait_bounded(accf_bar, 0u, err)) {
            tc_fence_after();
            float* out = gpart + ((int64_t)ks * N_pad + (int64_t)mt * BM + row) * p + (int64_t)pt * BN2;
#pragma unroll 1
            for (int c = 0; c < cols; c += 32) {
                float v[32];
                tmem_ld32(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)c, v);
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (c + k < cols) out[c + k] = v[k];
            }
        } else if (kb1 <= kb0) {
            float* out = gpart + ((int64_t)ks * N_pad + (int64_t)mt * BM + row) * p + (int64_t)pt * BN2;
            for (int c = 0; c < cols; ++c) out[c] = 0.0f;
        }
    }
#undef FULL_BAR
#undef EMPTY_BAR
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

// grad l_kj = (sum_s C_s[k, j] - m_j sum_i r_ki) / s_j (+ the prior gradient at scale c > 0).
__global__ void k_grad_finish(const float* __restrict__ gpart, int ksplit, const float* __restrict__ rsum_part,
                              int n_parts, int64_t N_pad, int64_t N, int p, const double* __restrict__ mean,
                              const double* __restrict__ sd, const float* __restrict__ B, PriorArgs pr, double c,
                              float* __restrict__ grad)
{
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    double rs = 0.0;
    for (int q = lane; q < n_parts; q += 32) rs += (double)rsum_part[(int64_t)q * N_pad + k];
    rs = warp_sum(rs);
    for (int j = lane; j < p; j += 32) {
        double g = 0.0;
        for (int q = 0; q < ksplit; ++q) g += (double)gpart[((int64_t)q * N_pad + k) * p + j];
        g = (g - mean[j] * rs) / sd[j];
        if (c > 0.0) {
            const float b = B[k * p + j];
            const double sg = (b > 0.0f) ? 1.0 : ((b < 0.0f) ? -1.0 : 0.0);
            g += pr.de ? -sg / c : -((double)pr.a + 1.0) * sg / ((double)pr.a * c + fabs((double)b));
        }
        grad[k * p + j] = (float)g;
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool make_map_2d(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                 uint32_t box_outer)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int STAGES, bool RESID>
cudaError_t launch_tc(const CUtensorMap& mapA, const CUtensorMap& mapB, const TcPlan& plan, int64_t n, int Kp,
                      const uint32_t* ybits, float* partial, int64_t N_pad, uint32_t* err, const ResidArgs* ra,
                      cudaStream_t st)
{
    using C = TcCfg<BN, STAGES>;
    k_loglik_tc<BN, STAGES, RESID><<<plan.grid, TC_THREADS, C::SMEM, st>>>(
        mapA, mapB, plan.n_tiles, plan.m_tiles, plan.kblocks, plan.ksteps, Kp, (int)n, partial, N_pad, err, ybits,
        ra ? ra->R : nullptr, ra ? ra->n_r : 0, ra ? ra->rsum_part : nullptr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t tc_init_attributes()
{
    cudaError_t e = cudaSuccess;
#define SET_SMEM(kern, bytes) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
    SET_SMEM((k_loglik_tc<256, 3, false>), (TcCfg<256, 3>::SMEM));
    SET_SMEM((k_loglik_tc<128, 4, false>), (TcCfg<128, 4>::SMEM));
    SET_SMEM((k_loglik_tc<256, 3, true>), (TcCfg<256, 3>::SMEM));
    SET_SMEM((k_loglik_tc<128, 4, true>), (TcCfg<128, 4>::SMEM));
    SET_SMEM((k_adjoint_tc<ADJ_BN_SMALL, 3>), (AdjCfg<ADJ_BN_SMALL, 3>::SMEM));
    SET_SMEM((k_adjoint_tc<256, 3>), (AdjCfg<256, 3>::SMEM));
#undef SET_SMEM
    return e;
}

TcPlan tc_plan(int64_t n, int p, int64_t N_pad, int num_sms)
{
    TcPlan pl;
    pl.BN = (n <= 128) ? 128 : 256;
    pl.n_tiles = (int)((n + pl.BN - 1) / pl.BN);
    pl.m_tiles = (int)(N_pad / BM);
    pl.ksteps = (p + 1 + 15) / 16;
    pl.kblocks = (pl.ksteps + 3) / 4;
    const int64_t units = (int64_t)pl.m_tiles * pl.n_tiles;
    pl.grid = (int)(units < num_sms ? units : num_sms);
    pl.n_parts = 2 * pl.n_tiles;
    return pl;
}

bool tc_make_map_A(CUtensorMap* map, const __nv_bfloat16* A, int64_t N_pad, int Kp)
{
    return make_map_2d(map, A, (uint64_t)(2 * Kp), (uint64_t)N_pad, BK, BM);
}

bool tc_make_map_B(CUtensorMap* map, const __nv_bfloat16* Gbf, int64_t n, int Kp, int BN)
{
    return make_map_2d(map, Gbf, (uint64_t)Kp, (uint64_t)n, BK, (uint32_t)BN);
}

cudaError_t launch_loglik_tc(const CUtensorMap& mapA, const CUtensorMap& mapB, const TcPlan& plan, int64_t n, int Kp,
                             const uint32_t* ybits, float* partial, int64_t N_pad, uint32_t* err, cudaStream_t st,
                             const ResidArgs* ra)
{
    if (ra) {
        if (plan.BN == 256) return launch_tc<256, 3, true>(mapA, mapB, plan, n, Kp, ybits, partial, N_pad, err, ra, st);
        return launch_tc<128, 4, true>(mapA, mapB, plan, n, Kp, ybits, partial, N_pad, err, ra, st);
    }
    if (plan.BN == 256) return launch_tc<256, 3, false>(mapA, mapB, plan, n, Kp, ybits, partial, N_pad, err, nullptr, st);
    return launch_tc<128, 4, false>(mapA, mapB, plan, n, Kp, ybits, partial, N_pad, err, nullptr, st);
}

AdjPlan adj_plan(int p, int64_t n, int64_t N_pad, int num_sms)
{
    AdjPlan a;
    a.n_r = (n + 63) / 64 * 64;
    a.kblocks = (int)(a.n_r / 64);
    a.BN2 = (p <= ADJ_BN_SMALL) ? ADJ_BN_SMALL : 256;
    a.p_tiles = (p + a.BN2 - 1) / a.BN2;
    a.m_tiles = (int)(N_pad / BM);
    const int base = a.m_tiles * a.p_tiles;
    int ks = num_sms / (base > 0 ? base : 1);
    if (ks < 1) ks = 1;
    if (ks > a.kblocks) ks = a.kblocks;
    if (ks > 8) ks = 8;
    a.ksplit = ks;
    a.grid = base * ks;
    return a;
}

bool adj_make_map_R(CUtensorMap* map, const __nv_bfloat16* R, int64_t N_pad, int64_t n_r)
{
    return make_map_2d(map, R, (uint64_t)(2 * n_r), (uint64_t)N_pad, BK, BM);
}

bool adj_make_map_GT(CUtensorMap* map, const __nv_bfloat16* GT, int p, int64_t n_r, int BN2)
{
    return make_map_2d(map, GT, (uint64_t)n_r, (uint64_t)p, BK, (uint32_t)BN2);
}

cudaError_t launch_adjoint_tc(const CUtensorMap& mapR, const CUtensorMap& mapGT, const AdjPlan& a, int p,
                              float* gpart, int64_t N_pad, uint32_t* err, cudaStream_t st)
{
    if (a.BN2 == ADJ_BN_SMALL) {
        k_adjoint_tc<ADJ_BN_SMALL, 3><<<a.grid, ADJ_THREADS, AdjCfg<ADJ_BN_SMALL, 3>::SMEM, st>>>(
            mapR, mapGT, a.m_tiles, a.p_tiles, a.kblocks, a.ksplit, (int)a.n_r, p, gpart, N_pad, err);
    } else {
        k_adjoint_tc<256, 3><<<a.grid, ADJ_THREADS, AdjCfg<256, 3>::SMEM, st>>>(mapR, mapGT, a.m_tiles, a.p_tiles,
                                                                               a.kblocks, a.ksplit, (int)a.n_r, p, gpart,
                                                                               N_pad, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_finish(const float* gpart, int ksplit, const float* rsum_part, int n_parts, int64_t N_pad,
                               int64_t N, int p, const double* mean, const double* sd, const float* B, PriorArgs pr,
                               double c, float* grad, cudaStream_t st)
{
    k_grad_finish<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(gpart, ksplit, rsum_part, n_parts, N_pad, N, p, mean, sd, B,
                                                           pr, c, grad);
    return cudaGetLastError();
}

}  // namespace spa
