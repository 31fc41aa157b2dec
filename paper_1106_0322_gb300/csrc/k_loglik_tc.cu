// k_loglik_tc.cu -- the particle log-likelihood on the 5th-generation tensor cores.
//
// Section 2's log-likelihood of particle k is l_k = sum_i [y_i eta_ki - softplus(eta_ki)],
// eta = X beta_k. Its first half is linear in beta: sum_i y_i eta_ki = beta_k . (X^T y), a
// p-length dot product that the move kernels form per particle. This kernel computes the
// n-length second half for N particles at once as a contraction followed by a row
// reduction that never leaves the chip:
//
//   eta2[k, i] = sum_j A[k, j] * Gb[i, j]       (tcgen05.mma, BF16 x BF16 -> FP32 in TMEM)
//   partial[c][k] = -sum_{i in chunk c} log2(1 + 2^eta2[k, i])   (epilogue warps, ex2/lg2)
//
// with A[k] = [hi(bt_k) | lo(bt_k)] the split-BF16 copy of bt_kj = beta_kj log2(e)/s_j
// (plus the offset -sum_j m_j bt_kj in the ones column), and Gb = [G, 1] the exact BF16
// genotypes. Both halves of A multiply the same G tile, so each pipeline stage carries
// A_hi, A_lo and G for one 64-wide k-block; eta2 = eta log2(e), so the softplus half of l
// is ln(2) * sum_c partial[c]. One partial per 32-individual chunk c: the chunk sums do not
// depend on the tile shape, so the result is the same for every BN the tuner picks.
//
// Tile: 128 particles (M, TMEM lanes) x BN individuals (N, TMEM columns). A persistent
// grid walks the (particle-tile, individual-tile) units in order, one range per CTA. Warp roles: warp 0
// issues TMA loads, warp 1 (one thread) issues the MMAs and owns TMEM, the epilogue warps
// drain the double-buffered accumulator (warp w reads TMEM lanes 32 (w % 4) .. +31 and
// one of EPI/4 column groups). Every wait is bounded.
#include "spa_device.cuh"
#include "spa_internal.h"

namespace spa {

namespace {

constexpr int BM = 128;
constexpr int BK = 64;  // BF16 per 128-byte swizzle row
// epilogue warps EW: 16 or 8 for the log-likelihood (the tile configuration's choice; 4 per
// TMEM lane quadrant hide the SFU and TMEM latencies best on most shapes), 8 for the residual
// variant, whose per-chunk state is larger
template <int EW>
struct Epi {
    static constexpr int WARPS = EW;
    static constexpr int THREADS = 64 + 32 * WARPS;
    static constexpr int GROUPS = WARPS / 4;  // column groups per tile
};
constexpr int ADJ_BN_SMALL = 208;  // p + padding <= 208 covers the p = 200 workloads in one N tile

// Shared-memory and TMEM plan, by the particle operand's residence AR:
//   0 streaming: every stage carries A_hi, A_lo and the G tile of one k-block;
//   1 resident in shared memory (K <= 256): the particle tile's A_hi | A_lo for all k-blocks
//     stays there while the CTA walks consecutive n-tiles of the same particle tile, and the
//     stages carry only G, halving what each SM pulls from L2;
//   2 resident in tensor memory (K <= 256): the epilogue warps copy the particle tile's rows
//     into TMEM columns beside the accumulators and the MMAs read A from there, so that shared
//     memory holds only G stages -- twice as many, which is what hides the G loads' latency.
//     With BN = 256 the accumulator is single-buffered (256 + 256 columns): the epilogue moves
//     it to registers and hands it back before doing its arithmetic.
constexpr int KB_RES = 4;  // k-blocks of a resident A (Kp <= 256)

template <int BN, int STAGES, int AR = 0>
struct TcCfg {
    static constexpr int A_TILE = BM * BK * 2;
    static constexpr int B_TILE = BN * BK * 2;
    // A compact resident A (BN = 224, whose four G stages fill the rest of shared memory):
    // three full k-blocks, then a last k-block at most 32 columns wide (A_hi, then A_lo
    // 8 KB on). Only shapes whose fourth k-block is narrow (or absent) take it.
    static constexpr bool COMPACT = AR == 1 && BN == 224;
    static constexpr int TAIL_LO = COMPACT ? BM * 32 * 2 : A_TILE;  // A_lo's offset in the last k-block
    static constexpr int A_RES = AR == 1 ? (COMPACT ? 3 * 2 * A_TILE + 2 * TAIL_LO : KB_RES * 2 * A_TILE) : 0;
    static constexpr int STAGE = AR ? B_TILE : 2 * A_TILE + B_TILE;
    // accumulator buffers, and the TMEM column of A (AR = 2): A_hi in 8 columns per K = 16
    // step (two BF16 per 32-bit column), then A_lo
    static constexpr int NACC = (AR == 2 && BN == 256) ? 1 : 2;
    static constexpr uint32_t A_COL = (uint32_t)(NACC * BN);
    static constexpr int BAR_OFF = A_RES + STAGES * STAGE;
    // full[S], empty[S], acc_full[2], acc_empty[2], drain, a_empty, a_full[KB_RES]
    static constexpr int NBARS = 2 * STAGES + 6 + KB_RES;
    static constexpr int SLOT_OFF = BAR_OFF + NBARS * 8;
    static constexpr int BYTES = SLOT_OFF + 16;
    static constexpr int SMEM = BYTES + 1024;  // slack for the 1024-byte alignment of the tiles
    static constexpr uint32_t TMEM_COLS = (AR == 2 || 2 * BN > 256) ? 512u : 256u;
    static_assert(STAGE % 1024 == 0, "tiles must stay 1024-byte aligned");
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(TMEM_COLS == 256 || TMEM_COLS == 512, "TMEM allocation must be a power of two");
    static_assert(AR != 2 || A_COL + 2 * KB_RES * 32 <= TMEM_COLS, "A_hi | A_lo must fit beside the accumulators");
};

// Sum over the first `valid` of 32 columns of softplus2(eta2) = log2(1 + 2^eta2): 32
// independent ex2/lg2 pairs, then a tree. (Folding the logarithms into one lg2 of the
// product of the (1 + 2^-|eta2|) factors was measured slower, both as a running product, a
// 32-long chain, and as a depth-5 product tree: the epilogue is bound by instruction issue,
// not by the SFU.)
__device__ __forceinline__ float sum_sp2_32(const uint32_t (&r)[32], int valid)
{
    float t[32];
    if (valid >= 32) {
#pragma unroll
        for (int k = 0; k < 32; ++k) t[k] = softplus2(__uint_as_float(r[k]));
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) t[k] = (k < valid) ? softplus2(__uint_as_float(r[k])) : 0.0f;
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

// A 4 x 4 transpose of 16-byte chunks across each aligned group of four lanes: on entry lane
// 4g + s holds chunks 0..3 of its own row s; on exit slot s of lane 4g + c holds chunk c of
// row s of the group. Two butterfly exchanges, across lane bit 0 and then bit 1: in each, a
// lane trades the two slots whose index bit differs from its own lane bit with its partner.
__device__ __forceinline__ void xpose4_u4(uint4 (&v)[4], int lane)
{
#pragma unroll
    for (int bit = 0; bit < 2; ++bit) {
        const int m = 1 << bit;
        const bool lb = (lane >> bit) & 1;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int q0 = bit == 0 ? 2 * k : k;  // the pair's slot with index bit `bit` clear
            const int q1 = q0 | m;                // and set
            const uint4 send = lb ? v[q0] : v[q1];
            uint4 recv;
            recv.x = __shfl_xor_sync(0xffffffffu, send.x, m);
            recv.y = __shfl_xor_sync(0xffffffffu, send.y, m);
            recv.z = __shfl_xor_sync(0xffffffffu, send.z, m);
            recv.w = __shfl_xor_sync(0xffffffffu, send.w, m);
            if (lb)
                v[q0] = recv;
            else
                v[q1] = recv;
        }
    }
}

// Residual mode: besides the softplus sum, r = y - logit^{-1}(eta) for the 32 columns of
// this chunk is stored as BF16 hi (row of R) and lo (row + n_r) and summed into rsum.
// eta2 = eta log2(e): with e = 2^-|eta2|, softplus2 = max(eta2, 0) + log2(1 + e) and
// logit^{-1}(eta) = 1/(1 + e) for eta >= 0, e/(1 + e) otherwise (one ex2 shared).
// FULL: all 32 columns are individuals (every chunk but the last of a region's row), so no
// column needs the valid-count test. The hi | lo split is taken two columns at a time (one
// paired conversion each for hi and lo), with the same round-to-nearest values as one at a time.
template <bool FULL>
__device__ __forceinline__ float resid_chunk(const float (&v)[32], int valid, uint32_t ybits,
                                             __nv_bfloat16* __restrict__ rrow, int64_t n_r, float& rsum)
{
    float sp[32];
    uint32_t hi2[16], lo2[16];  // BF16 pairs, column 2q in the low half
    float rs[32];
#pragma unroll
    for (int k = 0; k < 32; k += 2) {
        float r2[2];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const int kk = k + d;
            const float x = v[kk];
            const bool ok = FULL || kk < valid;
            const float e = ex2_approx(-fabsf(x));
            const float onepe = 1.0f + e;
            const float inv = rcp_approx(onepe);
            const float sig = (x >= 0.0f) ? inv : e * inv;
            const bool yk = (ybits >> kk) & 1u;
            sp[kk] = ok ? fmaxf(x, 0.0f) + lg2_approx(onepe) : 0.0f;
            const float r = ok ? (yk ? 1.0f : 0.0f) - sig : 0.0f;
            rs[kk] = r;
            r2[d] = r;
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(r2[0], r2[1]);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(r2[0] - hf.x, r2[1] - hf.y);
        hi2[k >> 1] = *reinterpret_cast<const uint32_t*>(&h);
        lo2[k >> 1] = *reinterpret_cast<const uint32_t*>(&l);
    }
    // 16-byte stores of the 32 hi and 32 lo values (rrow is 64-byte aligned), transposed in
    // groups of four lanes first, so that each store instruction writes eight rows' whole
    // 64-byte segments instead of one 16-byte piece of each of 32 rows
    uint4 h4[4], l4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h4[q] = make_uint4(hi2[4 * q], hi2[4 * q + 1], hi2[4 * q + 2], hi2[4 * q + 3]);
        l4[q] = make_uint4(lo2[4 * q], lo2[4 * q + 1], lo2[4 * q + 2], lo2[4 * q + 3]);
    }
    const int lane = threadIdx.x & 31;
    xpose4_u4(h4, lane);
    xpose4_u4(l4, lane);
    const int c4 = lane & 3;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        __nv_bfloat16* dst = rrow + (int64_t)(s - c4) * 2 * n_r + 8 * c4;
        *reinterpret_cast<uint4*>(dst) = h4[s];
        *reinterpret_cast<uint4*>(dst + n_r) = l4[s];
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)
#pragma unroll
        for (int k = 0; k < w; ++k) {
            sp[k] += sp[k + w];
            rs[k] += rs[k + w];
        }
    rsum = rs[0];
    return sp[0];
}

// The units of CTA b of G. Contiguous ranges of the row-major unit order, except with a
// resident A, at least one CTA per particle tile, and no longer longest range than the
// contiguous split's: then tile mt gets floor or ceil of G / m_tiles CTAs that split its
// n-tiles, so no CTA reloads A in the middle of its range.
__device__ __forceinline__ void tc_unit_range(bool ar, int m_tiles, int n_tiles, int b, int G, int64_t& u_begin,
                                              int64_t& u_end)
{
    const int64_t U = (int64_t)m_tiles * n_tiles;
    const int q = G / m_tiles, r = G % m_tiles;
    if (ar && q >= 1 && (n_tiles + q - 1) / q <= (U + G - 1) / G) {
        int mt, k, cnt;
        if (b < r * (q + 1)) {
            mt = b / (q + 1);
            k = b % (q + 1);
            cnt = q + 1;
        } else {
            const int b2 = b - r * (q + 1);
            mt = r + b2 / q;
            k = b2 % q;
            cnt = q;
        }
        u_begin = (int64_t)mt * n_tiles + (int64_t)n_tiles * k / cnt;
        u_end = (int64_t)mt * n_tiles + (int64_t)n_tiles * (k + 1) / cnt;
    } else {
        u_begin = U * b / G;
        u_end = U * (b + 1) / G;
    }
}

// What the pipeline needs about one unit: a particle tile (128 rows of A) against an n-tile
// (BN rows of G) of one region. `key` names the particle tile: consecutive units with the same
// key share the resident A.
struct TcUnit {
    const CUtensorMap* A;   // particle operand (64-column boxes) and, for a narrow last
    const CUtensorMap* At;  //   k-block, the tw-column boxes
    const CUtensorMap* B;   // genotype operand, likewise
    const CUtensorMap* Bt;
    const __nv_bfloat16* Araw;  // the particle operand itself (rows of 2 Kp), for a TMEM-resident A
    int tw, kblocks, ksteps, Kp, n, mt, nt;
    int64_t key;
    float* partial;
    int64_t N_pad;
    const uint32_t* ybits;
    __nv_bfloat16* R;
    int64_t n_r;
    float* rsum_part;
};

// AR = 2: this warp's share of particle tile t.mt's operand rows, copied into TMEM. Row `row`
// (one of the warp's own 32 lanes) takes the 16-byte chunks c of [A_hi | A_lo]: c < KC =
// 2 ksteps is A_hi's BF16 columns 8c..8c+7, c >= KC A_lo's 8(c - KC)..; chunk c goes to TMEM
// columns 4c..4c+3, and the GROUPS warps of one lane quadrant split the chunks between them.
template <int GROUPS>
__device__ __forceinline__ void ta_copy_A(const TcUnit& t, uint32_t taddr, int grp, int row)
{
    constexpr int BATCH = 8;  // 16-byte chunks in flight per thread
    const int KC = 2 * t.ksteps;
    const int c0 = (2 * KC * grp) / GROUPS, c1 = (2 * KC * (grp + 1)) / GROUPS;
    const uint4* a = reinterpret_cast<const uint4*>(t.Araw + ((int64_t)t.mt * BM + row) * (int64_t)(2 * t.Kp));
    const int lo_off = t.Kp / 8;  // chunks from A_hi's first column to A_lo's
    for (int cb = c0; cb < c1; cb += BATCH) {
        uint4 v[BATCH];
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            const int c = cb + k;
            if (c < c1) v[k] = __ldg(a + (c < KC ? c : lo_off + (c - KC)));
        }
#pragma unroll
        for (int k = 0; k < BATCH; ++k)  // warp-uniform condition: the stores are warp-collective
            if (cb + k < c1) tmem_st4(taddr + 4u * (uint32_t)(cb + k), v[k]);
    }
}

// One region, its maps passed as kernel parameters: the units of CTA b are tc_unit_range's.
struct TcSingleSource {
    const CUtensorMap *A, *B, *At, *Bt;
    const __nv_bfloat16* Araw;
    int tw, n_tiles, m_tiles, kblocks, ksteps, Kp, n;
    float* partial;
    int64_t N_pad;
    const uint32_t* ybits;
    __nv_bfloat16* R;
    int64_t n_r;
    float* rsum_part;

    __device__ __forceinline__ void range(bool ar, int b, int G, int64_t& ub, int64_t& ue) const
    {
        tc_unit_range(ar, m_tiles, n_tiles, b, G, ub, ue);
    }
    __device__ __forceinline__ int64_t key(int64_t u) const { return u / n_tiles; }
    __device__ __forceinline__ TcUnit unit(int64_t u) const
    {
        TcUnit t;
        t.A = A;
        t.At = At;
        t.B = B;
        t.Bt = Bt;
        t.Araw = Araw;
        t.tw = tw;
        t.kblocks = kblocks;
        t.ksteps = ksteps;
        t.Kp = Kp;
        t.n = n;
        t.mt = (int)(u / n_tiles);
        t.nt = (int)(u % n_tiles);
        t.key = t.mt;
        t.partial = partial;
        t.N_pad = N_pad;
        t.ybits = ybits;
        t.R = R;
        t.n_r = n_r;
        t.rsum_part = rsum_part;
        return t;
    }
    __device__ __forceinline__ void prefetch(int64_t) const
    {
        tma_prefetch_desc(A);
        tma_prefetch_desc(B);
        if (tw) {
            tma_prefetch_desc(At);
            tma_prefetch_desc(Bt);
        }
    }
};

// Many regions in one launch: regs[r] holds region r's maps and sizes, its units are the
// global units [regs[r].unit0, regs[r + 1].unit0), and CTA b takes the global units
// [cta_units[b], cta_units[b + 1]) (split by the host in proportion to the work).
struct TcGroupedSource {
    const TcRegion* regs;
    int R;
    const int64_t* cta_units;

    __device__ __forceinline__ void range(bool, int b, int, int64_t& ub, int64_t& ue) const
    {
        ub = cta_units[b];
        ue = cta_units[b + 1];
    }
    __device__ __forceinline__ int region_of(int64_t u) const
    {
        int lo = 0, hi = R - 1;  // the last region whose first unit is <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (regs[mid].unit0 <= u)
                lo = mid;
            else
                hi = mid - 1;
        }
        return lo;
    }
    __device__ __forceinline__ int64_t key(int64_t u) const
    {
        const int r = region_of(u);
        return ((int64_t)r << 32) | ((u - regs[r].unit0) / regs[r].n_tiles);
    }
    __device__ __forceinline__ TcUnit unit(int64_t u) const
    {
        const int r = region_of(u);
        const TcRegion& g = regs[r];
        const int64_t lu = u - g.unit0;
        TcUnit t;
        t.A = &g.A;
        t.At = &g.At;
        t.B = &g.B;
        t.Bt = &g.Bt;
        t.Araw = nullptr;  // grouped launches keep A in shared memory (AR < 2)
        t.tw = g.tw;
        t.kblocks = g.kblocks;
        t.ksteps = g.ksteps;
        t.Kp = g.Kp;
        t.n = g.n;
        t.mt = (int)(lu / g.n_tiles);
        t.nt = (int)(lu % g.n_tiles);
        t.key = ((int64_t)r << 32) | t.mt;
        t.partial = g.partial;
        t.N_pad = g.N_pad;
        t.ybits = g.ybits;
        t.R = g.R;
        t.n_r = g.n_r;
        t.rsum_part = g.rsum_part;
        return t;
    }
    __device__ __forceinline__ void prefetch(int64_t u) const
    {
        const TcRegion& g = regs[region_of(u)];
        tma_prefetch_desc(&g.A);
        tma_prefetch_desc(&g.B);
        if (g.tw) {
            tma_prefetch_desc(&g.At);
            tma_prefetch_desc(&g.Bt);
        }
    }
};

// The pipeline of one CTA over units [u_begin, u_end) of `src`.
template <int BN, int STAGES, bool RESID, int AR, int EW, class Src>
__device__ __forceinline__ void loglik_tc_body(const Src& src, uint32_t* __restrict__ err, uint64_t wait_ns, int stall)
{
    using C = TcCfg<BN, STAGES, AR>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t stage0 = sbase + C::A_RES;  // first pipeline stage
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = sbase + C::BAR_OFF;
    const uint32_t drain_bar = bar0 + 8 * (2 * STAGES + 4);
    const uint32_t aempty_bar = bar0 + 8 * (2 * STAGES + 5);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::SLOT_OFF);
#define FULL_BAR(s) (bar0 + 8u * (uint32_t)(s))
#define EMPTY_BAR(s) (bar0 + 8u * (uint32_t)(STAGES + (s)))
#define ACCF_BAR(b) (bar0 + 8u * (uint32_t)(2 * STAGES + (b)))
#define ACCE_BAR(b) (bar0 + 8u * (uint32_t)(2 * STAGES + 2 + (b)))
// AR = 1: one per k-block of the resident A, so that the first MMAs of an epoch need only
// their own k-block of A, not all of it. AR = 2: AFULL_BAR(0) alone, arrived at by every
// epilogue warp once its share of A is in TMEM.
#define AFULL_BAR(kb) (bar0 + 8u * (uint32_t)(2 * STAGES + 6 + (kb)))

    int64_t u_begin, u_end;
    src.range(AR, (int)blockIdx.x, (int)gridDim.x, u_begin, u_end);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(FULL_BAR(s), 1);
            mbar_init(EMPTY_BAR(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(ACCF_BAR(b), 1);
            mbar_init(ACCE_BAR(b), Epi<EW>::WARPS);
        }
        mbar_init(drain_bar, 1);
        mbar_init(aempty_bar, 1);
        for (int kb = 0; kb < KB_RES; ++kb) mbar_init(AFULL_BAR(kb), (AR == 2 && kb == 0) ? Epi<EW>::WARPS : 1);
        mbar_fence_init();
    }
    if (warp == 0 && lane == 0 && u_begin < u_end) src.prefetch(u_begin);
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // everything above is independent of the previous kernel; what follows reads A and
    // writes the partials the previous kernel may still be reading
    grid_dependency_wait();
    grid_launch_dependents();

    // The last k-block of a unit is `tw` (16 or 32) columns wide when the K extent does not
    // fill it: its tiles come from the narrow maps (32- or 64-byte swizzle) and carry fewer bytes.
    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            int epoch = -1;         // A-resident: one epoch per run of units with the same key
            int64_t cur_key = -1;
            int a_issued = 0;       // k-blocks of the current epoch's A sent out
            // bit kb: the parity of AFULL(kb)'s current phase. Each barrier keeps its own phase,
            // because regions of one grouped launch can have different numbers of k-blocks,
            // so not every epoch uses every AFULL(kb).
            uint32_t a_par = 0;
            for (int64_t u = u_begin; u < u_end && ok; ++u) {
                const TcUnit t = src.unit(u);
                const int kb_last = t.kblocks - 1;
                const uint32_t a_tail = t.tw ? (uint32_t)(BM * t.tw * 2) : (uint32_t)C::A_TILE;
                const uint32_t b_tail = t.tw ? (uint32_t)(BN * t.tw * 2) : (uint32_t)C::B_TILE;
                bool a_first = false;  // the epoch's first unit: A's k-blocks go out between its G stages
                if (C::COMPACT && t.kblocks == KB_RES && t.tw == 0) {  // would overrun the compact A
                    atomicOr(err, DERR_INPUT);
                    ok = false;
                    break;
                }
                if (AR == 1 && t.key != cur_key) {
                    ++epoch;
                    // the previous epoch's MMAs must be done with the resident A
                    if (epoch > 0 && !mbar_wait_bounded(aempty_bar, (uint32_t)((epoch - 1) & 1), err, wait_ns)) {
                        ok = false;
                        break;
                    }
                    if (epoch > 0 && (t.key >> 32) != (cur_key >> 32)) src.prefetch(u);  // a new region
                    a_first = true;
                    a_issued = 0;
                    cur_key = t.key;
                } else if (AR != 1 && u > u_begin && (t.key >> 32) != (cur_key >> 32)) {
                    src.prefetch(u);
                }
                if (AR != 1) cur_key = t.key;
                for (int kb = 0; kb < t.kblocks; ++kb) {
                    if (AR == 1 && a_first) {
                        const uint32_t a = sbase + (uint32_t)(kb * 2 * C::A_TILE);
                        const bool tail = t.tw && kb == kb_last;
                        const CUtensorMap* ma = tail ? t.At : t.A;
                        const uint32_t lo = (tail || kb == 3) ? (uint32_t)C::TAIL_LO : (uint32_t)C::A_TILE;
                        mbar_arrive_expect_tx(AFULL_BAR(kb), tail ? 2u * a_tail : 2u * (uint32_t)C::A_TILE);
                        tma_load_2d(a, ma, AFULL_BAR(kb), kb * BK, t.mt * BM);
                        tma_load_2d(a + lo, ma, AFULL_BAR(kb), t.Kp + kb * BK, t.mt * BM);
                        a_par ^= 1u << kb;
                        ++a_issued;
                    }
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded(EMPTY_BAR(s), ph ^ 1u, err, wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = stage0 + s * C::STAGE;
                    const bool tail = t.tw && kb == kb_last;
                    const CUtensorMap* ma = tail ? t.At : t.A;
                    const CUtensorMap* mb = tail ? t.Bt : t.B;
                    const uint32_t bytes = AR ? (tail ? b_tail : (uint32_t)C::B_TILE)
                                              : (tail ? 2u * a_tail + b_tail : (uint32_t)C::STAGE);
                    mbar_arrive_expect_tx(FULL_BAR(s), bytes);
                    if (AR) {
                        tma_load_2d(st, mb, FULL_BAR(s), kb * BK, t.nt * BN);
                    } else {
                        tma_load_2d(st, ma, FULL_BAR(s), kb * BK, t.mt * BM);
                        tma_load_2d(st + C::A_TILE, ma, FULL_BAR(s), t.Kp + kb * BK, t.mt * BM);
                        tma_load_2d(st + 2 * C::A_TILE, mb, FULL_BAR(s), kb * BK, t.nt * BN);
                    }
                    ++it;
                }
            }
            // Never leave with a copy in flight: the most recent use of each stage must have landed,
            // and so must the last resident A.
            const uint32_t last = it < (uint32_t)STAGES ? it : (uint32_t)STAGES;
            for (uint32_t k = 1; k <= last; ++k) {
                const uint32_t i2 = it - k;
                mbar_drain(FULL_BAR(i2 % STAGES), (i2 / STAGES) & 1u, err);
            }
            if (AR == 1 && epoch >= 0)  // the phases last armed (their parity bits were flipped since)
                for (int kb = 0; kb < a_issued; ++kb) mbar_drain(AFULL_BAR(kb), ((a_par >> kb) & 1u) ^ 1u, err);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16_f32(BM, BN);
            uint32_t it = 0;
            int lt = 0;
            bool ok = true;
            int64_t cur_key = -1;
            uint32_t a_par = 0;  // bit kb: the parity of AFULL(kb)'s phase to wait for next
            int ta_epoch = 0;    // AR = 2: epochs whose A this thread has waited for
            // Injected stall (tests of the timeout path): wait first on the drain barrier,
            // which nothing arrives at before this thread's own final commit, so the wait
            // runs out after wait_ns; no MMA has been issued, and the other roles give up and
            // drain as after any timeout.
            if (stall && !mbar_wait_bounded(drain_bar, 0u, err, wait_ns)) ok = false;
            for (int64_t u = u_begin; u < u_end && ok; ++u, ++lt) {
                const TcUnit t = src.unit(u);
                const int kb_last = t.kblocks - 1;
                const uint32_t tail_row = t.tw ? (uint32_t)(t.tw * 2) : 128u;
                const uint32_t b = (uint32_t)(lt % C::NACC), aph = (uint32_t)((lt / C::NACC) & 1);
                if (!mbar_wait_bounded(ACCE_BAR(b), aph ^ 1u, err, wait_ns)) {
                    ok = false;
                    break;
                }
                bool a_first = false;  // the epoch's first unit waits for (each k-block of) A
                if (AR && t.key != cur_key) {
                    a_first = true;
                    cur_key = t.key;
                }
                if (AR == 2 && a_first) {
                    if (!mbar_wait_bounded(AFULL_BAR(0), (uint32_t)(ta_epoch & 1), err, wait_ns)) {
                        ok = false;
                        break;
                    }
                    ++ta_epoch;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + b * (uint32_t)BN;
                for (int kb = 0; kb < t.kblocks; ++kb) {
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
                    if (AR == 1 && a_first) {
                        if (!mbar_wait_bounded(AFULL_BAR(kb), (a_par >> kb) & 1u, err, wait_ns)) {
                            ok = false;
                            break;
                        }
                        a_par ^= 1u << kb;
                    }
                    if (!mbar_wait_bounded(FULL_BAR(s), ph, err, wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = stage0 + s * C::STAGE;
                    const uint32_t rb = (t.tw && kb == kb_last) ? tail_row : 128u;
                    const uint64_t bg = sdesc_swz(AR ? st : st + 2 * C::A_TILE, rb);
                    const int nks = (t.ksteps - 4 * kb) < 4 ? (t.ksteps - 4 * kb) : 4;
                    if (AR == 2) {
                        // A_hi of k-step g in TMEM columns A_COL + 8 g, A_lo 8 ksteps further on
                        const uint32_t ahi = tmem_base + C::A_COL + 32u * (uint32_t)kb;
                        const uint32_t alo = ahi + 8u * (uint32_t)t.ksteps;
                        for (int ks = 0; ks < nks; ++ks)
                            umma_bf16_ta(d, ahi + 8u * ks, bg + 2u * ks, IDESC, (kb | ks) != 0 ? 1u : 0u);
                        for (int ks = 0; ks < nks; ++ks) umma_bf16_ta(d, alo + 8u * ks, bg + 2u * ks, IDESC, 1u);
                    } else {
                        const uint32_t a = AR ? sbase + (uint32_t)(kb * 2 * C::A_TILE) : st;
                        const uint32_t lo = (AR && (rb != 128u || kb == 3)) ? (uint32_t)C::TAIL_LO : (uint32_t)C::A_TILE;
                        const uint64_t ahi = sdesc_swz(a, rb);
                        const uint64_t alo = sdesc_swz(a + lo, rb);
                        for (int ks = 0; ks < nks; ++ks)  // +32 bytes per K = 16 step inside the swizzle row
                            umma_bf16(d, ahi + 2u * ks, bg + 2u * ks, IDESC, (kb | ks) != 0 ? 1u : 0u);
                        for (int ks = 0; ks < nks; ++ks) umma_bf16(d, alo + 2u * ks, bg + 2u * ks, IDESC, 1u);
                    }
                    umma_commit(EMPTY_BAR(s));
                    ++it;
                }
                if (!ok) break;
                umma_commit(ACCF_BAR(b));
                // the resident A is free once this unit's MMAs are done, if the next unit
                // belongs to another particle tile
                if (AR && u + 1 < u_end && src.key(u + 1) != t.key) umma_commit(aempty_bar);
            }
            // Wait for every MMA this thread issued before TMEM can be released.
            umma_commit(drain_bar);
            mbar_drain(drain_bar, 0u, err);
        }
    } else {
        // --------------------------------------------------------------- epilogue
        using E = Epi<EW>;
        // 32-column chunks per warp and tile, rounded up: with BN = 224 the second column group
        // has 3 chunks, and its fourth load reads TMEM columns past the tile (inside the
        // allocation), which the valid-column count then skips
        constexpr int CPW = (BN / 32 + E::GROUPS - 1) / E::GROUPS;
        const int quad = warp & 3;                // TMEM lane quadrant this warp may access
        const int grp = (warp - 2) >> 2;          // column group
        const int row = quad * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        const int col0 = grp * CPW * 32;
        int lt = 0;
        int64_t ta_key = -1;  // AR = 2: the particle tile whose A is in TMEM
        int ta_epoch = 0;
        for (int64_t u = u_begin; u < u_end; ++u, ++lt) {
            const TcUnit t = src.unit(u);
            if (AR == 2 && t.key != ta_key) {
                // the previous epoch's MMAs are done with A (their commit); then this warp copies
                // its share of the new particle tile's rows into TMEM and says so
                if (ta_epoch > 0 && !mbar_wait_bounded(aempty_bar, (uint32_t)((ta_epoch - 1) & 1), err, wait_ns)) break;
                tc_fence_after();
                ta_copy_A<E::GROUPS>(t, tmem_base + C::A_COL + lane_addr, grp, row);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(AFULL_BAR(0));
                ta_key = t.key;
                ++ta_epoch;
            }
            const uint32_t b = (uint32_t)(lt % C::NACC), aph = (uint32_t)((lt / C::NACC) & 1);
            if (!mbar_wait_bounded(ACCF_BAR(b), aph, err, wait_ns)) break;
            tc_fence_after();
            // valid columns from col0 on: up to the last individual and to the tile's edge (a
            // rounded-up chunk count reaches past BN when BN / 32 is odd)
            const int valid0 = min(t.n - t.nt * BN, BN) - col0;
            const uint32_t tbase = tmem_base + lane_addr + b * (uint32_t)BN + (uint32_t)col0;
            const int64_t prow = (int64_t)t.mt * BM + row;
            const int64_t gc0 = ((int64_t)t.nt * BN + col0) >> 5;  // global index of the first chunk
            float* __restrict__ partial = t.partial;
            if (!RESID) {
                // all of this warp's chunks in flight at once, then the buffer goes back to the MMA
                uint32_t r[CPW][32];
#pragma unroll
                for (int ch = 0; ch < CPW; ++ch) tmem_ld32_async(tbase + (uint32_t)(32 * ch), r[ch]);
#pragma unroll
                for (int ch = 0; ch < CPW; ++ch) tmem_wait_ld(r[ch]);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(ACCE_BAR(b));
#pragma unroll
                for (int ch = 0; ch < CPW; ++ch) {
                    const int valid = valid0 - 32 * ch;
                    if (valid <= 0) break;
                    partial[(gc0 + ch) * t.N_pad + prow] = -sum_sp2_32(r[ch], valid);
                }
            } else {
                for (int ch = 0; ch < CPW; ++ch) {
                    const int valid = valid0 - 32 * ch;
                    if (valid <= 0) break;
                    uint32_t r[32];
                    tmem_ld32_async(tbase + (uint32_t)(32 * ch), r);
                    tmem_wait_ld(r);
                    float v[32];
#pragma unroll
                    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
                    const int64_t i0 = (int64_t)t.nt * BN + col0 + 32 * ch;
                    float rs;
                    const uint32_t yb = __ldg(t.ybits + (i0 >> 5));
                    __nv_bfloat16* rrow = t.R + prow * 2 * t.n_r + i0;
                    const float sp = valid >= 32 ? resid_chunk<true>(v, valid, yb, rrow, t.n_r, rs)
                                                 : resid_chunk<false>(v, valid, yb, rrow, t.n_r, rs);
                    partial[(gc0 + ch) * t.N_pad + prow] = -sp;
                    t.rsum_part[(gc0 + ch) * t.N_pad + prow] = rs;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(ACCE_BAR(b));
            }
        }
    }
#undef FULL_BAR
#undef EMPTY_BAR
#undef ACCF_BAR
#undef ACCE_BAR
#undef AFULL_BAR
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

template <int BN, int STAGES, bool RESID, int AR, int EW>
__global__ void __launch_bounds__(Epi<EW>::THREADS, 1)
    k_loglik_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const __grid_constant__ CUtensorMap mapAt, const __grid_constant__ CUtensorMap mapBt,
                const __nv_bfloat16* __restrict__ Araw, int tw,
                int n_tiles, int m_tiles, int kblocks, int ksteps, int Kp, int n, float* __restrict__ partial,
                int64_t N_pad,
                uint32_t* __restrict__ err, const uint32_t* __restrict__ ybits, __nv_bfloat16* __restrict__ R,
                int64_t n_r, float* __restrict__ rsum_part, uint64_t wait_ns, int stall)
{
    const TcSingleSource src{&mapA, &mapB, &mapAt, &mapBt, Araw, tw, n_tiles, m_tiles, kblocks, ksteps, Kp, n,
                             partial, N_pad, ybits, R, n_r, rsum_part};
    loglik_tc_body<BN, STAGES, RESID, AR, EW>(src, err, wait_ns, stall);
}

// The same pipeline over the units of many regions (a batched sweep's move): region tables
// and per-CTA unit ranges in global memory.
template <int BN, int STAGES, bool RESID, int AR, int EW>
__global__ void __launch_bounds__(Epi<EW>::THREADS, 1)
    k_loglik_tc_grouped(const TcRegion* __restrict__ regs, int R, const int64_t* __restrict__ cta_units,
                        uint32_t* __restrict__ err, uint64_t wait_ns)
{
    const TcGroupedSource src{regs, R, cta_units};
    loglik_tc_body<BN, STAGES, RESID, AR, EW>(src, err, wait_ns, 0);
}

// ----------------------------------------------------------------------- adjoint
// C[k, j] = sum_i r_ki g_ij for 128 particles x BN2 markers, contracting over the
// individuals of one K-split range: A = [R_hi | R_lo] (N_pad x 2 n_r), B = G^T (markers x
// n_r, exact BF16), both K-major with the 128-byte swizzle. A unit is one output tile (mt,
// pt) of one K-split ks; a CTA takes units blockIdx.x, blockIdx.x + gridDim.x, ... (one unit
// each when the grid covers them all), with a double-buffered accumulator in TMEM so that a
// unit's MMAs overlap the previous unit's copy-out. Warps 2..5 copy the FP32 accumulator to
// gpart[ks][particle][marker], 32 x 32 blocks at a time through a shared-memory transpose:
// a lane holds one particle's row of a block after tcgen05.ld, and a warp's stores then write
// whole 128-byte row segments instead of 32 rows' single words per instruction. Every unit
// runs the same MMAs whichever CTA takes it, so the partials do not depend on the grid. The final gradient (C - m_j sum_i r_ki) / s_j is
// formed by k_grad_finish.
constexpr int ADJ_THREADS = 64 + 32 * 4;

template <int BN2, int STAGES>
struct AdjCfg {
    static constexpr int A_TILE = BM * BK * 2;
    static constexpr int B_TILE = BN2 * BK * 2;
    static constexpr int STAGE = 2 * A_TILE + B_TILE;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int NBARS = 2 * STAGES + 5;  // full[S], empty[S], acc_full[2], acc_empty[2], drain
    static constexpr int SLOT_OFF = BAR_OFF + NBARS * 8;
    // one 32 x 33 FP32 transpose buffer per epilogue warp (the padding column keeps both the
    // row writes and the column reads free of bank conflicts)
    static constexpr int XPOSE_OFF = SLOT_OFF + 16;
    static constexpr int XPOSE_FLOATS = 32 * 33;
    static constexpr int SMEM = XPOSE_OFF + 4 * XPOSE_FLOATS * 4 + 1024;
    static constexpr uint32_t ACC_STRIDE = 256;  // TMEM columns between the two accumulator buffers
    static constexpr uint32_t TMEM_COLS = 512;
    static_assert(STAGE % 1024 == 0, "tiles must stay 1024-byte aligned");
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(BN2 % 16 == 0 && BN2 <= 256, "MMA N");
};

template <int BN2, int STAGES>
__global__ void __launch_bounds__(ADJ_THREADS, 1)
    k_adjoint_tc(const __grid_constant__ CUtensorMap mapR, const __grid_constant__ CUtensorMap mapGT, int m_tiles,
                 int p_tiles, int kblocks, int ksplit, int n_r, int p, float* __restrict__ gpart, int64_t N_pad,
                 uint32_t* __restrict__ err, uint64_t wait_ns, int r_hint)
{
    using C = AdjCfg<BN2, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = sbase + C::BAR_OFF;
    const uint32_t drain_bar = bar0 + 8u * (uint32_t)(2 * STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::SLOT_OFF);
#define FULL_BAR(s) (bar0 + 8u * (uint32_t)(s))
#define EMPTY_BAR(s) (bar0 + 8u * (uint32_t)(STAGES + (s)))
#define ACCF_BAR(b) (bar0 + 8u * (uint32_t)(2 * STAGES + (b)))
#define ACCE_BAR(b) (bar0 + 8u * (uint32_t)(2 * STAGES + 2 + (b)))
    const int units = m_tiles * p_tiles * ksplit;
    // unit u = (mt, pt, ks), ks fastest; its K range [kb0, kb1) of k-blocks
    auto decode = [&](int u, int& mt, int& pt, int& kb0, int& kb1, int& ks) {
        ks = u % ksplit;
        pt = (u / ksplit) % p_tiles;
        mt = u / (ksplit * p_tiles);
        kb0 = (int)((int64_t)kblocks * ks / ksplit);
        kb1 = (int)((int64_t)kblocks * (ks + 1) / ksplit);
    };

    if (threadIdx.x == 0) {
        for (int q = 0; q < STAGES; ++q) {
            mbar_init(FULL_BAR(q), 1);
            mbar_init(EMPTY_BAR(q), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(ACCF_BAR(b), 1);
            mbar_init(ACCE_BAR(b), 4);  // the four epilogue warps
        }
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
    // launched as a programmatic dependent of the residual pass: the prologue above overlaps
    // its tail, and R is read only after it has finished
    grid_dependency_wait();
    grid_launch_dependents();

    if (warp == 0) {
        if (lane == 0) {
            // R is read once, here: with r_hint its lines go first when L2 needs room, ahead
            // of the particle state that the move kernel reads next
            const uint64_t r_pol = r_hint ? l2_policy_evict_first() : 0;
            uint32_t it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
                int mt, pt, kb0, kb1, ks;
                decode(u, mt, pt, kb0, kb1, ks);
                for (int kb = kb0; kb < kb1; ++kb) {
                    const uint32_t q = it % STAGES, ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded(EMPTY_BAR(q), ph ^ 1u, err, wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + q * C::STAGE;
                    mbar_arrive_expect_tx(FULL_BAR(q), (uint32_t)C::STAGE);
                    if (r_hint) {
                        tma_load_2d_hint(st, &mapR, FULL_BAR(q), kb * BK, mt * BM, r_pol);
                        tma_load_2d_hint(st + C::A_TILE, &mapR, FULL_BAR(q), n_r + kb * BK, mt * BM, r_pol);
                    } else {
                        tma_load_2d(st, &mapR, FULL_BAR(q), kb * BK, mt * BM);
                        tma_load_2d(st + C::A_TILE, &mapR, FULL_BAR(q), n_r + kb * BK, mt * BM);
                    }
                    tma_load_2d(st + 2 * C::A_TILE, &mapGT, FULL_BAR(q), kb * BK, pt * BN2);
                    ++it;
                }
            }
            const uint32_t last = it < (uint32_t)STAGES ? it : (uint32_t)STAGES;
            for (uint32_t k = 1; k <= last; ++k) {
                const uint32_t i2 = it - k;
                mbar_drain(FULL_BAR(i2 % STAGES), (i2 / STAGES) & 1u, err);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16_f32(BM, BN2);
            uint32_t it = 0;
            int lt = 0;  // units with a non-empty K range, which use an accumulator buffer
            bool ok = true;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
                int mt, pt, kb0, kb1, ks;
                decode(u, mt, pt, kb0, kb1, ks);
                if (kb1 <= kb0) continue;
                const uint32_t b = (uint32_t)(lt & 1), aph = (uint32_t)((lt >> 1) & 1);
                if (!mbar_wait_bounded(ACCE_BAR(b), aph ^ 1u, err, wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + b * C::ACC_STRIDE;
                for (int kb = kb0; kb < kb1; ++kb) {
                    const uint32_t q = it % STAGES, ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded(FULL_BAR(q), ph, err, wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + q * C::STAGE;
                    const uint64_t ahi = sdesc_sw128(st), alo = sdesc_sw128(st + C::A_TILE);
                    const uint64_t bg = sdesc_sw128(st + 2 * C::A_TILE);
#pragma unroll
                    for (int k = 0; k < 4; ++k) umma_bf16(d, ahi + 2u * k, bg + 2u * k, IDESC, (kb > kb0 || k) ? 1u : 0u);
#pragma unroll
                    for (int k = 0; k < 4; ++k) umma_bf16(d, alo + 2u * k, bg + 2u * k, IDESC, 1u);
                    umma_commit(EMPTY_BAR(q));
                    ++it;
                }
                if (!ok) break;
                umma_commit(ACCF_BAR(b));
                ++lt;
            }
            umma_commit(drain_bar);
            mbar_drain(drain_bar, 0u, err);
        }
    } else {
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        float* xp = reinterpret_cast<float*>(smem + C::XPOSE_OFF) + quad * C::XPOSE_FLOATS;
        int lt = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x) {
            int mt, pt, kb0, kb1, ks;
            decode(u, mt, pt, kb0, kb1, ks);
            const int cols = (p - pt * BN2) < BN2 ? (p - pt * BN2) : BN2;
            float* out = gpart + ((int64_t)ks * N_pad + (int64_t)mt * BM + row) * p + (int64_t)pt * BN2;
            if (kb1 <= kb0) {
                for (int c = 0; c < cols; ++c) out[c] = 0.0f;
                continue;
            }
            const uint32_t b = (uint32_t)(lt & 1), aph = (uint32_t)((lt >> 1) & 1);
            if (!mbar_wait_bounded(ACCF_BAR(b), aph, err, wait_ns)) break;
            tc_fence_after();
            // this warp's 32 rows, from row quad * 32 of the tile
            float* out0 = gpart + ((int64_t)ks * N_pad + (int64_t)mt * BM + quad * 32) * p + (int64_t)pt * BN2;
#pragma unroll 1
            for (int c = 0; c < cols; c += 32) {
                float v[32];
                tmem_ld32(tmem_base + ((uint32_t)(quad * 32) << 16) + b * C::ACC_STRIDE + (uint32_t)c, v);
#pragma unroll
                for (int k = 0; k < 32; ++k) xp[lane * 33 + k] = v[k];
                __syncwarp();
                if (c + lane < cols) {
#pragma unroll 8
                    for (int r = 0; r < 32; ++r) out0[(int64_t)r * p + c + lane] = xp[r * 33 + lane];
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(ACCE_BAR(b));
            ++lt;
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

// grad l_kj = (sum_s C_s[k, j] - m_j sum_i r_ki) / s_j (+ the prior gradient at scale c > 0).
// A block of 8 warps takes 8 particles, one warp each. First the residual sums sum_i r_ki from
// the chunk sums rsum_part[q][k]: thread t adds chunks q = t/8, t/8 + 32, ... of particle t % 8,
// so the 8 threads of a group read one 32-byte sector per chunk (with one lane per chunk, as a
// warp per particle would, each load touches its own sector), and the 32 compensated partial
// sums of a particle are combined in slice order. Then each warp finishes its particle's row
// (lane j reads marker j of every K-split partial), C - m_j sum r by one fused multiply-add.
// The row is taken GF_U markers per lane at a time with the K-split count KS fixed at compile
// time, so that all KS x GF_U partial loads and the GF_U state loads of a batch are in flight
// together: the loads are L2 hits, and issued one dependent batch at a time their latency,
// not bandwidth, set the kernel's duration. Each marker's partials are still added in K-split
// order, so the gradient is the same bit for bit.
constexpr int GF_PARTICLES = 8;
constexpr int GF_U = 4;

template <int KS>
__global__ void __launch_bounds__(256) k_grad_finish(const float* __restrict__ gpart,
                                                     const float* __restrict__ rsum_part, int n_parts, int64_t N_pad,
                                                     int64_t N, int p, const float* __restrict__ mean_f,
                                                     const float* __restrict__ inv_sd, const float* __restrict__ B,
                                                     PriorArgs pr, double c, float* __restrict__ grad)
{
    __shared__ float2 part[32][GF_PARTICLES];
    __shared__ float rsum[GF_PARTICLES];
    grid_dependency_wait();  // the adjoint GEMM has finished
    grid_launch_dependents();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k0 = (int64_t)blockIdx.x * GF_PARTICLES;
    {
        const int kk = threadIdx.x % GF_PARTICLES, slice = threadIdx.x / GF_PARTICLES;
        const int64_t k = k0 + kk;
        FSum rq;
        if (k < N)
            for (int q = slice; q < n_parts; q += 32) rq.add(rsum_part[(int64_t)q * N_pad + k]);
        part[slice][kk] = make_float2(rq.s, rq.c);
    }
    __syncthreads();
    if (threadIdx.x < GF_PARTICLES) {
        FSum rq;
        for (int s2 = 0; s2 < 32; ++s2) {
            const float2 v = part[s2][threadIdx.x];
            rq.add(v.x);
            rq.c += v.y;
        }
        rsum[threadIdx.x] = (float)rq.value();
    }
    __syncthreads();
    const int64_t k = k0 + w;
    if (k >= N) return;
    const float rs = rsum[w];
    const float a1 = pr.a + 1.0f, ac = (float)((double)pr.a * c), inv_c = c > 0.0 ? (float)(1.0 / c) : 0.0f;
    for (int j0 = lane; j0 < p; j0 += 32 * GF_U) {
        float x[KS][GF_U], b[GF_U];
#pragma unroll
        for (int u = 0; u < GF_U; ++u) {
            const int j = j0 + 32 * u;
            const bool in = j < p;
#pragma unroll
            for (int q = 0; q < KS; ++q) x[q][u] = in ? gpart[((int64_t)q * N_pad + k) * p + j] : 0.0f;
            b[u] = (in && c > 0.0) ? B[k * p + j] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < GF_U; ++u) {
            const int j = j0 + 32 * u;
            if (j >= p) break;
            FSum g;
#pragma unroll
            for (int q = 0; q < KS; ++q) g.add(x[q][u]);
            float gv = fmaf(-mean_f[j], rs, g.value()) * inv_sd[j];
            if (c > 0.0) {
                const float bj = b[u];
                const float sg = (bj > 0.0f) ? 1.0f : ((bj < 0.0f) ? -1.0f : 0.0f);
                gv += pr.de ? -sg * inv_c : -a1 * sg / (ac + fabsf(bj));
            }
            grad[k * p + j] = gv;
        }
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
                 uint32_t box_outer, CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int STAGES, bool RESID, int AR, int EW>
cudaError_t launch_tc(const TcMaps& m, const TcPlan& plan, int64_t n, int Kp,
                      const uint32_t* ybits, float* partial, int64_t N_pad, uint32_t* err, const ResidArgs* ra,
                      uint64_t wait_ns, int stall, cudaStream_t st)
{
    using C = TcCfg<BN, STAGES, AR>;
    // programmatic dependent launch: the prologue (barriers, TMEM, descriptor prefetch)
    // overlaps the previous kernel's tail; the kernel waits for it before touching data
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.grid);
    cfg.blockDim = dim3(Epi<EW>::THREADS);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool tail = plan.tw != 0;
    return cudaLaunchKernelEx(&cfg, k_loglik_tc<BN, STAGES, RESID, AR, EW>, m.A, m.B, tail ? m.At : m.A, tail ? m.Bt : m.B,
                              m.Araw, plan.tw, plan.n_tiles, plan.m_tiles,
                              plan.kblocks, plan.ksteps, Kp, (int)n, partial, N_pad, err, ybits, ra ? ra->R : nullptr,
                              ra ? ra->n_r : (int64_t)0, ra ? ra->rsum_part : nullptr, wait_ns, stall);
}

}  // namespace

cudaError_t tc_init_attributes()
{
    cudaError_t e = cudaSuccess;
#define SET_SMEM(kern, bytes) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
#define SET_TC(BN_, S_, R_, AR_, EW_)                                                          \
    SET_SMEM((k_loglik_tc<BN_, S_, R_, AR_, EW_>), (TcCfg<BN_, S_, AR_>::SMEM));                \
    SET_SMEM((k_loglik_tc_grouped<BN_, S_, R_, AR_, EW_>), (TcCfg<BN_, S_, AR_>::SMEM))
    SET_TC(256, 3, false, true, 16);
    SET_TC(256, 3, false, false, 16);
    SET_TC(128, 4, false, true, 16);
    SET_TC(128, 4, false, false, 16);
    SET_TC(256, 3, false, true, 8);
    SET_TC(256, 3, false, false, 8);
    SET_TC(128, 6, false, true, 16);
    SET_TC(256, 3, true, true, 8);
    SET_TC(256, 3, true, false, 8);
    SET_TC(128, 4, true, true, 8);
    SET_TC(128, 4, true, false, 8);
    SET_TC(224, 4, false, true, 8);
    SET_TC(224, 4, true, true, 8);
#define SET_TC1(BN_, S_, AR_, EW_) SET_SMEM((k_loglik_tc<BN_, S_, false, AR_, EW_>), (TcCfg<BN_, S_, AR_>::SMEM))
    SET_TC1(256, 6, 2, 8);
    SET_TC1(128, 12, 2, 16);
#undef SET_TC1
#undef SET_TC
    SET_SMEM((k_adjoint_tc<ADJ_BN_SMALL, 3>), (AdjCfg<ADJ_BN_SMALL, 3>::SMEM));
    SET_SMEM((k_adjoint_tc<256, 3>), (AdjCfg<256, 3>::SMEM));
#undef SET_SMEM
    return e;
}

int tc_config_bn(int cfg) { return (cfg == 1 || cfg == 3 || cfg == 5) ? 128 : (cfg == 6 ? 224 : 256); }

bool tc_config_valid(int cfg, int64_t p)
{
    const int ksteps = (int)((p + 1 + 15) / 16), kblocks = (ksteps + 3) / 4;
    const bool resident = kblocks <= KB_RES;
    const bool narrow_last = kblocks < KB_RES || ksteps - 4 * (kblocks - 1) <= 2;  // fits a compact A
    if (cfg < 0 || cfg >= TC_CONFIGS) return false;
    if (cfg >= 3 && !resident) return false;
    return cfg != 6 || narrow_last;
}

TcPlan tc_plan(int64_t n, int p, int64_t N_pad, int num_sms, int cfg)
{
    TcPlan pl;
    pl.cfg = tc_config_valid(cfg, p) ? cfg : ((n <= 128) ? 1 : 0);  // an invalid choice falls back
    pl.BN = tc_config_bn(pl.cfg);
    pl.n_tiles = (int)((n + pl.BN - 1) / pl.BN);
    pl.m_tiles = (int)(N_pad / BM);
    pl.ksteps = (p + 1 + 15) / 16;
    pl.kblocks = (pl.ksteps + 3) / 4;
    const int64_t units = (int64_t)pl.m_tiles * pl.n_tiles;
    pl.grid = (int)(units < num_sms ? units : num_sms);
    pl.n_parts = (int)((n + 31) / 32);
    const int last = pl.ksteps - 4 * (pl.kblocks - 1);  // k-steps of the last k-block
    pl.tw = (last == 1 || last == 2) ? 16 * last : 0;
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

static CUtensorMapSwizzle tail_swizzle(int tw) { return tw == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B; }

bool tc_make_map_A_tail(CUtensorMap* map, const __nv_bfloat16* A, int64_t N_pad, int Kp, int tw)
{
    if (!tw) return true;
    return make_map_2d(map, A, (uint64_t)(2 * Kp), (uint64_t)N_pad, (uint32_t)tw, BM, tail_swizzle(tw));
}

bool tc_make_map_B_tail(CUtensorMap* map, const __nv_bfloat16* Gbf, int64_t n, int Kp, int BN, int tw)
{
    if (!tw) return true;
    return make_map_2d(map, Gbf, (uint64_t)Kp, (uint64_t)n, (uint32_t)tw, (uint32_t)BN, tail_swizzle(tw));
}

// Every kernel a tile configuration and mode launches: VISIT(BN, STAGES, RESID, AR, EW), and
// VISIT_TA(BN, STAGES, EW) for the TMEM-resident kernels (a no-op where those do not apply, so
// that the next line's shared-memory-resident kernel runs instead). The residual variant always
// has 8 epilogue warps and A in shared memory; configurations 3-5 exist only with the particle
// operand resident (their streaming fallbacks are configuration 1's or 2's).
#define TC_FOR_CONFIG(cfg, resid, ar, VISIT, VISIT_TA)                                \
    do {                                                                              \
        if (resid) {                                                                  \
            if (tc_config_bn(cfg) == 224) {                                           \
                if (ar) VISIT(224, 4, true, true, 8);                                 \
                VISIT(256, 3, true, false, 8);                                        \
            }                                                                         \
            if (tc_config_bn(cfg) == 256) {                                           \
                if (ar) VISIT(256, 3, true, true, 8);                                 \
                VISIT(256, 3, true, false, 8);                                        \
            }                                                                         \
            if (ar) VISIT(128, 4, true, true, 8);                                     \
            VISIT(128, 4, true, false, 8);                                            \
        }                                                                             \
        switch (cfg) {                                                                \
        case 6:                                                                       \
            if (ar) VISIT(224, 4, false, true, 8);                                    \
            VISIT(256, 3, false, false, 8);                                           \
        case 4:                                                                       \
            if (ar) VISIT_TA(256, 6, 8);                                              \
            if (ar) VISIT(256, 3, false, true, 8);                                    \
            VISIT(256, 3, false, false, 8);                                           \
        case 5:                                                                       \
            if (ar) VISIT_TA(128, 12, 16);                                            \
            if (ar) VISIT(128, 6, false, true, 16);                                   \
            VISIT(128, 4, false, false, 16);                                          \
        case 2:                                                                       \
            if (ar) VISIT(256, 3, false, true, 8);                                    \
            VISIT(256, 3, false, false, 8);                                           \
        case 1:                                                                       \
            if (ar) VISIT(128, 4, false, true, 16);                                   \
            VISIT(128, 4, false, false, 16);                                          \
        case 3:                                                                       \
            if (ar) VISIT(128, 6, false, true, 16);                                   \
            VISIT(128, 4, false, false, 16);                                          \
        default:                                                                      \
            if (ar) VISIT(256, 3, false, true, 16);                                   \
            VISIT(256, 3, false, false, 16);                                          \
        }                                                                             \
    } while (0)

cudaError_t launch_loglik_tc(const TcMaps& maps, const TcPlan& plan, int64_t n, int Kp,
                             const uint32_t* ybits, float* partial, int64_t N_pad, uint32_t* err, cudaStream_t st,
                             const ResidArgs* ra, uint64_t wait_ns, int stall)
{
    if (wait_ns == 0) wait_ns = WAIT_LIMIT_DEFAULT_NS;
    // A stays resident when all its k-blocks fit (K <= 256)
    const bool ar = plan.kblocks <= KB_RES;
#define TC_LAUNCH(BN_, S_, R_, AR_, EW_) \
    return launch_tc<BN_, S_, R_, AR_, EW_>(maps, plan, n, Kp, ybits, partial, N_pad, err, ra, wait_ns, stall, st)
#define TC_LAUNCH_TA(BN_, S_, EW_) \
    return launch_tc<BN_, S_, false, 2, EW_>(maps, plan, n, Kp, ybits, partial, N_pad, err, ra, wait_ns, stall, st)
    TC_FOR_CONFIG(plan.cfg, ra != nullptr, ar, TC_LAUNCH, TC_LAUNCH_TA);
#undef TC_LAUNCH_TA
#undef TC_LAUNCH
}

bool tc_plan_resident(const TcPlan& plan) { return plan.kblocks <= KB_RES; }

template <int BN, int STAGES, bool RESID, int AR, int EW>
static cudaError_t launch_grouped(const TcRegion* regs, int R, const int64_t* cta_units, int grid, uint32_t* err,
                                  cudaStream_t st, uint64_t wait_ns)
{
    using C = TcCfg<BN, STAGES, AR>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(Epi<EW>::THREADS);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_loglik_tc_grouped<BN, STAGES, RESID, AR, EW>, regs, R, cta_units, err, wait_ns);
}

cudaError_t launch_loglik_tc_grouped(const TcRegion* regs, int R, const int64_t* cta_units, int grid, int cfg, bool ar,
                                     bool resid, uint32_t* err, cudaStream_t st, uint64_t wait_ns)
{
    if (wait_ns == 0) wait_ns = WAIT_LIMIT_DEFAULT_NS;
#define G_LAUNCH(BN_, S_, R_, AR_, EW_) \
    return launch_grouped<BN_, S_, R_, AR_, EW_>(regs, R, cta_units, grid, err, st, wait_ns)
#define G_LAUNCH_TA(BN_, S_, EW_) (void)0  // grouped launches keep A in shared memory
    TC_FOR_CONFIG(cfg, resid, ar, G_LAUNCH, G_LAUNCH_TA);
#undef G_LAUNCH_TA
#undef G_LAUNCH
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
                              float* gpart, int64_t N_pad, uint32_t* err, cudaStream_t st, uint64_t wait_ns, int max_ctas,
                              bool r_last_use_hint)
{
    const int r_hint = r_last_use_hint ? 1 : 0;
    if (wait_ns == 0) wait_ns = WAIT_LIMIT_DEFAULT_NS;
    const unsigned grid = (unsigned)((max_ctas > 0 && max_ctas < a.grid) ? max_ctas : a.grid);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(ADJ_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (a.BN2 == ADJ_BN_SMALL) {
        cfg.dynamicSmemBytes = AdjCfg<ADJ_BN_SMALL, 3>::SMEM;
        return cudaLaunchKernelEx(&cfg, k_adjoint_tc<ADJ_BN_SMALL, 3>, mapR, mapGT, a.m_tiles, a.p_tiles, a.kblocks,
                                  a.ksplit, (int)a.n_r, p, gpart, N_pad, err, wait_ns, r_hint);
    }
    cfg.dynamicSmemBytes = AdjCfg<256, 3>::SMEM;
    return cudaLaunchKernelEx(&cfg, k_adjoint_tc<256, 3>, mapR, mapGT, a.m_tiles, a.p_tiles, a.kblocks, a.ksplit,
                              (int)a.n_r, p, gpart, N_pad, err, wait_ns, r_hint);
}

cudaError_t launch_grad_finish(const float* gpart, int ksplit, const float* rsum_part, int n_parts, int64_t N_pad,
                               int64_t N, int p, const float* mean_f, const float* inv_sd, const float* B, PriorArgs pr,
                               double c, float* grad, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((N + GF_PARTICLES - 1) / GF_PARTICLES));
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define GF_CASE(KS_) \
    case KS_:        \
        return cudaLaunchKernelEx(&cfg, k_grad_finish<KS_>, gpart, rsum_part, n_parts, N_pad, N, p, mean_f, inv_sd, B, pr, c, grad)
    switch (ksplit) {
        GF_CASE(1);
        GF_CASE(2);
        GF_CASE(3);
        GF_CASE(4);
        GF_CASE(5);
        GF_CASE(6);
        GF_CASE(7);
        GF_CASE(8);
    default:
        return cudaErrorInvalidValue;  // adj_plan keeps the K-split in 1..8
    }
#undef GF_CASE
}

}  // namespace spa
