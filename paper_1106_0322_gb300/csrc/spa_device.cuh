// spa_device.cuh -- device helpers shared by the library's kernels (sm_103a).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), one round
// (x0,x1,x2,x3) -> (hi(B x2) ^ x1 ^ k0, lo(B x2), hi(A x0) ^ x3 ^ k1, lo(A x0)),
// A = 0xD2511F53, B = 0xCD9E8D57, key bumped by (0x9E3779B9, 0xBB67AE85) between
// rounds. The stream layout (counter = what is drawn) is a specification:
//   init prior draws   (j/2, particle, 0, 1<<16)      u[2(j%2)] -> V_j, u[2(j%2)+1] bit 31 -> sign
//   move normals       (j/4, particle, t, 2<<16 | m)  Box-Muller on (u0,u1), (u2,u3)
//   MH uniform         (0,   particle, t, 3<<16 | m)  u0
//   resampling uniform (0,   0,        t, 4<<16)      u0
// key = (seed & 0xffffffff, seed >> 32). Open uniforms are (k + 1/2) 2^-23 with k the
// top 23 bits (exact in FP32); the resampling uniform is (top 24 bits) 2^-24 in [0,1).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace spa {

// ------------------------------------------------------------------ error word bits
enum : uint32_t {
    DERR_NONFINITE = 1u,  // non-finite log-likelihood or log-weight
    DERR_TIMEOUT = 2u,    // a bounded wait gave up
    DERR_INPUT = 4u,      // invalid input data found on the device
    DERR_ESS = 8u,        // ESS < 1 (all weights non-finite)
};

constexpr uint32_t TAG_INIT = 1u, TAG_NORMAL = 2u, TAG_ACCEPT = 3u, TAG_RESAMPLE = 4u, TAG_SITE = 5u;

// ---------------------------------------------------------------------- Philox
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hiA = __umulhi(0xD2511F53u, x.x), loA = 0xD2511F53u * x.x;
        const uint32_t hiB = __umulhi(0xCD9E8D57u, x.z), loB = 0xCD9E8D57u * x.z;
        x = make_uint4(hiB ^ x.y ^ k.x, loB, hiA ^ x.w ^ k.y, loA);
    }
    return x;
}

__device__ __forceinline__ uint2 seed_key(uint64_t seed)
{
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// (k + 1/2) 2^-23, k = top 23 bits: exact in single precision, in (0,1).
__device__ __forceinline__ float u01_open_f(uint32_t u) { return ((float)(u >> 9) + 0.5f) * 1.1920928955078125e-7f; }
__device__ __forceinline__ double u01_open_d(uint32_t u) { return ((double)(u >> 9) + 0.5) * 1.1920928955078125e-7; }
// top 24 bits / 2^24 in [0,1)
__device__ __forceinline__ double u01_d(uint32_t u) { return (double)(u >> 8) * 5.9604644775390625e-8; }

// Four standard normals (Box-Muller) of one Philox block.
__device__ __forceinline__ float4 normals4(uint64_t seed, uint32_t blk, uint32_t particle, uint32_t t, uint32_t m)
{
    const uint4 u = philox4x32_10(make_uint4(blk, particle, t, (TAG_NORMAL << 16) | m), seed_key(seed));
    float s0, c0, s1, c1;
    const float r0 = sqrtf(-2.0f * logf(u01_open_f(u.x)));
    const float r1 = sqrtf(-2.0f * logf(u01_open_f(u.z)));
    sincospif(2.0f * u01_open_f(u.y), &s0, &c0);
    sincospif(2.0f * u01_open_f(u.w), &s1, &c1);
    return make_float4(r0 * c0, r0 * s0, r1 * c1, r1 * s1);
}

// One draw from Gt(a, c) (a = +inf: double exponential) by inversion of the tail
// P(|beta| > x) = (1 + x/(a c))^-a: |beta| = a c (V^{-1/a} - 1) = a c expm1(-log(V)/a).
__device__ __forceinline__ float prior_draw(uint64_t seed, uint32_t particle, uint32_t j, float a, float c, bool de)
{
    const uint4 u = philox4x32_10(make_uint4(j >> 1, particle, 0u, TAG_INIT << 16), seed_key(seed));
    const uint32_t uv = (j & 1u) ? u.z : u.x;
    const uint32_t us = (j & 1u) ? u.w : u.y;
    const float lv = logf(u01_open_f(uv));
    const float mag = de ? -c * lv : a * c * expm1f(-lv / a);
    return (us >> 31) ? -mag : mag;
}

// ------------------------------------------------- compensated FP32 summation
// A float pair (s, c) whose value is s + c. Each addition uses the error-free TwoSum
// transformation (Knuth; Moller), so a sum of k terms carries an error of about
// 2^-24 |sum| + k 2^-48 sum|x|: double-like accuracy at FP32 cost. On GB300 the
// CUDA-core FP64 rate is a small fraction of FP32, so per-element sums use this.
struct FSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = s + x;
        const float z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
    __device__ __forceinline__ void add(FSum o)
    {
        add(o.s);
        c += o.c;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ FSum warp_sum(FSum v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FSum w;
        w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
        w.c = __shfl_xor_sync(0xffffffffu, v.c, o);
        v.add(w);
    }
    return v;
}

// ---------------------------------------------------------- reductions / helpers
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization
// may start before its predecessor finishes; this waits until the predecessor grid has
// completed and its memory is visible (a no-op for kernels launched without the attribute).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel's blocks be scheduled once every block of this grid has passed here
// (they still wait for this grid's completion before reading its results).
__device__ __forceinline__ void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// -------------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// The default limit of a bounded wait (a context can set another, spa_set_wait_limit).
constexpr uint64_t WAIT_LIMIT_DEFAULT_NS = 4000000000ull;
// The limit of a drain: the wait for a CTA's own copies and MMAs in flight before it frees
// TMEM and exits.
constexpr uint64_t DRAIN_LIMIT_NS = 100000000ull;

// Wait until the phase with the given parity of barrier `bar` has completed. Gives up
// after `limit_ns` (setting DERR_TIMEOUT) or as soon as another thread has given up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t* err,
                                                  uint64_t limit_ns = WAIT_LIMIT_DEFAULT_NS)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t spin = 1;; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 63u) == 0u) {
            if (*reinterpret_cast<volatile uint32_t*>(err) & DERR_TIMEOUT) return false;
            if (globaltimer_ns() - t0 > limit_ns) {
                atomicOr(err, DERR_TIMEOUT);
                return false;
            }
        }
    }
}

// The drain before a CTA frees TMEM or exits: wait for this CTA's own asynchronous work
// (TMA copies into its shared memory, its MMAs) to complete. Unlike mbar_wait_bounded it does
// not stop when another thread has given up -- that is exactly when the work in flight must
// still land -- and only its own limit (DRAIN_LIMIT_NS) ends it.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity, uint32_t* err)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t spin = 1;; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 63u) == 0u && globaltimer_ns() - t0 > DRAIN_LIMIT_NS) {
            atomicOr(err, DERR_TIMEOUT);
            return false;
        }
    }
}

// ------------------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
// 2-D tiled load of the box at element coordinates (x = innermost, y) into shared memory,
// completing `bytes` on barrier `bar`. x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int32_t x, int32_t y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// An L2 cache policy under which the lines an access touches become the first candidates
// for eviction (for data read for the last time).
__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// tma_load_2d with an L2 cache-policy hint for the lines it reads.
__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const CUtensorMap* map, uint32_t bar, int32_t x, int32_t y,
                                                 uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(pol)
        : "memory");
}

// --------------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (sm_100 format) for a K-major operand tile stored
// with the 128-byte swizzle: rows of 64 BF16 (128 B), 8-row atoms of 1024 B.
//   [0,14) start address >> 4, [16,30) leading byte offset >> 4 (unused here),
//   [32,46) stride byte offset >> 4 (1024 B between 8-row groups), [46,48) = 1,
//   [61,64) layout = 2 (128-byte swizzle). The tile base must be 1024-byte aligned.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t smem_addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}
// The same for a K-major tile with rows of `row_bytes` = 64 (64-byte swizzle, layout 4) or
// 32 (32-byte swizzle, layout 6): 8-row groups are 8 * row_bytes apart.
__device__ __forceinline__ uint64_t sdesc_swz(uint32_t smem_addr, uint32_t row_bytes)
{
    if (row_bytes == 128u) return sdesc_sw128(smem_addr);
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)((8u * row_bytes) >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)(row_bytes == 64u ? 4u : 6u) << 61;
    return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B (both K-major), FP32 accumulate:
//   [4,6) D format = 1 (F32), [7,10) A = 1 (BF16), [10,13) B = 1 (BF16),
//   [15] A major = 0 (K), [16] B major = 0 (K), [17,23) N >> 3, [24,29) M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T for one K = 16 slice; accumulate != 0 adds to D.
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T for one K = 16 slice, A read from tensor memory: row m of
// A in lane m, K packed two BF16 per 32-bit column (even k in the low half), 8 columns per slice.
__device__ __forceinline__ void umma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Each thread of the warp writes 4 consecutive 32-bit columns of its TMEM lane (the warp's
// 32 lanes start at taddr's lane field); tmem_wait_st() before the writes are relied on.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint4 v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Arrive once on `bar` when every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Each thread of the warp reads 32 consecutive 32-bit columns of its TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Asynchronous form: issue the load into r, then tmem_wait_ld(r) before reading r. The
// wait names r as in/out operands so the compiler cannot move reads of r above it.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// ------------------------------------------------------------ fast base-2 math
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// softplus in base-2 units: log2(1 + 2^x) = max(x, 0) + log2(1 + 2^-|x|).
__device__ __forceinline__ float softplus2(float x)
{
    return fmaxf(x, 0.0f) + lg2_approx(1.0f + ex2_approx(-fabsf(x)));
}

}  // namespace spa
