// k_store.cu -- the genotype store: column statistics and GEMM operands.
//
// Section 3 standardises the columns of X to mean zero and unit standard deviation;
// x_ij = (g_ij - m_j)/s_j with the population sd. The store keeps G exact: the BF16
// operand holds g in {0,1,2} (exact) and a column of ones, so that
//   eta_i = sum_j x_ij beta_j = sum_j g_ij bt_j + o,  bt_j = beta_j/s_j, o = -sum_j m_j bt_j,
// is a plain contraction of exact genotypes. Column sums are exact integer atomics, so
// the statistics do not depend on the order of accumulation.
#include "spa_device.cuh"
#include "spa_internal.h"

namespace spa {

namespace {

constexpr int SUM_ROWS = 8;     // threadIdx.y extent
constexpr int SUM_SPLITS = 16;  // row splits (gridDim.y)

__global__ void k_store_sums(const int8_t* __restrict__ G, const uint8_t* __restrict__ y, int64_t n, int64_t p,
                             unsigned long long* __restrict__ sums, uint32_t* __restrict__ err)
{
    __shared__ unsigned long long red[3][SUM_ROWS][32];
    __shared__ unsigned long long ycount[SUM_ROWS][32];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t j = (int64_t)blockIdx.x * 32 + tx;
    unsigned long long s1 = 0, s2 = 0, sy = 0, ny = 0;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.y * SUM_ROWS + ty; i < n; i += (int64_t)SUM_ROWS * gridDim.y) {
        const uint8_t yi = y[i];
        if (yi > 1) bad = true;
        if (blockIdx.x == 0 && tx == 0) ny += yi;
        if (j < p) {
            const int g = G[i * p + j];
            if (g < 0 || g > 2) bad = true;
            s1 += (unsigned)g;
            s2 += (unsigned)(g * g);
            sy += (unsigned)(g * (int)(yi & 1u));
        }
    }
    if (bad) atomicOr(err, DERR_INPUT);
    red[0][ty][tx] = s1;
    red[1][ty][tx] = s2;
    red[2][ty][tx] = sy;
    ycount[ty][tx] = ny;
    __syncthreads();
    if (ty == 0) {
        for (int r = 1; r < SUM_ROWS; ++r) {
            s1 += red[0][r][tx];
            s2 += red[1][r][tx];
            sy += red[2][r][tx];
            ny += ycount[r][tx];
        }
        if (j < p) {
            atomicAdd(&sums[j], s1);
            atomicAdd(&sums[p + j], s2);
            atomicAdd(&sums[2 * p + j], sy);
        }
        if (blockIdx.x == 0 && tx == 0) atomicAdd(&sums[3 * p], ny);
    }
}

// colf[0..p) = 1/s_j, colf[p..2p) = v_j and colf[2p..3p) = v_j log2(e) in FP32, where
// v = X^T y is the coefficient vector of the linear half of the log-likelihood,
// sum_i y_i eta_i = beta . v.
__global__ void k_store_stats(int64_t n, int64_t p, const unsigned long long* __restrict__ sums,
                              double* __restrict__ mean, double* __restrict__ sd, double* __restrict__ v,
                              float* __restrict__ l2e_over_s, float* __restrict__ mean_f, float* __restrict__ colf,
                              uint32_t* __restrict__ err)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p) return;
    const long long S1 = (long long)sums[j], S2 = (long long)sums[p + j], SY = (long long)sums[2 * p + j];
    const long long NY = (long long)sums[3 * p];
    const long long nn = (long long)n;
    // n^2 var = n S2 - S1^2 and n sum_i y_i (g_ij - m_j) = n SY - NY S1, both exact integers.
    const long long var_num = nn * S2 - S1 * S1;
    const double m = (double)S1 / (double)nn;
    const double s = sqrt((double)var_num) / (double)nn;
    if (var_num <= 0) {
        atomicOr(err, DERR_INPUT);
        return;
    }
    mean[j] = m;
    sd[j] = s;
    const double vj = (double)(nn * SY - NY * S1) / ((double)nn * s);
    v[j] = vj;
    l2e_over_s[j] = (float)(LOG2E / s);
    mean_f[j] = (float)m;
    colf[j] = (float)(1.0 / s);
    colf[p + j] = (float)vj;
    colf[2 * p + j] = (float)(vj * LOG2E);
}

// BF16 operand rows (g_i0..g_i,p-1, 1, 0 ... 0) of width Kp and the FP32 standardised X.
__global__ void k_store_pack(const int8_t* __restrict__ G, int64_t n, int64_t p, int Kp,
                             const double* __restrict__ mean, const double* __restrict__ sd,
                             __nv_bfloat16* __restrict__ Gbf, float* __restrict__ Xf)
{
    const int64_t total = n * (int64_t)Kp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / Kp;
        const int64_t j = e - i * Kp;
        float g = 0.0f;
        if (j < p) {
            g = (float)G[i * p + j];
            Xf[i * p + j] = (float)(((double)g - mean[j]) / sd[j]);
        } else if (j == p) {
            g = 1.0f;
        }
        Gbf[e] = __float2bfloat16_rn(g);
    }
}

// G^T as BF16 [p][n_r] (zero beyond n) for the adjoint, and y as floats.
__global__ void k_store_pack_t(const int8_t* __restrict__ G, const uint8_t* __restrict__ y, int64_t n, int64_t p,
                               int64_t n_r, __nv_bfloat16* __restrict__ GT, float* __restrict__ yv)
{
    const int64_t total = p * n_r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / n_r;
        const int64_t i = e - j * n_r;
        GT[e] = __float2bfloat16_rn(i < n ? (float)G[i * p + j] : 0.0f);
        if (j == 0 && i < n) yv[i] = (float)y[i];
    }
}

// XT2[j][i] = x_ij log2(e): the standardised genotypes marker-major, for the
// single-coordinate kernel's coalesced column reads. 32 x 32 tiles through shared memory.
__global__ void k_store_xt2(const float* __restrict__ Xf, int64_t n, int64_t p, float* __restrict__ XT2)
{
    __shared__ float tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r, j = j0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < n && j < p) ? Xf[i * p + j] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t j = j0 + r, i = i0 + threadIdx.x;
        if (i < n && j < p) XT2[j * n + i] = (float)((double)tile[threadIdx.x][r] * LOG2E);
    }
}

__global__ void k_store_ybits(const uint8_t* __restrict__ y, int64_t n, int64_t words, uint32_t* __restrict__ ybits)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= words) return;
    uint32_t v = 0u;
    for (int k = 0; k < 32; ++k) {
        const int64_t i = w * 32 + k;
        if (i < n && y[i]) v |= 1u << k;
    }
    ybits[w] = v;
}

}  // namespace

cudaError_t launch_store_xt2(const float* Xf, int64_t n, int64_t p, float* XT2, cudaStream_t st)
{
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((p + 31) / 32));
    k_store_xt2<<<grid, dim3(32, 8), 0, st>>>(Xf, n, p, XT2);
    return cudaGetLastError();
}

cudaError_t launch_store_ybits(const uint8_t* y, int64_t n, int64_t words, uint32_t* ybits, cudaStream_t st)
{
    k_store_ybits<<<(unsigned)((words + 127) / 128), 128, 0, st>>>(y, n, words, ybits);
    return cudaGetLastError();
}

cudaError_t launch_store_pack_t(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, int64_t n_r,
                                __nv_bfloat16* GT, float* yv, cudaStream_t st)
{
    const int64_t total = p * n_r;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    k_store_pack_t<<<blocks, 256, 0, st>>>(G, y, n, p, n_r, GT, yv);
    return cudaGetLastError();
}

cudaError_t launch_store_sums(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, unsigned long long* sums,
                              uint32_t* err, cudaStream_t st)
{
    dim3 block(32, SUM_ROWS);
    dim3 grid((unsigned)((p + 31) / 32), SUM_SPLITS);
    k_store_sums<<<grid, block, 0, st>>>(G, y, n, p, sums, err);
    return cudaGetLastError();
}

cudaError_t launch_store_finish(const int8_t* G, int64_t n, int64_t p, int Kp, const unsigned long long* sums,
                                double* mean, double* sd, double* v, float* l2e_over_s, float* mean_f, float* colf,
                                __nv_bfloat16* Gbf, float* Xf, uint32_t* err, cudaStream_t st)
{
    k_store_stats<<<(unsigned)((p + 127) / 128), 128, 0, st>>>(n, p, sums, mean, sd, v, l2e_over_s, mean_f, colf, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = n * (int64_t)Kp;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    k_store_pack<<<blocks, 256, 0, st>>>(G, n, p, Kp, mean, sd, Gbf, Xf);
    return cudaGetLastError();
}

}  // namespace spa
