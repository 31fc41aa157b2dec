// k_loglik_simt.cu -- the plain FP32 path: the same log-likelihood on CUDA cores (FFMA).
//
// eta = X beta with the standardised FP32 X (Section 3) and FP32 accumulation, then
// softplus(eta) = max(eta, 0) + log1p(exp(-|eta|)) with the accurate FP32 functions, summed
// per particle over each 64-individual tile (the linear half sum_i y_i eta_i = beta . X^T y
// is a p-length dot product the move kernels form). The gradient path (mode 1) keeps the
// full y eta - softplus(eta) per tile for its log-likelihood output. This is the comparator the split-BF16
// tensor-core path is measured against; it is also the gradient (adjoint) kernel pair
// behind spa_grad: grad l = X^T (y - logit^{-1}(eta)).
#include "spa_device.cuh"
#include "spa_internal.h"

namespace spa {

namespace {

constexpr int TP = 64;  // particles per CTA tile
constexpr int TI = SIMT_TILE_N;  // individuals per CTA tile
constexpr int TK = 16;  // k-chunk

__device__ __forceinline__ float softplus_acc(float x) { return fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x))); }

// 256 threads = 16 x 16; thread (ty, tx) owns particles ty*4..+3 and individuals tx*4..+3.
// mode 0: partial = -sum over the tile of softplus(eta); mode 1: partial = sum over the tile
// of y eta - softplus(eta), and eta stored to eta_out [N][n].
template <int MODE>
__global__ void __launch_bounds__(256) k_eta_tile(const float* __restrict__ B, const float* __restrict__ Xf,
                                                  const uint8_t* __restrict__ y, int64_t N, int64_t n, int p,
                                                  float* __restrict__ partial, int64_t N_pad, float* __restrict__ eta_out)
{
    __shared__ float Bs[TK][TP + 4];
    __shared__ float Xs[TK][TI + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * TP;  // particle tile
    const int64_t r0 = (int64_t)blockIdx.y * TI;  // individual tile
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
    for (int k0 = 0; k0 < p; k0 += TK) {
        for (int e = threadIdx.x; e < TP * TK; e += 256) {
            const int r = e / TK, kk = e - r * TK;
            const int64_t gi = i0 + r;
            const int gk = k0 + kk;
            Bs[kk][r] = (gi < N && gk < p) ? B[gi * p + gk] : 0.0f;
            const int64_t gr = r0 + r;
            Xs[kk][r] = (gr < n && gk < p) ? Xf[gr * p + gk] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = Bs[kk][ty * 4 + q];
                b[q] = Xs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int z = 0; z < 4; ++z) acc[x][z] = fmaf(a[x], b[z], acc[x][z]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int64_t gi = i0 + ty * 4 + x;
        float s = 0.0f;
#pragma unroll
        for (int z = 0; z < 4; ++z) {
            const int64_t gr = r0 + tx * 4 + z;
            if (gr < n) {
                const float e = acc[x][z];
                if (MODE == 0) {
                    s -= softplus_acc(e);
                } else {
                    s += (y[gr] ? e : 0.0f) - softplus_acc(e);
                    if (gi < N) eta_out[gi * n + gr] = e;
                }
            }
        }
        // reduce over the 16 threads (tx) that share these particles: lanes differ in bits 0..3
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (tx == 0 && gi < N) partial[(int64_t)blockIdx.y * N_pad + gi] = s;
    }
}

// grad[i, j] = sum_r x_rj (y_r - logit^{-1}(eta[i, r])) (+ prior gradient at scale c).
__global__ void __launch_bounds__(256) k_grad_tile(const float* __restrict__ eta, const float* __restrict__ Xf,
                                                   const uint8_t* __restrict__ y, const float* __restrict__ B, int64_t N,
                                                   int64_t n, int p, float* __restrict__ grad, PriorArgs pr, double c)
{
    __shared__ float Rs[TK][TP + 4];  // residuals [individual][particle]
    __shared__ float Xs[TK][TP + 4];  // genotypes [individual][marker]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * TP;  // particle tile
    const int j0 = blockIdx.y * TP;               // marker tile
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
    for (int64_t r0 = 0; r0 < n; r0 += TK) {
        for (int e = threadIdx.x; e < TP * TK; e += 256) {
            const int q = e / TK, kk = e - q * TK;
            const int64_t gr = r0 + kk;
            const int64_t gi = i0 + q;
            float rv = 0.0f;
            if (gr < n && gi < N) {
                const float et = eta[gi * n + gr];
                rv = (y[gr] ? 1.0f : 0.0f) - 1.0f / (1.0f + expf(-et));
            }
            Rs[kk][q] = rv;
            const int gj = j0 + q;
            Xs[kk][q] = (gr < n && gj < p) ? Xf[gr * p + gj] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = Rs[kk][ty * 4 + q];
                b[q] = Xs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int z = 0; z < 4; ++z) acc[x][z] = fmaf(a[x], b[z], acc[x][z]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int64_t gi = i0 + ty * 4 + x;
#pragma unroll
        for (int z = 0; z < 4; ++z) {
            const int gj = j0 + tx * 4 + z;
            if (gi < N && gj < p) {
                float g = acc[x][z];
                if (c > 0.0) {
                    const float b = B[gi * p + gj];
                    const float sg = (b > 0.0f) ? 1.0f : ((b < 0.0f) ? -1.0f : 0.0f);
                    g += pr.de ? (float)(-sg / c) : (float)(-((double)pr.a + 1.0) * sg / ((double)pr.a * c + fabs((double)b)));
                }
                grad[gi * p + gj] = g;
            }
        }
    }
}

__global__ void k_sum_partials(const float* __restrict__ partial, int n_parts, int64_t N_pad, int64_t N,
                               double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int k = 0; k < n_parts; ++k) s += (double)partial[(int64_t)k * N_pad + i];
    out[i] = s;
}

}  // namespace

cudaError_t launch_loglik_simt(const float* beta_p, const float* Xf, const uint8_t* y, int64_t N, int64_t n, int p,
                               float* partial, int64_t N_pad, cudaStream_t st)
{
    dim3 grid((unsigned)((N + TP - 1) / TP), (unsigned)((n + TI - 1) / TI));
    k_eta_tile<0><<<grid, 256, 0, st>>>(beta_p, Xf, y, N, n, p, partial, N_pad, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_grad_simt(const float* B, const float* Xf, const uint8_t* y, int64_t N, int64_t n, int p,
                             float* eta_scratch, float* grad, double* ll, PriorArgs pr, double c, cudaStream_t st)
{
    // the log-likelihood partials live in the tail of the eta scratch (allocated N*n + n_tiles*N)
    const int n_tiles = (int)((n + TI - 1) / TI);
    float* partial = eta_scratch + N * n;
    dim3 g1((unsigned)((N + TP - 1) / TP), (unsigned)n_tiles);
    k_eta_tile<1><<<g1, 256, 0, st>>>(B, Xf, y, N, n, p, partial, N, eta_scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2((unsigned)((N + TP - 1) / TP), (unsigned)((p + TP - 1) / TP));
    k_grad_tile<<<g2, 256, 0, st>>>(eta_scratch, Xf, y, B, N, n, p, grad, pr, c);
    e = cudaGetLastError();
    if (e != cudaSuccess || !ll) return e;
    k_sum_partials<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(partial, n_tiles, N, N, ll);
    return cudaGetLastError();
}

}  // namespace spa
