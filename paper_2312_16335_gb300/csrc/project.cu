// Projection GEMM on the CUDA cores (float32): Y = X P^T (Eq. 1: q -> A q, x -> B x).
#include "common.cuh"

namespace lv {

constexpr int PT_M = 64, PT_N = 64, PT_K = 32;

// 256 threads, each computes a 4 x 4 block of the 64 x 64 output tile.
__global__ void __launch_bounds__(256) project_fp32_kernel(const float *__restrict__ X, int64_t n, int D,
                                                           const float *__restrict__ P, int d,
                                                           float *__restrict__ Y, int ldy) {
    __shared__ __align__(16) float As[PT_K][PT_M + 4];
    __shared__ __align__(16) float Bs[PT_K][PT_N + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * PT_M;
    const int col0 = blockIdx.y * PT_N;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < D; k0 += PT_K) {
        for (int t = threadIdx.x; t < PT_M * PT_K; t += 256) {
            int r = t / PT_K, c = t % PT_K;
            int64_t gr = row0 + r;
            int gc = k0 + c;
            As[c][r] = (gr < n && gc < D) ? X[gr * D + gc] : 0.0f;
            int pr = col0 + r;
            Bs[c][r] = (pr < d && gc < D) ? P[(int64_t)pr * D + gc] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < PT_K; ++kk) {
            // one 16-byte shared load per operand (rows of 68 floats keep them aligned)
            const float4 a4 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 b4 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t r = row0 + ty * 4 + i;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int c = col0 + tx * 4 + j;
            if (c < ldy) Y[r * ldy + c] = c < d ? acc[i][j] : 0.0f;
        }
    }
}

// Copy rows of X (n x D) into Y (n x ldy), zero-padded (identity projection).
__global__ void pad_rows_kernel(const float *__restrict__ X, int64_t n, int D, float *__restrict__ Y, int ldy) {
    int64_t r = blockIdx.x;
    for (int c = threadIdx.x; c < ldy; c += blockDim.x) Y[r * ldy + c] = c < D ? X[r * D + c] : 0.0f;
}

int launch_project_fp32(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy,
                        cudaStream_t st) {
    if (n == 0) return LV_OK;
    dim3 grd((unsigned)((n + PT_M - 1) / PT_M), (unsigned)((ldy + PT_N - 1) / PT_N));
    project_fp32_kernel<<<grd, 256, 0, st>>>(X, n, D, P, d, Y, ldy);
    LV_CHECK_LAUNCH("project_fp32_kernel");
    return LV_OK;
}

int launch_pad_rows(const float *X, int64_t n, int D, float *Y, int ldy, cudaStream_t st) {
    if (n == 0) return LV_OK;
    pad_rows_kernel<<<(unsigned)n, 128, 0, st>>>(X, n, D, Y, ldy);
    LV_CHECK_LAUNCH("pad_rows_kernel");
    return LV_OK;
}


}  // namespace lv
