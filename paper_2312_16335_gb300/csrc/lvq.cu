// LVQ encoding (quant() of Sec. 2: LVQ, per-vector scalar quantisation around the
// dataset mean) and the FP64 column mean.  One warp per vector.
#include <cuda_fp16.h>

#include "common.cuh"

namespace lv {

constexpr double FIX = 1048576.0;  // 2^20: fixed point of the mean in the build score

// Column mean: each block owns 32 columns and sums rows in a fixed order (per-thread
// strided partial sums reduced in a fixed tree) so the result is deterministic.
__global__ void column_mean_kernel(const float *__restrict__ X, int64_t n, int dim,
                                   float *__restrict__ mean) {
    __shared__ double part[8][33];
    int col = blockIdx.x * 32 + threadIdx.x;
    double acc = 0.0;
    if (col < dim)
        for (int64_t i = threadIdx.y; i < n; i += 8) acc += (double)X[i * dim + col];
    part[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && col < dim) {
        double s = 0.0;
        for (int t = 0; t < 8; ++t) s += part[t][threadIdx.x];
        mean[col] = (float)(s / (double)n);
    }
}

template <int BITS>
__global__ void lvq_encode_kernel(const float *__restrict__ V, int64_t n, int dim,
                                  const float *__restrict__ mean, uint8_t *__restrict__ rec,
                                  int64_t stride, int code_bytes) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const float *v = V + i * dim;
    // pass 1: min / max of v - mean
    float lo = INFINITY, hi = -INFINITY;
    int64_t smu = 0, smu2 = 0;
    bool mean_ok = true;
    for (int j = lane; j < dim; j += 32) {
        float x = __fsub_rn(v[j], mean[j]);
        lo = fminf(lo, x);
        hi = fmaxf(hi, x);
        float mj = mean[j];
        if (!(fabsf(mj) < 8.0f)) mean_ok = false;
        long long mi = __double2ll_rn((double)mj * FIX);
        smu += mi;
        smu2 += mi * mi;
    }
    for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(FULL, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, o));
        smu += __shfl_xor_sync(FULL, smu, o);
        smu2 += __shfl_xor_sync(FULL, smu2, o);
    }
    mean_ok = __all_sync(FULL, mean_ok);
    const float levels = (float)((1 << BITS) - 1);
    const float delta = __fdiv_rn(__fsub_rn(hi, lo), levels);
    uint8_t *r = rec + i * stride;
    int64_t msum = 0, csum = 0;
    // pass 2: codes
    if (BITS == 8) {
        for (int j = lane; j < code_bytes; j += 32) {
            uint32_t c = 0;
            if (j < dim) {
                float x = __fsub_rn(v[j], mean[j]);
                if (delta > 0.0f) {
                    float t = __fdiv_rn(__fsub_rn(x, lo), delta);
                    float f = floorf(__fadd_rn(t, 0.5f));
                    f = fminf(fmaxf(f, 0.0f), levels);
                    c = (uint32_t)f;
                }
                msum += (long long)__double2ll_rn((double)mean[j] * FIX) * (long long)c;
                csum += c;
            }
            r[j] = (uint8_t)c;
        }
    } else {
        for (int b = lane; b < code_bytes; b += 32) {
            uint32_t pk = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int j = 2 * b + h;
                uint32_t c = 0;
                if (j < dim) {
                    float x = __fsub_rn(v[j], mean[j]);
                    if (delta > 0.0f) {
                        float t = __fdiv_rn(__fsub_rn(x, lo), delta);
                        float f = floorf(__fadd_rn(t, 0.5f));
                        f = fminf(fmaxf(f, 0.0f), levels);
                        c = (uint32_t)f;
                    }
                    msum += (long long)__double2ll_rn((double)mean[j] * FIX) * (long long)c;
                    csum += c;
                }
                pk |= c << (4 * h);
            }
            r[b] = (uint8_t)pk;
        }
    }
    for (int o = 16; o; o >>= 1) {
        msum += __shfl_xor_sync(FULL, msum, o);
        csum += __shfl_xor_sync(FULL, csum, o);
    }
    if (lane == 0) {
        const float inv = (float)(1.0 / FIX);
        float mu1 = __fmul_rn(__ll2float_rn(smu), inv);
        float mf = __fmul_rn(__ll2float_rn(msum), inv);
        float G = __fadd_rn(__fmul_rn(lo, mu1), __fmul_rn(delta, mf));
        float H = __fmul_rn(delta, __ll2float_rn(csum));
        if (!mean_ok) G = H = __int_as_float(0x7fc00000);
        float4 cst = make_float4(delta, lo, G, H);
        *reinterpret_cast<float4 *>(r + code_bytes) = cst;
        // zero the tail padding of the record
        for (int64_t t = code_bytes + 16; t < stride; t += 4) *reinterpret_cast<uint32_t *>(r + t) = 0u;
    }
}

__global__ void fp32_record_kernel(const float *__restrict__ X, int64_t n, int dim,
                                   uint8_t *__restrict__ rec, int64_t stride) {
    const int64_t i = blockIdx.x;
    float *r = reinterpret_cast<float *>(rec + i * stride);
    const int nw = (int)(stride / 4);
    for (int j = threadIdx.x; j < nw; j += blockDim.x) r[j] = j < dim ? X[i * dim + j] : 0.0f;
}

// sum mui^2 * 2^-40 as float (the build score's constant term)
__global__ void mu2_kernel(const float *__restrict__ mean, int dim, float *__restrict__ out) {
    int64_t s = 0;
    for (int j = threadIdx.x; j < dim; j += 32) {
        long long mi = __double2ll_rn((double)mean[j] * FIX);
        s += mi * mi;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (threadIdx.x == 0) *out = __fmul_rn(__ll2float_rn(s), (float)(1.0 / (FIX * FIX)));
}

int launch_column_mean(const float *X, int64_t n, int dim, float *mean, cudaStream_t st) {
    dim3 blk(32, 8), grd((dim + 31) / 32);
    column_mean_kernel<<<grd, blk, 0, st>>>(X, n, dim, mean);
    LV_CHECK_LAUNCH("column_mean_kernel");
    return LV_OK;
}

// FP16 secondary records: x rounded to IEEE half (round to nearest even), the padding zeroed.
__global__ void fp16_record_kernel(const float *__restrict__ X, int64_t n, int dim, int64_t stride,
                                   uint8_t *__restrict__ out) {
    const int64_t halves = stride / 2;
    const int64_t total = n * halves;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / halves, j = t - i * halves;
        const __half h = j < dim ? __float2half_rn(X[i * dim + j]) : __float2half_rn(0.f);
        reinterpret_cast<__half *>(out + i * stride)[j] = h;
    }
}

int launch_fp16_records(const float *X, int64_t n, int dim, int64_t stride, uint8_t *out, cudaStream_t st) {
    if (n == 0) return LV_OK;
    fp16_record_kernel<<<1024, 256, 0, st>>>(X, n, dim, stride, out);
    LV_CHECK_LAUNCH("fp16_record_kernel");
    return LV_OK;
}

// L2 index: the second constants chunk {N, ||x||^2, 0, 0} of LVQ records.  N = <y, y> by the build
// score's own arithmetic (the sum of squared codes and the record's constants, see leanvec.h); the
// squared norm defaults to N until the original vectors set it (set_sqnorm_kernel).  One warp per
// record.
template <int BITS>
__global__ void lvq_self_norm_kernel(uint8_t *__restrict__ rec, int64_t n, int64_t stride, int code_bytes, int dim,
                                     float mu2) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    uint8_t *r = rec + i * stride;
    int P = 0;
    for (int b = lane; b < code_bytes; b += 32) {
        const uint32_t v = r[b];
        if (BITS == 8)
            P += (int)(v * v);
        else
            P += (int)((v & 15u) * (v & 15u) + (v >> 4) * (v >> 4));
    }
    for (int o = 16; o; o >>= 1) P += __shfl_xor_sync(FULL, P, o);
    if (lane == 0) {
        const float4 k = *reinterpret_cast<const float4 *>(r + code_bytes);
        const float N = build_pair_score(mu2, (float)dim, k.x, k.y, k.z, k.w, k.x, k.y, k.z, k.w, P);
        *reinterpret_cast<float4 *>(r + code_bytes + 16) = make_float4(N, N, 0.f, 0.f);
    }
}

// ||x_i||^2 of the original vectors (squares exact in FP64, FP64 sum, rounded to float32) into the
// float at byte offset `off` of every record.  One warp per vector.
__global__ void set_sqnorm_kernel(uint8_t *__restrict__ rec, int64_t n, int64_t stride, int off,
                                  const float *__restrict__ X, int D) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    double s = 0.0;
    for (int j = lane; j < D; j += 32) {
        const double x = (double)X[i * (int64_t)D + j];
        s += x * x;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) *reinterpret_cast<float *>(rec + i * stride + off) = (float)s;
}

int launch_lvq_self_norms(uint8_t *rec, int64_t n, int dim, int bits, int64_t stride, int code_bytes, float mu2,
                          cudaStream_t st) {
    if (n == 0) return LV_OK;
    const int wpb = 8;
    const int64_t blocks = (n + wpb - 1) / wpb;
    if (bits == 8)
        lvq_self_norm_kernel<8><<<(unsigned)blocks, wpb * 32, 0, st>>>(rec, n, stride, code_bytes, dim, mu2);
    else
        lvq_self_norm_kernel<4><<<(unsigned)blocks, wpb * 32, 0, st>>>(rec, n, stride, code_bytes, dim, mu2);
    LV_CHECK_LAUNCH("lvq_self_norm_kernel");
    return LV_OK;
}

int launch_set_sqnorms(uint8_t *rec, int64_t n, int64_t stride, int off, const float *X, int D, cudaStream_t st) {
    if (n == 0) return LV_OK;
    const int wpb = 8;
    set_sqnorm_kernel<<<(unsigned)((n + wpb - 1) / wpb), wpb * 32, 0, st>>>(rec, n, stride, off, X, D);
    LV_CHECK_LAUNCH("set_sqnorm_kernel");
    return LV_OK;
}

int launch_lvq_encode(const float *V, int64_t n, int dim, const float *mean, int bits,
                      uint8_t *rec, cudaStream_t st, int metric) {
    RecGeom g;
    if (!rec_geom(dim, bits, g, metric) || bits == 32) return fail(LV_ERR_ARG, "lvq_encode: bits must be 4 or 8");
    if (n == 0) return LV_OK;
    const int wpb = 8;
    int64_t blocks = (n + wpb - 1) / wpb;
    if (bits == 8)
        lvq_encode_kernel<8><<<(unsigned)blocks, wpb * 32, 0, st>>>(V, n, dim, mean, rec, g.stride, g.code_bytes);
    else
        lvq_encode_kernel<4><<<(unsigned)blocks, wpb * 32, 0, st>>>(V, n, dim, mean, rec, g.stride, g.code_bytes);
    LV_CHECK_LAUNCH("lvq_encode_kernel");
    return LV_OK;
}

int launch_fp32_records(const float *X, int64_t n, int dim, uint8_t *rec, int64_t stride, cudaStream_t st) {
    if (n == 0) return LV_OK;
    fp32_record_kernel<<<(unsigned)n, 128, 0, st>>>(X, n, dim, rec, stride);
    LV_CHECK_LAUNCH("fp32_record_kernel");
    return LV_OK;
}

int launch_mu2(const float *mean, int dim, float *out, cudaStream_t st) {
    mu2_kernel<<<1, 32, 0, st>>>(mean, dim, out);
    LV_CHECK_LAUNCH("mu2_kernel");
    return LV_OK;
}

}  // namespace lv
