// LVQ encoding (quant() of Sec. 2: LVQ, per-vector scalar quantisation around the
// dataset mean) and the FP64 column mean.  One warp per vector.
#include <cuda_fp16.h>

#include "common.cuh"

namespace lv {

constexpr double FIX = 1048576.0;  // 2^20: fixed point of the mean in the build score

// Column mean, deterministic (a fixed summation order that depends on n and dim only).
// Stage 1: block (c, r) sums the rows of chunk r (CM_ROWS rows) for the 4 x 32 columns of tile
// c, each warp a strided subset of the rows (float4 loads along the row when the rows are
// 16-byte aligned) in compensated float32 (Knuth's TwoSum keeps each addition's rounding
// error in a second float32: about 44 significant bits, FP64 being a slow pipe here); the
// warps' (sum, error) pairs are combined in FP64 in order; stage 2 adds the chunks in FP64
// in order and rounds the mean to float32.
constexpr int CM_ROWS = 2048, CM_COLS = 128;

struct Comp {
    float s = 0.f, e = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(s, x);
        const float bb = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(x, bb));
        s = t;
        e = __fadd_rn(e, err);
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};

template <bool VEC>
__global__ void __launch_bounds__(256) column_sum_kernel(const float *__restrict__ X, int64_t n, int dim,
                                                         double *__restrict__ part) {
    __shared__ double red[8][CM_COLS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * CM_COLS + 4 * lane;
    const int64_t r0 = (int64_t)blockIdx.y * CM_ROWS, r1 = min(n, r0 + CM_ROWS);
    Comp a0, a1, a2, a3;
    if (VEC) {
        if (c0 < dim)
            for (int64_t i = r0 + warp; i < r1; i += 8) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(X + i * dim + c0));
                a0.add(v.x);
                a1.add(v.y);
                a2.add(v.z);
                a3.add(v.w);
            }
    } else {
        for (int64_t i = r0 + warp; i < r1; i += 8) {
            const float *row = X + i * dim;
            if (c0 < dim) a0.add(row[c0]);
            if (c0 + 1 < dim) a1.add(row[c0 + 1]);
            if (c0 + 2 < dim) a2.add(row[c0 + 2]);
            if (c0 + 3 < dim) a3.add(row[c0 + 3]);
        }
    }
    red[warp][4 * lane] = a0.value();
    red[warp][4 * lane + 1] = a1.value();
    red[warp][4 * lane + 2] = a2.value();
    red[warp][4 * lane + 3] = a3.value();
    __syncthreads();
    if (threadIdx.x < CM_COLS) {
        const int c = blockIdx.x * CM_COLS + threadIdx.x;
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        if (c < dim) part[(int64_t)blockIdx.y * dim + c] = s;
    }
}

__global__ void column_mean_final_kernel(const double *__restrict__ part, int chunks, int64_t n, int dim,
                                         float *__restrict__ mean) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= dim) return;
    double s = 0.0;
    for (int r = 0; r < chunks; ++r) s += part[(int64_t)r * dim + c];
    mean[c] = (float)(s / (double)n);
}

// LVQ encode with 16-byte loads (dim % 4 == 0, 16-byte aligned rows): one warp per vector, a
// persistent grid; lane l holds the float4 chunks l, l + 32, .. (at most KMAX) of v - mean in
// registers between the min/max pass and the code pass.  The fixed-point mean (mui = mean_i
// 2^20, exact for |mean_i| < 8) and its sums are computed once per block in shared memory.
// Same arithmetic as lvq_encode_kernel, so the records are bit-identical.
template <int BITS, int KMAX, int G>
__global__ void __launch_bounds__(256) lvq_encode_vec_kernel(const float *__restrict__ V, int64_t n, int dim,
                                                             const float *__restrict__ mean, uint8_t *__restrict__ rec,
                                                             int64_t stride, int code_bytes) {
    extern __shared__ uint8_t sm_raw[];
    float *smean = reinterpret_cast<float *>(sm_raw);
    int *smi = reinterpret_cast<int *>(smean + dim);
    __shared__ long long s_mu;
    __shared__ int s_bad;
    if (threadIdx.x == 0) {
        s_mu = 0;
        s_bad = 0;
    }
    __syncthreads();
    long long pmu = 0;
    int bad = 0;
    for (int j = threadIdx.x; j < dim; j += blockDim.x) {
        const float mj = mean[j];
        if (!(fabsf(mj) < 8.0f)) bad = 1;
        const long long mi = __double2ll_rn((double)mj * FIX);
        smean[j] = mj;
        smi[j] = (int)mi;  // only read when every |mean_j| < 8 (then |mi| < 2^23)
        pmu += mi;
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_mu), (unsigned long long)pmu);
    if (bad) atomicOr(&s_bad, 1);
    __syncthreads();
    const bool mean_ok = !s_bad;
    const long long smu = s_mu;
    // G lanes per vector (32: one warp; 16: two vectors per warp for short vectors)
    const int lane = threadIdx.x & (G - 1);
    const int nc = dim >> 2;  // float4 chunks per vector
    const float levels = (float)((1 << BITS) - 1);
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    const int64_t g0 = (int64_t)blockIdx.x * (blockDim.x / G) + (threadIdx.x >> 5) * (32 / G);
    // every lane of a warp stays in the loop while any of its groups has a vector (shuffles)
    for (int64_t w0 = g0; w0 < n; w0 += groups) {
        const int64_t i = w0 + (threadIdx.x & 31) / G;
        const bool act = i < n;
        const int64_t ii = act ? i : w0;
        const float4 *v4 = reinterpret_cast<const float4 *>(V + ii * dim);
        float4 x[KMAX];
        float lo = INFINITY, hi = -INFINITY;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int c = lane + G * k;
            if (c < nc) {
                const float4 v = __ldg(v4 + c);
                const float4 m = *reinterpret_cast<const float4 *>(smean + 4 * c);
                x[k] = make_float4(__fsub_rn(v.x, m.x), __fsub_rn(v.y, m.y), __fsub_rn(v.z, m.z), __fsub_rn(v.w, m.w));
                lo = fminf(fminf(lo, fminf(x[k].x, x[k].y)), fminf(x[k].z, x[k].w));
                hi = fmaxf(fmaxf(hi, fmaxf(x[k].x, x[k].y)), fmaxf(x[k].z, x[k].w));
            }
        }
        for (int o = G / 2; o; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(FULL, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, o));
        }
        const float delta = __fdiv_rn(__fsub_rn(hi, lo), levels);
        uint8_t *r = rec + ii * stride;
        long long msum = 0;
        int csum = 0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int c = lane + G * k;
            if (act && c < nc) {
                const float xs[4] = {x[k].x, x[k].y, x[k].z, x[k].w};
                uint32_t cw[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t q = 0;
                    if (delta > 0.0f) {
                        float t = __fdiv_rn(__fsub_rn(xs[e], lo), delta);
                        float f = floorf(__fadd_rn(t, 0.5f));
                        f = fminf(fmaxf(f, 0.0f), levels);
                        q = (uint32_t)f;
                    }
                    cw[e] = q;
                    msum += (long long)(smi[4 * c + e] * (int)q);
                    csum += (int)q;
                }
                if (BITS == 8)
                    *reinterpret_cast<uint32_t *>(r + 4 * c) = cw[0] | (cw[1] << 8) | (cw[2] << 16) | (cw[3] << 24);
                else
                    *reinterpret_cast<uint16_t *>(r + 2 * c) =
                        (uint16_t)(cw[0] | (cw[1] << 4) | (cw[2] << 8) | (cw[3] << 12));
            }
        }
        // zero the code padding (whole 16-bit units: the code bytes end on an even offset)
        const int used = BITS == 8 ? dim : dim / 2;
        if (act)
            for (int b = used + 2 * lane; b < code_bytes; b += 2 * G) *reinterpret_cast<uint16_t *>(r + b) = 0;
        for (int o = G / 2; o; o >>= 1) {
            msum += __shfl_xor_sync(FULL, msum, o);
            csum += __shfl_xor_sync(FULL, csum, o);
        }
        if (act && lane == 0) {
            const float inv = (float)(1.0 / FIX);
            float mu1 = __fmul_rn(__ll2float_rn(smu), inv);
            float mf = __fmul_rn(__ll2float_rn(msum), inv);
            float Gt = __fadd_rn(__fmul_rn(lo, mu1), __fmul_rn(delta, mf));
            float Ht = __fmul_rn(delta, __int2float_rn(csum));
            if (!mean_ok) Gt = Ht = __int_as_float(0x7fc00000);
            *reinterpret_cast<float4 *>(r + code_bytes) = make_float4(delta, lo, Gt, Ht);
        }
        if (act)
            for (int64_t t = code_bytes + 16 + 4 * lane; t < stride; t += 4 * G) *reinterpret_cast<uint32_t *>(r + t) = 0u;
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
    if (n <= 0 || dim <= 0) return LV_OK;
    const int64_t chunks = (n + CM_ROWS - 1) / CM_ROWS;
    if (chunks >= 65536) return fail(LV_ERR_ARG, "column_mean: more than 2^27 rows");
    double *part = nullptr;
    int rc = tmp_alloc((void **)&part, sizeof(double) * (size_t)chunks * dim, st);
    if (rc) return rc;
    dim3 grd((unsigned)((dim + CM_COLS - 1) / CM_COLS), (unsigned)chunks);
    if (dim % 4 == 0 && ((uintptr_t)X & 15) == 0)
        column_sum_kernel<true><<<grd, 256, 0, st>>>(X, n, dim, part);
    else
        column_sum_kernel<false><<<grd, 256, 0, st>>>(X, n, dim, part);
    column_mean_final_kernel<<<(dim + 127) / 128, 128, 0, st>>>(part, (int)chunks, n, dim, mean);
    cudaError_t e = cudaGetLastError();
    tmp_free(part, st);
    if (e != cudaSuccess) return cuda_fail(e, "column mean kernels");
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
    const int nc = dim / 4;
    if (dim % 4 == 0 && ((uintptr_t)V & 15) == 0 && nc <= 32 * 8) {
        int dev = 0, sms = 0;
        LV_CUDA(cudaGetDevice(&dev));
        LV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const size_t smem = (size_t)dim * 8;
        const unsigned grid = (unsigned)std::min<int64_t>(blocks, (int64_t)sms * 8);
        auto go = [&](auto kern) -> int {
            if (smem > 48 * 1024) LV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<grid, wpb * 32, smem, st>>>(V, n, dim, mean, rec, g.stride, g.code_bytes);
            LV_CHECK_LAUNCH("lvq_encode_vec_kernel");
            return LV_OK;
        };
        // short vectors (dim <= 256): two per warp, 16 lanes each
        if (bits == 8) {
            if (nc <= 64) return go(lvq_encode_vec_kernel<8, 4, 16>);
            if (nc <= 128) return go(lvq_encode_vec_kernel<8, 4, 32>);
            return go(lvq_encode_vec_kernel<8, 8, 32>);
        }
        if (nc <= 64) return go(lvq_encode_vec_kernel<4, 4, 16>);
        if (nc <= 128) return go(lvq_encode_vec_kernel<4, 4, 32>);
        return go(lvq_encode_vec_kernel<4, 8, 32>);
    }
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
