// Learning the projections: second moments K = sum x x^T (Sec. 2.2 "Efficiency"),
// an FP64 symmetric eigensolver (cyclic Jacobi rotations, round-robin pair order so
// that the D/2 rotations of a round are independent), and LeanVec-ID (Sec. 2.1:
// A = B = the d leading eigenvectors of K_X).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace lv {

// ------------------------------------------------------------ Gram matrix (FP32)
constexpr int GT = 64, GK = 32;

// K[a][b] = sum_i X[i][a] X[i][b]; 256 threads, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) gram_fp32_kernel(const float *__restrict__ X, int64_t n, int D,
                                                        float *__restrict__ K) {
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int a0 = blockIdx.y * GT, b0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int64_t i0 = 0; i0 < n; i0 += GK) {
        for (int t = threadIdx.x; t < GK * GT; t += 256) {
            const int r = t / GT, c = t % GT;
            const int64_t gi = i0 + r;
            As[r][c] = (gi < n && a0 + c < D) ? X[gi * D + a0 + c] : 0.0f;
            Bs[r][c] = (gi < n && b0 + c < D) ? X[gi * D + b0 + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[kk][ty * 4 + u];
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tx * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = a0 + ty * 4 + u;
        if (r >= D) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = b0 + tx * 4 + v;
            if (c < D) K[(int64_t)r * D + c] = acc[u][v];
        }
    }
}

int launch_gram_fp32(const float *X, int64_t n, int D, float *K, cudaStream_t st) {
    dim3 grd((D + GT - 1) / GT, (D + GT - 1) / GT);
    gram_fp32_kernel<<<grd, 256, 0, st>>>(X, n, D, K);
    LV_CHECK_LAUNCH("gram_fp32_kernel");
    return LV_OK;
}

// ---------------------------------------------------------- FP64 Jacobi eigh
// Round r of the round-robin schedule on Dp (even) indices pairs slot i:
//   i = 0: (r, Dp - 1);  i > 0: ((r + i) mod (Dp - 1), (r - i) mod (Dp - 1)).
__device__ __forceinline__ void rr_pair(int r, int i, int Dp, int &p, int &q) {
    const int m = Dp - 1;
    if (i == 0) {
        p = r % m;
        q = m;
    } else {
        p = (r + i) % m;
        q = ((r - i) % m + m) % m;
    }
    if (p > q) {
        int t = p;
        p = q;
        q = t;
    }
}

// Rotation J (J_pp = J_qq = c, J_pq = s, J_qp = -s) that zeroes A'_pq of J^T A J.
__global__ void jacobi_rot_kernel(const double *__restrict__ A, int Dp, int r, double2 *__restrict__ cs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Dp / 2) return;
    int p, q;
    rr_pair(r, i, Dp, p, q);
    const double apq = A[(int64_t)p * Dp + q];
    double c = 1.0, s = 0.0;
    const double app = A[(int64_t)p * Dp + p], aqq = A[(int64_t)q * Dp + q];
    if (apq != 0.0 && fabs(apq) > 1e-300) {
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        c = 1.0 / sqrt(t * t + 1.0);
        s = t * c;
    }
    cs[i] = make_double2(c, s);
}

// rows p, q of A  <-  (c A_p - s A_q, s A_p + c A_q)   for every pair of the round
__global__ void jacobi_rows_kernel(double *__restrict__ A, int Dp, int r, const double2 *__restrict__ cs) {
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Dp) return;
    int p, q;
    rr_pair(r, i, Dp, p, q);
    const double2 k = cs[i];
    const double a = A[(int64_t)p * Dp + j], b = A[(int64_t)q * Dp + j];
    A[(int64_t)p * Dp + j] = k.x * a - k.y * b;
    A[(int64_t)q * Dp + j] = k.y * a + k.x * b;
}

// columns p, q of A and V  <-  (c X_p - s X_q, s X_p + c X_q)
__global__ void jacobi_cols_kernel(double *__restrict__ A, double *__restrict__ V, int Dp, int r,
                                   const double2 *__restrict__ cs) {
    const int i = blockIdx.y;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= Dp) return;
    int p, q;
    rr_pair(r, i, Dp, p, q);
    const double2 k = cs[i];
    double *ar = A + (int64_t)row * Dp;
    double a = ar[p], b = ar[q];
    ar[p] = k.x * a - k.y * b;
    ar[q] = k.y * a + k.x * b;
    double *vr = V + (int64_t)row * Dp;
    a = vr[p];
    b = vr[q];
    vr[p] = k.x * a - k.y * b;
    vr[q] = k.y * a + k.x * b;
}

// One whole round in one kernel: block i owns the pair (p, q) = rr_pair(r, i) and writes rows
// p and q of J^T A J (its own rotation mixes the two rows, then every pair's rotation mixes
// the columns of both rows) and rows p and q of V J.  The pairs partition the indices, so
// the blocks touch disjoint rows; the arithmetic is the row pass followed by the column pass
// of the two kernels above, with coalesced row accesses only.
__global__ void __launch_bounds__(256) jacobi_round_kernel(double *__restrict__ A, double *__restrict__ V, int Dp,
                                                           int r, const double2 *__restrict__ cs) {
    extern __shared__ double rows_sm[];
    double *rp = rows_sm, *rq = rows_sm + Dp, *vp = rows_sm + 2 * Dp, *vq = rows_sm + 3 * Dp;
    int p, q;
    rr_pair(r, blockIdx.x, Dp, p, q);
    const double2 k = cs[blockIdx.x];
    double *Ap = A + (int64_t)p * Dp, *Aq = A + (int64_t)q * Dp;
    double *Vp = V + (int64_t)p * Dp, *Vq = V + (int64_t)q * Dp;
    for (int j = threadIdx.x; j < Dp; j += blockDim.x) {
        const double a = Ap[j], b = Aq[j];
        rp[j] = k.x * a - k.y * b;
        rq[j] = k.y * a + k.x * b;
        vp[j] = Vp[j];
        vq[j] = Vq[j];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Dp / 2; t += blockDim.x) {
        int pp, qq;
        rr_pair(r, t, Dp, pp, qq);
        const double2 kk = cs[t];
        double a = rp[pp], b = rp[qq];
        rp[pp] = kk.x * a - kk.y * b;
        rp[qq] = kk.y * a + kk.x * b;
        a = rq[pp];
        b = rq[qq];
        rq[pp] = kk.x * a - kk.y * b;
        rq[qq] = kk.y * a + kk.x * b;
        a = vp[pp];
        b = vp[qq];
        vp[pp] = kk.x * a - kk.y * b;
        vp[qq] = kk.y * a + kk.x * b;
        a = vq[pp];
        b = vq[qq];
        vq[pp] = kk.x * a - kk.y * b;
        vq[qq] = kk.y * a + kk.x * b;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < Dp; j += blockDim.x) {
        Ap[j] = rp[j];
        Aq[j] = rq[j];
        Vp[j] = vp[j];
        Vq[j] = vq[j];
    }
}

// out[0] = sum of squared off-diagonal entries, out[1] = sum of squared diagonal entries
__global__ void jacobi_offnorm_kernel(const double *__restrict__ A, int Dp, double *__restrict__ out) {
    __shared__ double so[256], sd[256];
    double o = 0.0, d = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)Dp * Dp;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double v = A[t];
        if (t / Dp == t % Dp)
            d += v * v;
        else
            o += v * v;
    }
    so[threadIdx.x] = o;
    sd[threadIdx.x] = d;
    __syncthreads();
    for (int s = 128; s; s >>= 1) {
        if (threadIdx.x < s) {
            so[threadIdx.x] += so[threadIdx.x + s];
            sd[threadIdx.x] += sd[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(out, so[0]);
        atomicAdd(out + 1, sd[0]);
    }
}

__global__ void pad_copy_kernel(const double *__restrict__ K, int D, double *__restrict__ A, double *__restrict__ V,
                                int Dp) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)Dp * Dp) return;
    const int i = (int)(t / Dp), j = (int)(t % Dp);
    A[t] = (i < D && j < D) ? K[(int64_t)i * D + j] : 0.0;
    V[t] = i == j ? 1.0 : 0.0;
}

// evecs[r] = column idx[r] of V (first D entries), sign: largest-|.| entry positive
// (first index on ties); evals[r] = A[idx[r]][idx[r]].
__global__ void gather_eig_kernel(const double *__restrict__ A, const double *__restrict__ V, int Dp, int D,
                                  const int *__restrict__ idx, int nout, double *__restrict__ evals,
                                  double *__restrict__ evecs) {
    const int r = blockIdx.x;
    if (r >= nout) return;
    const int c = idx[r];
    __shared__ double sv[256];
    __shared__ int si[256];
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
        const double v = fabs(V[(int64_t)i * Dp + c]);
        if (v > best || (v == best && i < bi)) {
            best = v;
            bi = i;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s; s >>= 1) {
        if (threadIdx.x < s) {
            const double v = sv[threadIdx.x + s];
            const int j = si[threadIdx.x + s];
            if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && j < si[threadIdx.x])) {
                sv[threadIdx.x] = v;
                si[threadIdx.x] = j;
            }
        }
        __syncthreads();
    }
    const double sign = V[(int64_t)si[0] * Dp + c] < 0.0 ? -1.0 : 1.0;
    for (int i = threadIdx.x; i < D; i += blockDim.x) evecs[(int64_t)r * D + i] = sign * V[(int64_t)i * Dp + c];
    if (threadIdx.x == 0 && evals) evals[r] = A[(int64_t)c * Dp + c];
}

__global__ void diag_kernel(const double *__restrict__ A, int Dp, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Dp) out[i] = A[(int64_t)i * Dp + i];
}

__global__ void f32_to_f64_kernel(const float *__restrict__ a, int64_t n, double *__restrict__ b) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) b[t] = (double)a[t];
}

__global__ void f64_to_f32_kernel(const double *__restrict__ a, int64_t n, float *__restrict__ b) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) b[t] = (float)a[t];
}

bool eigh_top_ok(int D, int nout);
int eigh_top(const double *K, int D, int nout, double *evals, double *evecs, cudaStream_t st);

// Eigen-decomposition of symmetric K (D x D FP64, device).  Writes the nout leading
// eigenpairs (descending eigenvalue) to evals (nullable) / evecs (nout x D).  Fewer than D pairs
// of a matrix of 8 .. 4096 rows: tridiagonal reduction + bisection + inverse iteration
// (eigh_tri.cu); all of them: cyclic Jacobi.
int eigh_impl(const double *K, int D, int nout, double *evals, double *evecs, cudaStream_t st, int *sweeps_out) {
    if (nout < D && eigh_top_ok(D, nout)) {
        if (sweeps_out) *sweeps_out = 0;
        return eigh_top(K, D, nout, evals, evecs, st);
    }
    const int Dp = D + (D & 1);
    double *A = nullptr, *V = nullptr, *acc = nullptr, *dg = nullptr;
    double2 *cs = nullptr;
    int *idx_d = nullptr;
    int rc = LV_OK;
    std::vector<double> diag(Dp);
    std::vector<int> order(Dp);
    double host_acc[2];
    int sweep = 0;
    bool fused = (size_t)Dp * 32 <= 200 * 1024;  // four rows of Dp doubles in shared memory
    cudaGraphExec_t sweep_exec = nullptr;
    auto launch_sweep = [&](cudaStream_t s) {
        for (int r = 0; r < Dp - 1; ++r) {
            jacobi_rot_kernel<<<(Dp / 2 + 127) / 128, 128, 0, s>>>(A, Dp, r, cs);
            if (fused) {
                jacobi_round_kernel<<<Dp / 2, 256, (size_t)Dp * 32, s>>>(A, V, Dp, r, cs);
            } else {
                jacobi_rows_kernel<<<dim3((Dp + 127) / 128, Dp / 2), 128, 0, s>>>(A, Dp, r, cs);
                jacobi_cols_kernel<<<dim3((Dp + 127) / 128, Dp / 2), 128, 0, s>>>(A, V, Dp, r, cs);
            }
        }
    };
    if (tmp_alloc((void **)&A, sizeof(double) * Dp * Dp, st) || tmp_alloc((void **)&V, sizeof(double) * Dp * Dp, st) ||
        tmp_alloc((void **)&acc, 2 * sizeof(double), st) || tmp_alloc((void **)&cs, sizeof(double2) * Dp / 2, st) ||
        tmp_alloc((void **)&idx_d, sizeof(int) * Dp, st) || tmp_alloc((void **)&dg, sizeof(double) * Dp, st)) {
        rc = fail(LV_ERR_OOM, "eigh: allocation failed");
        goto done;
    }
    pad_copy_kernel<<<(unsigned)(((int64_t)Dp * Dp + 255) / 256), 256, 0, st>>>(K, D, A, V, Dp);
    // one sweep = Dp - 1 rounds of (rotation angles, fused round); captured once into a CUDA
    // graph (launched per sweep), else launched directly
    if (fused && Dp * 32 > 48 * 1024 &&
        cudaFuncSetAttribute(jacobi_round_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, Dp * 32) != cudaSuccess) {
        cudaGetLastError();
        fused = false;
    }
    {
        cudaStream_t cap = nullptr;
        cudaGraph_t graph = nullptr;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            launch_sweep(cap);
            if (cudaStreamEndCapture(cap, &graph) != cudaSuccess ||
                cudaGraphInstantiate(&sweep_exec, graph, 0) != cudaSuccess)
                sweep_exec = nullptr;
        }
        cudaGetLastError();  // a failed capture falls back to direct launches
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    }
    for (sweep = 0; sweep < 40; ++sweep) {
        cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
        jacobi_offnorm_kernel<<<128, 256, 0, st>>>(A, Dp, acc);
        cudaMemcpyAsync(host_acc, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "eigh: kernel failure");
            goto done;
        }
        const double tot = host_acc[0] + host_acc[1];
        if (!(host_acc[0] > 1e-28 * tot) || tot == 0.0) break;
        if (sweep_exec) {
            if (cudaGraphLaunch(sweep_exec, st) != cudaSuccess) {
                rc = fail(LV_ERR_CUDA, "eigh: sweep graph launch failed");
                goto done;
            }
        } else {
            launch_sweep(st);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "jacobi kernels");
            goto done;
        }
    }
    // sort eigenvalues descending (stable by index); the padding index (D) is dropped
    {
        diag_kernel<<<(Dp + 255) / 256, 256, 0, st>>>(A, Dp, dg);
        cudaMemcpyAsync(diag.data(), dg, sizeof(double) * Dp, cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "eigh: diagonal copy failed");
            goto done;
        }
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.begin() + D, [&](int a, int b) { return diag[a] > diag[b]; });
        cudaMemcpyAsync(idx_d, order.data(), sizeof(int) * D, cudaMemcpyHostToDevice, st);
        gather_eig_kernel<<<nout, 256, 0, st>>>(A, V, Dp, D, idx_d, nout, evals, evecs);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "eigh: gather failed");
            goto done;
        }
    }
done:
    if (sweep_exec) {
        cudaStreamSynchronize(st);
        cudaGraphExecDestroy(sweep_exec);
    }
    if (sweeps_out) *sweeps_out = sweep;
    tmp_free(A, st);
    tmp_free(V, st);
    tmp_free(acc, st);
    tmp_free(cs, st);
    tmp_free(idx_d, st);
    tmp_free(dg, st);
    return rc;
}

int second_moment_bf16(const float *X, int64_t n, int D, float *K, int *status, cudaStream_t st);

int launch_f32_to_f64(const float *a, int64_t n, double *b, cudaStream_t st) {
    f32_to_f64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, b);
    LV_CHECK_LAUNCH("f32_to_f64_kernel");
    return LV_OK;
}

int launch_f64_to_f32(const double *a, int64_t n, float *b, cudaStream_t st) {
    f64_to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, b);
    LV_CHECK_LAUNCH("f64_to_f32_kernel");
    return LV_OK;
}

}  // namespace lv

using namespace lv;

extern "C" {

int leanvec_second_moment(const float *X, int64_t n, int D, float *K, int precision, lv_stream_t stream) {
    if (!X || !K || n <= 0 || D <= 0) return fail(LV_ERR_ARG, "second_moment: invalid sizes or null pointer");
    if (precision == LV_PREC_FP32) return launch_gram_fp32(X, n, D, K, (cudaStream_t)stream);
    if (precision != LV_PREC_BF16) return fail(LV_ERR_ARG, "second_moment: precision must be LV_PREC_FP32 or LV_PREC_BF16");
    cudaStream_t st = (cudaStream_t)stream;
    int *status = nullptr, h = 0;
    if (tmp_alloc((void **)&status, sizeof(int), st)) return fail(LV_ERR_OOM, "second_moment: allocation failed");
    int rc = cudaMemsetAsync(status, 0, sizeof(int), st) == cudaSuccess ? LV_OK : fail(LV_ERR_CUDA, "memset failed");
    if (rc == LV_OK) rc = second_moment_bf16(X, n, D, K, status, st);
    if (rc == LV_OK && cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = fail(LV_ERR_CUDA, "second_moment: status copy failed");
    if (rc == LV_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(LV_ERR_CUDA, "second_moment: sync failed");
    if (rc == LV_OK && h) rc = fail(LV_ERR_TIMEOUT, "second_moment: a tensor-core pipeline wait timed out");
    tmp_free(status, st);
    return rc;
}

int leanvec_eigh(const double *K, int D, double *evals, double *evecs, lv_stream_t stream) {
    if (!K || !evecs || D <= 1) return fail(LV_ERR_ARG, "eigh: invalid sizes or null pointer");
    return eigh_impl(K, D, D, evals, evecs, (cudaStream_t)stream, nullptr);
}

int leanvec_fit_id(const float *X, int64_t n, int D, int d, float *A_out, float *B_out, int precision,
                   lv_stream_t stream) {
    if (!X || !A_out || n <= 0 || D <= 1 || d <= 0 || d > D)
        return fail(LV_ERR_ARG, "fit_id: invalid sizes or null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    float *K = nullptr;
    double *K64 = nullptr, *P = nullptr;
    int rc = LV_OK;
    if (tmp_alloc((void **)&K, sizeof(float) * D * D, st) || tmp_alloc((void **)&K64, sizeof(double) * D * D, st) ||
        tmp_alloc((void **)&P, sizeof(double) * (size_t)d * D, st)) {
        rc = fail(LV_ERR_OOM, "fit_id: allocation failed");
    }
    if (rc == LV_OK) rc = leanvec_second_moment(X, n, D, K, precision, stream);
    if (rc == LV_OK) rc = launch_f32_to_f64(K, (int64_t)D * D, K64, st);
    if (rc == LV_OK) rc = eigh_impl(K64, D, d, nullptr, P, st, nullptr);
    if (rc == LV_OK) rc = launch_f64_to_f32(P, (int64_t)d * D, A_out, st);
    if (rc == LV_OK && B_out && B_out != A_out)
        if (cudaMemcpyAsync(B_out, A_out, sizeof(float) * (size_t)d * D, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = fail(LV_ERR_CUDA, "fit_id: copy failed");
    if (rc == LV_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(LV_ERR_CUDA, "fit_id: sync failed");
    tmp_free(K, st);
    tmp_free(K64, st);
    tmp_free(P, st);
    return rc;
}

}  // extern "C"
