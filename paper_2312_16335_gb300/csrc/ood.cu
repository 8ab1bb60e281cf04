// LeanVec-OOD projection learning (Sec. 2.2 - 2.4):
//   loss  f(A, B) = tr(A K_Q A^T B K_X B^T) + tr(K_Q K_X) - 2 tr(K_Q A^T B K_X)
//   grads dA = 2 B K_X B^T A K_Q - 2 B K_X K_Q,  dB = 2 A K_Q A^T B K_X - 2 A K_Q K_X
//   Frank-Wolfe BCD (Algorithm 1): LMO over the spectral-norm ball = polar factor of -grad,
//     step 1 / (t + 1)^alpha or the exact quadratic line search, stop at relative
//     loss change <= tol;
//   eigenvector search (Algorithm 2): P(beta) = d leading eigenvectors of
//     K_beta = (1 - beta)/m K_Q + beta/n K_X, beta by bounded Brent minimisation.
// Losses and gradients are float32 GEMMs on the CUDA cores (d x D x D); the
// eigendecompositions (K_beta, and C C^T for the polar factor) and the step-size solve
// are FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace lv {

int eigh_impl(const double *K, int D, int nout, double *evals, double *evecs, cudaStream_t st, int *sweeps_out);
int launch_gram_fp32(const float *X, int64_t n, int D, float *K, cudaStream_t st);
int second_moment_bf16(const float *X, int64_t n, int D, float *K, int *status, cudaStream_t st);

// ------------------------------------------------------------- small GEMM
// C (M x N, ldc) = alpha * op(A) op(B) + beta * C, float32 or float64, op = transpose
// when the flag is set (A is M x K, or K x M when transposed; B is K x N or N x K).
template <typename T>
__global__ void __launch_bounds__(256) gemm_small_kernel(int M, int N, int K, T alpha, const T *__restrict__ A, int lda,
                                                         bool ta, const T *__restrict__ B, int ldb, bool tb, T beta,
                                                         T *__restrict__ C, int ldc) {
    __shared__ T As[16][65];
    __shared__ T Bs[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            const int kk = t / 64, i = t % 64;
            const int r = r0 + i, k = k0 + kk, c = c0 + i;
            As[kk][i] = (r < M && k < K) ? (ta ? A[(int64_t)k * lda + r] : A[(int64_t)r * lda + k]) : T(0);
            Bs[kk][i] = (c < N && k < K) ? (tb ? B[(int64_t)c * ldb + k] : B[(int64_t)k * ldb + c]) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[kk][ty * 4 + u];
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tx * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = r0 + ty * 4 + u;
        if (r >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = c0 + tx * 4 + v;
            if (c >= N) continue;
            T *o = C + (int64_t)r * ldc + c;
            *o = alpha * acc[u][v] + (beta == T(0) ? T(0) : beta * *o);
        }
    }
}

template <typename T>
static int gemm_small(int M, int N, int K, T alpha, const T *A, int lda, bool ta, const T *B, int ldb, bool tb, T beta,
                      T *C, int ldc, cudaStream_t st) {
    dim3 grd((N + 63) / 64, (M + 63) / 64);
    gemm_small_kernel<T><<<grd, 256, 0, st>>>(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc);
    LV_CHECK_LAUNCH("gemm_small_kernel");
    return LV_OK;
}

// out[slot] += <X, Y>_F (sum of elementwise products), FP64 accumulation of float32 data
__global__ void frob_dot_kernel(const float *__restrict__ X, const float *__restrict__ Y, int64_t n, double *out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        s += (double)X[t] * (double)Y[t];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, sh[0]);
}

// <X^T, Y>_F for square X, Y (= tr(X Y) for symmetric use)
__global__ void trace_prod_kernel(const float *__restrict__ X, const float *__restrict__ Y, int n, double *out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        s += (double)X[(int64_t)i * n + j] * (double)Y[(int64_t)j * n + i];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, sh[0]);
}

// Z = a X + b Y (float32; Z may alias X or Y)
__global__ void axpby_kernel(float a, const float *X, float b, const float *Y, int64_t n, float *Z) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) Z[t] = a * X[t] + b * Y[t];
}

// Kb = a Kq + b Kx in FP64 from float32
__global__ void kbeta_kernel(double a, const float *__restrict__ Kq, double b, const float *__restrict__ Kx, int64_t n,
                             double *__restrict__ Kb) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) Kb[t] = a * (double)Kq[t] + b * (double)Kx[t];
}

__global__ void f32_to_f64_k(const float *__restrict__ a, int64_t n, double *__restrict__ b) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) b[t] = (double)a[t];
}

__global__ void f64_to_f32_k(const double *__restrict__ a, int64_t n, float *__restrict__ b) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) b[t] = (float)a[t];
}

// W = U diag(w) U^T with w_i = 1/sqrt(lambda_i) (0 for lambda_i <= 1e-12 lambda_max); U rows = eigvecs
__global__ void inv_sqrt_kernel(const double *__restrict__ evals, const double *__restrict__ U, int d,
                                double *__restrict__ W) {
    const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    const double lmax = evals[0];
    double s = 0.0;
    for (int r = 0; r < d; ++r) {
        const double l = evals[r];
        const double w = (l > 1e-12 * lmax && l > 0.0) ? 1.0 / sqrt(l) : 0.0;
        s += U[(int64_t)r * d + i] * w * U[(int64_t)r * d + j];
    }
    W[(int64_t)i * d + j] = s;
}

// ---------------------------------------------------------------- context
struct OodCtx {
    int D, d;
    int64_t n, m;
    float *KX, *KQ;           // D x D
    float *t1, *t2, *t3;      // d x D scratch
    float *s1, *s2;           // d x d scratch
    float *S;                 // d x D LMO result
    float *P_id;              // d x D ID solution (for the zero-gradient reading)
    double *G64, *C64, *W64, *S64, *ev64, *U64;  // polar factor work (d x d / d x D)
    double *acc;              // 8 scalars
    double trQX;              // tr(K_Q K_X)
    cudaStream_t st;
};

static int red_frob(OodCtx &c, const float *X, const float *Y, int64_t n, double *out_host) {
    LV_CUDA(cudaMemsetAsync(c.acc, 0, sizeof(double), c.st));
    frob_dot_kernel<<<64, 256, 0, c.st>>>(X, Y, n, c.acc);
    LV_CHECK_LAUNCH("frob_dot_kernel");
    LV_CUDA(cudaMemcpyAsync(out_host, c.acc, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    LV_CUDA(cudaStreamSynchronize(c.st));
    return LV_OK;
}

// f(A, B) = tr(A K_Q A^T B K_X B^T) + tr(K_Q K_X) - 2 tr(K_Q A^T B K_X)
static int ood_loss_dev(OodCtx &c, const float *A, const float *B, double *f) {
    const int D = c.D, d = c.d;
    int rc;
    // t1 = A K_Q, s1 = t1 A^T ; t2 = B K_X, s2 = t2 B^T
    if ((rc = gemm_small<float>(d, D, D, 1.f, A, D, false, c.KQ, D, false, 0.f, c.t1, D, c.st))) return rc;
    if ((rc = gemm_small<float>(d, d, D, 1.f, c.t1, D, false, A, D, true, 0.f, c.s1, d, c.st))) return rc;
    if ((rc = gemm_small<float>(d, D, D, 1.f, B, D, false, c.KX, D, false, 0.f, c.t2, D, c.st))) return rc;
    if ((rc = gemm_small<float>(d, d, D, 1.f, c.t2, D, false, B, D, true, 0.f, c.s2, d, c.st))) return rc;
    // t3 = t2 K_Q = B K_X K_Q ; tr(K_Q A^T B K_X) = <A, B K_X K_Q>_F
    if ((rc = gemm_small<float>(d, D, D, 1.f, c.t2, D, false, c.KQ, D, false, 0.f, c.t3, D, c.st))) return rc;
    LV_CUDA(cudaMemsetAsync(c.acc, 0, 2 * sizeof(double), c.st));
    trace_prod_kernel<<<16, 256, 0, c.st>>>(c.s1, c.s2, d, c.acc);
    frob_dot_kernel<<<64, 256, 0, c.st>>>(A, c.t3, (int64_t)d * D, c.acc + 1);
    LV_CHECK_LAUNCH("loss reductions");
    double h[2];
    LV_CUDA(cudaMemcpyAsync(h, c.acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    LV_CUDA(cudaStreamSynchronize(c.st));
    *f = h[0] + c.trQX - 2.0 * h[1];
    return LV_OK;
}

// gradient wrt the first block: g = 2 (Y K_Y Y^T Z - Y K_Y) K_Z, where (Y, K_Y) is the other
// block and (Z, K_Z) the block being differentiated: dA uses (B, K_X) and (A, K_Q),
// dB uses (A, K_Q) and (B, K_X).  Result in `g` (d x D).
static int ood_grad_dev(OodCtx &c, const float *Y, const float *KY, const float *Z, const float *KZ, float *g) {
    const int D = c.D, d = c.d;
    int rc;
    if ((rc = gemm_small<float>(d, D, D, 1.f, Y, D, false, KY, D, false, 0.f, c.t1, D, c.st))) return rc;  // Y K_Y
    if ((rc = gemm_small<float>(d, d, D, 1.f, c.t1, D, false, Y, D, true, 0.f, c.s1, d, c.st))) return rc;  // Y K_Y Y^T
    // t2 = s1 Z - t1
    if ((rc = gemm_small<float>(d, D, d, 1.f, c.s1, d, false, Z, D, false, 0.f, c.t2, D, c.st))) return rc;
    axpby_kernel<<<(unsigned)(((int64_t)d * D + 255) / 256), 256, 0, c.st>>>(1.f, c.t2, -1.f, c.t1, (int64_t)d * D,
                                                                           c.t2);
    LV_CHECK_LAUNCH("axpby_kernel");
    return gemm_small<float>(d, D, D, 2.f, c.t2, D, false, KZ, D, false, 0.f, g, D, c.st);
}

// S = argmax_{||S||_op <= 1} <S, C> = polar factor (C C^T)^{-1/2} C (FP64 eig of C C^T)
static int polar_dev(OodCtx &c, const float *C, float *S) {
    const int D = c.D, d = c.d;
    const int64_t nd = (int64_t)d * D;
    f32_to_f64_k<<<(unsigned)((nd + 255) / 256), 256, 0, c.st>>>(C, nd, c.C64);
    LV_CHECK_LAUNCH("f32_to_f64_k");
    int rc = gemm_small<double>(d, d, D, 1.0, c.C64, D, false, c.C64, D, true, 0.0, c.G64, d, c.st);
    if (rc) return rc;
    rc = eigh_impl(c.G64, d, d, c.ev64, c.U64, c.st, nullptr);
    if (rc) return rc;
    inv_sqrt_kernel<<<dim3((d + 127) / 128, d), 128, 0, c.st>>>(c.ev64, c.U64, d, c.W64);
    LV_CHECK_LAUNCH("inv_sqrt_kernel");
    rc = gemm_small<double>(d, D, d, 1.0, c.W64, d, false, c.C64, D, false, 0.0, c.S64, D, c.st);
    if (rc) return rc;
    f64_to_f32_k<<<(unsigned)((nd + 255) / 256), 256, 0, c.st>>>(c.S64, nd, S);
    LV_CHECK_LAUNCH("f64_to_f32_k");
    return LV_OK;
}

// d leading eigenvectors (rows, float32) of the FP64 matrix Kb (D x D)
static int top_eigvecs_dev(OodCtx &c, double *Kb, float *P, double *Pwork) {
    int rc = eigh_impl(Kb, c.D, c.d, nullptr, Pwork, c.st, nullptr);
    if (rc) return rc;
    const int64_t nd = (int64_t)c.d * c.D;
    f64_to_f32_k<<<(unsigned)((nd + 255) / 256), 256, 0, c.st>>>(Pwork, nd, P);
    LV_CHECK_LAUNCH("f64_to_f32_k");
    return LV_OK;
}

// Bounded Brent minimisation of a scalar function on [a, b] (Brent 1973, "Algorithms for
// minimization without derivatives", ch. 5: golden-section steps with parabolic
// interpolation), absolute tolerance xatol.
template <class F>
static int brent_min(F &&func, double a, double b, double xatol, int maxit, double *xbest, double *fbest, int *nev) {
    const double golden = 0.5 * (3.0 - std::sqrt(5.0));
    double x = a + golden * (b - a), w = x, v = x;
    double fx;
    int rc = func(x, &fx);
    if (rc) return rc;
    int evals = 1;
    double fw = fx, fv = fx, d = 0.0, e = 0.0;
    for (int it = 0; it < maxit; ++it) {
        const double xm = 0.5 * (a + b);
        const double tol1 = std::sqrt(2.2e-16) * std::fabs(x) + xatol / 3.0, tol2 = 2.0 * tol1;
        if (std::fabs(x - xm) <= tol2 - 0.5 * (b - a)) break;
        bool golden_step = true;
        if (std::fabs(e) > tol1) {
            // parabola through (v, fv), (w, fw), (x, fx)
            double r = (x - w) * (fx - fv), q = (x - v) * (fx - fw), p = (x - v) * q - (x - w) * r;
            q = 2.0 * (q - r);
            if (q > 0.0) p = -p;
            q = std::fabs(q);
            const double etemp = e;
            e = d;
            if (std::fabs(p) < std::fabs(0.5 * q * etemp) && p > q * (a - x) && p < q * (b - x)) {
                d = p / q;
                const double u = x + d;
                if (u - a < tol2 || b - u < tol2) d = xm - x >= 0.0 ? tol1 : -tol1;
                golden_step = false;
            }
        }
        if (golden_step) {
            e = (x >= xm) ? a - x : b - x;
            d = golden * e;
        }
        const double u = std::fabs(d) >= tol1 ? x + d : x + (d >= 0.0 ? tol1 : -tol1);
        double fu;
        rc = func(u, &fu);
        if (rc) return rc;
        ++evals;
        if (fu <= fx) {
            if (u >= x)
                a = x;
            else
                b = x;
            v = w;
            fv = fw;
            w = x;
            fw = fx;
            x = u;
            fx = fu;
        } else {
            if (u < x)
                a = u;
            else
                b = u;
            if (fu <= fw || w == x) {
                v = w;
                fv = fw;
                w = u;
                fw = fu;
            } else if (fu <= fv || v == x || v == w) {
                v = u;
                fv = fu;
            }
        }
    }
    *xbest = x;
    *fbest = fx;
    *nev = evals;
    return LV_OK;
}

// W = U diag(min(1, 1/sigma_i)) U^T with sigma_i^2 the eigenvalues of A A^T
__global__ void clip_scale_kernel(const double *__restrict__ evals, const double *__restrict__ U, int d,
                                  double *__restrict__ W) {
    const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    double s = 0.0;
    for (int r = 0; r < d; ++r) {
        const double l = evals[r];
        const double w = l > 1.0 ? 1.0 / sqrt(l) : 1.0;
        s += U[(int64_t)r * d + i] * w * U[(int64_t)r * d + j];
    }
    W[(int64_t)i * d + j] = s;
}

}  // namespace lv

using namespace lv;

extern "C" {

int leanvec_spectral_clip(float *A, int d, int D, lv_stream_t stream) {
    if (!A || d <= 0 || D <= 0 || d > D) return fail(LV_ERR_ARG, "spectral_clip: invalid sizes or null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t dD = (size_t)d * D, dd = (size_t)d * d;
    double *A64 = nullptr, *G = nullptr, *ev = nullptr, *U = nullptr, *W = nullptr, *R = nullptr;
    int rc = LV_OK;
    if (tmp_alloc((void **)&A64, 8 * dD, st) || tmp_alloc((void **)&G, 8 * dd, st) ||
        tmp_alloc((void **)&ev, 8 * (size_t)d, st) || tmp_alloc((void **)&U, 8 * dd, st) ||
        tmp_alloc((void **)&W, 8 * dd, st) || tmp_alloc((void **)&R, 8 * dD, st))
        rc = fail(LV_ERR_OOM, "spectral_clip: allocation failed");
    if (rc == LV_OK) {
        f32_to_f64_k<<<(unsigned)((dD + 255) / 256), 256, 0, st>>>(A, (int64_t)dD, A64);
        rc = gemm_small<double>(d, d, D, 1.0, A64, D, false, A64, D, true, 0.0, G, d, st);
    }
    if (rc == LV_OK) rc = d > 1 ? eigh_impl(G, d, d, ev, U, st, nullptr) : LV_OK;
    if (rc == LV_OK && d == 1) {
        // 1 x 1: sigma^2 = G, U = 1
        double one = 1.0;
        cudaMemcpyAsync(ev, G, 8, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(U, &one, 8, cudaMemcpyHostToDevice, st);
    }
    if (rc == LV_OK) {
        clip_scale_kernel<<<dim3((d + 127) / 128, d), 128, 0, st>>>(ev, U, d, W);
        rc = gemm_small<double>(d, D, d, 1.0, W, d, false, A64, D, false, 0.0, R, D, st);
    }
    if (rc == LV_OK) {
        f64_to_f32_k<<<(unsigned)((dD + 255) / 256), 256, 0, st>>>(R, (int64_t)dD, A);
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = fail(LV_ERR_CUDA, "spectral_clip: sync failed");
    }
    tmp_free(A64, st);
    tmp_free(G, st);
    tmp_free(ev, st);
    tmp_free(U, st);
    tmp_free(W, st);
    tmp_free(R, st);
    return rc;
}

int leanvec_fit_ood(const float *X, int64_t n, const float *Q, int64_t m, int D, int d, const lv_fit_opts *opts,
                    float *A_out, float *B_out, lv_fit_report *rep, lv_stream_t stream) {
    if (!X || !Q || !A_out || !B_out || !opts) return fail(LV_ERR_ARG, "fit_ood: null pointer");
    if (n <= 0 || m <= 0 || D <= 1 || d <= 0 || d > D) return fail(LV_ERR_ARG, "fit_ood: invalid sizes");
    if (opts->method < LV_FIT_FW || opts->method > LV_FIT_ES_FW) return fail(LV_ERR_ARG, "fit_ood: unknown method");
    if (opts->precision != LV_PREC_FP32 && opts->precision != LV_PREC_BF16)
        return fail(LV_ERR_ARG, "fit_ood: second-moment precision must be LV_PREC_FP32 or LV_PREC_BF16");
    cudaStream_t st = (cudaStream_t)stream;
    OodCtx c;
    memset(&c, 0, sizeof(c));
    c.D = D;
    c.d = d;
    c.n = n;
    c.m = m;
    c.st = st;
    const size_t DD = (size_t)D * D, dD = (size_t)d * D, dd = (size_t)d * d;
    std::vector<void *> allocs;
    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (tmp_alloc(p, bytes, st) != LV_OK) return false;
        allocs.push_back(*p);
        return true;
    };
    int rc = LV_OK;
    int *status = nullptr;
    double *Kb = nullptr, *Pw = nullptr;
    float *Bnew = nullptr, *g = nullptr;
    bool ok = alloc((void **)&c.KX, 4 * DD) && alloc((void **)&c.KQ, 4 * DD) && alloc((void **)&c.t1, 4 * dD) &&
              alloc((void **)&c.t2, 4 * dD) && alloc((void **)&c.t3, 4 * dD) && alloc((void **)&c.s1, 4 * dd) &&
              alloc((void **)&c.s2, 4 * dd) && alloc((void **)&c.S, 4 * dD) && alloc((void **)&c.P_id, 4 * dD) &&
              alloc((void **)&c.G64, 8 * dd) && alloc((void **)&c.C64, 8 * dD) && alloc((void **)&c.W64, 8 * dd) &&
              alloc((void **)&c.S64, 8 * dD) && alloc((void **)&c.ev64, 8 * (size_t)d) &&
              alloc((void **)&c.U64, 8 * dd) && alloc((void **)&c.acc, 8 * 8) && alloc((void **)&Kb, 8 * DD) &&
              alloc((void **)&Pw, 8 * dD) && alloc((void **)&Bnew, 4 * dD) && alloc((void **)&g, 4 * dD) &&
              alloc((void **)&status, sizeof(int));
    lv_fit_report R;
    memset(&R, 0, sizeof(R));
    const int maxit = opts->max_iter > 0 ? opts->max_iter : 500;
    const double alpha = opts->alpha > 0.f ? opts->alpha : 0.5;
    const double tol = opts->tol > 0.f ? opts->tol : 1e-3;
    auto second = [&](const float *Y, int64_t rows, float *K) -> int {
        if (opts->precision == LV_PREC_BF16) return second_moment_bf16(Y, rows, D, K, status, st);
        return launch_gram_fp32(Y, rows, D, K, st);
    };
    if (!ok) {
        rc = fail(LV_ERR_OOM, "fit_ood: allocation failed");
        goto done;
    }
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) {
        rc = fail(LV_ERR_CUDA, "fit_ood: memset failed");
        goto done;
    }
    if ((rc = second(X, n, c.KX)) || (rc = second(Q, m, c.KQ))) goto done;
    {
        // tr(K_Q K_X)
        LV_CUDA(cudaMemsetAsync(c.acc, 0, sizeof(double), st));
        trace_prod_kernel<<<64, 256, 0, st>>>(c.KQ, c.KX, D, c.acc);
        if (cudaMemcpyAsync(&c.trQX, c.acc, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "fit_ood: reduction failed");
            goto done;
        }
    }
    // ID solution (used by the zero-gradient reading of the first FW step)
    {
        f32_to_f64_k<<<(unsigned)((DD + 255) / 256), 256, 0, st>>>(c.KX, (int64_t)DD, Kb);
        if ((rc = top_eigvecs_dev(c, Kb, c.P_id, Pw))) goto done;
    }
    if (opts->method == LV_FIT_ES || opts->method == LV_FIT_ES_FW) {
        // Algorithm 2: Brent over beta of f(P(beta), P(beta))
        auto func = [&](double beta, double *fv) -> int {
            kbeta_kernel<<<(unsigned)((DD + 255) / 256), 256, 0, st>>>((1.0 - beta) / (double)m, c.KQ, beta / (double)n,
                                                                      c.KX, (int64_t)DD, Kb);
            int r2 = top_eigvecs_dev(c, Kb, A_out, Pw);
            if (r2) return r2;
            return ood_loss_dev(c, A_out, A_out, fv);
        };
        double beta = 0.0, fb = 0.0;
        int nev = 0;
        rc = brent_min(func, 0.0, 1.0, opts->es_xatol > 0 ? opts->es_xatol : 1e-5, 500, &beta, &fb, &nev);
        if (rc) goto done;
        if ((rc = func(beta, &fb))) goto done;  // leave P(beta*) in A_out
        LV_CUDA(cudaMemcpyAsync(B_out, A_out, 4 * dD, cudaMemcpyDeviceToDevice, st));
        R.beta = beta;
        R.evaluations = nev + 1;
        R.loss = fb;
    }
    if (opts->method == LV_FIT_FW || opts->method == LV_FIT_ES_FW) {
        // Algorithm 1 from A0 = B0 = 0 (FW) or from the ES solution (ES + FW)
        if (opts->method == LV_FIT_FW) {
            LV_CUDA(cudaMemsetAsync(A_out, 0, 4 * dD, st));
            LV_CUDA(cudaMemsetAsync(B_out, 0, 4 * dD, st));
        }
        const bool ls = opts->line_search != 0 || opts->method == LV_FIT_ES_FW;
        double f_prev;
        if ((rc = ood_loss_dev(c, A_out, B_out, &f_prev))) goto done;
        R.loss0 = f_prev;
        if (rep && rep->loss_trace && rep->trace_capacity > 0) rep->loss_trace[0] = f_prev;
        int it = 0;
        for (int t = 0; t < maxit; ++t) {
            it = t + 1;
            const double gamma = 1.0 / std::pow((double)(t + 1), alpha);
            for (int blk = 0; blk < 2; ++blk) {
                float *Z = blk == 0 ? A_out : B_out;
                const float *Y = blk == 0 ? B_out : A_out;
                const float *KY = blk == 0 ? c.KX : c.KQ, *KZ = blk == 0 ? c.KQ : c.KX;
                if ((rc = ood_grad_dev(c, Y, KY, Z, KZ, g))) goto done;
                double gn2;
                if ((rc = red_frob(c, g, g, (int64_t)dD, &gn2))) goto done;
                if (gn2 == 0.0) {
                    LV_CUDA(cudaMemcpyAsync(c.S, c.P_id, 4 * dD, cudaMemcpyDeviceToDevice, st));
                } else {
                    // C = -g; the polar factor of -g is minus the polar factor of g
                    if ((rc = polar_dev(c, g, c.S))) goto done;
                    axpby_kernel<<<(unsigned)((dD + 255) / 256), 256, 0, st>>>(-1.f, c.S, 0.f, c.S, (int64_t)dD, c.S);
                }
                double step = gamma;
                if (ls) {
                    // f(Z + s (S - Z)) is quadratic in s: s* = -<g, S - Z> / (2 <Dl K_Z Dl^T, Y K_Y Y^T>)
                    float *Dl = Bnew;
                    axpby_kernel<<<(unsigned)((dD + 255) / 256), 256, 0, st>>>(1.f, c.S, -1.f, Z, (int64_t)dD, Dl);
                    double slope, curv;
                    if ((rc = red_frob(c, g, Dl, (int64_t)dD, &slope))) goto done;
                    if ((rc = gemm_small<float>(d, D, D, 1.f, Y, D, false, KY, D, false, 0.f, c.t1, D, st))) goto done;
                    if ((rc = gemm_small<float>(d, d, D, 1.f, c.t1, D, false, Y, D, true, 0.f, c.s1, d, st))) goto done;
                    if ((rc = gemm_small<float>(d, D, D, 1.f, Dl, D, false, KZ, D, false, 0.f, c.t2, D, st))) goto done;
                    if ((rc = gemm_small<float>(d, d, D, 1.f, c.t2, D, false, Dl, D, true, 0.f, c.s2, d, st))) goto done;
                    if ((rc = red_frob(c, c.s1, c.s2, (int64_t)dd, &curv))) goto done;
                    step = curv > 0.0 ? std::min(1.0, std::max(0.0, -slope / (2.0 * curv))) : (slope < 0.0 ? 1.0 : 0.0);
                }
                axpby_kernel<<<(unsigned)((dD + 255) / 256), 256, 0, st>>>((float)(1.0 - step), Z, (float)step, c.S,
                                                                          (int64_t)dD, Z);
                LV_CHECK_LAUNCH("FW update");
            }
            double f;
            if ((rc = ood_loss_dev(c, A_out, B_out, &f))) goto done;
            if (rep && rep->loss_trace && it < rep->trace_capacity) rep->loss_trace[it] = f;
            const bool stop = f_prev > 0.0 ? std::fabs(f - f_prev) / f_prev <= tol : true;
            f_prev = f;
            if (stop) break;
        }
        R.iterations = it;
        R.loss = f_prev;
    }
    {
        int h = 0;
        if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "fit_ood: final sync failed");
            goto done;
        }
        if (h) rc = fail(LV_ERR_TIMEOUT, "fit_ood: a tensor-core pipeline wait timed out");
    }
done:
    cudaStreamSynchronize(st);
    if (rep) {
        double *trace = rep->loss_trace;
        int cap = rep->trace_capacity;
        *rep = R;
        rep->loss_trace = trace;
        rep->trace_capacity = cap;
    }
    for (void *p : allocs) tmp_free(p, st);
    return rc;
}

}  // extern "C"
