// Differentiation form of the LeanVec-OOD loss over explicit sample pairs
// (problem "leanvec_orthonormal" / Eq. "leanvec_loss" written per pair):
//   r_ij = q_j^T x_i - (A q_j)^T (B x_i),   L = sum_ij r_ij^2 / (n m)
//   dL/dA = -2/(nm) sum_ij r_ij (B x_i) q_j^T = -2/(nm) (R X')^T Q
//   dL/dB = -2/(nm) sum_ij r_ij (A q_j) x_i^T = -2/(nm) (R^T Q')^T X
// with Q' = Q A^T (m x d), X' = X B^T (n x d) and R (m x n) the residual matrix.
// Tensor-core forms: r_ij = qt_j^T x_i with qt_j = q_j - B^T A q_j formed first in float32, so that
// no tile product carries the cancellation.  The loss (D % 4 == 0) is a fused sum of squares of
// tf32x3 tile products; the gradients (D % 8 == 0, d <= 128) recompute each residual tile in TMEM
// (bf16x3) and contract it there with X' or Q' (tf32x3) -- R is never stored (ood_loss_bwd_tc).
// Other shapes: 64 x 64 pair tiles are recomputed from Q, X, Q', X' on the CUDA cores in float32
// (one kernel walks the database tiles for each query tile: loss, U = R X'; another the query tiles
// for each database tile: V = R^T Q').
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "common.cuh"

namespace lv {

int launch_project_fp32(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy,
                        cudaStream_t st);

constexpr int PT = 64;    // pair tile
constexpr int PK = 16;    // k step
constexpr int DMAX = 256; // largest d

// R tile (PT x PT, rows = "row set", cols = "col set") into smem Rs:
//   Rs[r][c] = <P_r, Q_c> - <P'_r, Q'_c>, P rows of (rows x D), P' rows of (rows x d)
__device__ __forceinline__ void residual_tile(const float *__restrict__ P, const float *__restrict__ Pp, int64_t r0,
                                              int64_t nr, const float *__restrict__ Qm, const float *__restrict__ Qp,
                                              int64_t c0, int64_t nc, int D, int d, float (*As)[PT + 4],
                                              float (*Bs)[PT + 4], float (*Rs)[PT + 1]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int pass = 0; pass < 2; ++pass) {
        const float *Am = pass == 0 ? P : Pp;
        const float *Bm = pass == 0 ? Qm : Qp;
        const int K = pass == 0 ? D : d;
        const float sgn = pass == 0 ? 1.f : -1.f;
        for (int k0 = 0; k0 < K; k0 += PK) {
            for (int t = threadIdx.x; t < PK * PT; t += 256) {
                const int kk = t % PK, i = t / PK;
                const int64_t ra = r0 + i, cb = c0 + i;
                const int k = k0 + kk;
                As[kk][i] = (ra < nr && k < K) ? Am[ra * K + k] : 0.f;
                Bs[kk][i] = (cb < nc && k < K) ? sgn * Bm[cb * K + k] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < PK; ++kk) {
                // one 16-byte shared load per operand (rows of PT + 4 floats keep them aligned)
                const float4 a4 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
                const float4 b4 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
                const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t r = r0 + ty * 4 + u, c = c0 + tx * 4 + v;
            Rs[ty * 4 + u][tx * 4 + v] = (r < nr && c < nc) ? acc[u][v] : 0.f;
        }
    __syncthreads();
}

// For the row tile blockIdx.x of this block (rows of P): loop over the column tiles of column
// split blockIdx.y (columns [y cs, (y + 1) cs)), accumulate the loss partial (sum r^2 into
// lossp[y * gridDim.x + x], when lossp != NULL) and Out_y[rows] = R * Colp over the split
// (PT x d, split y's partial at Out + y * nr * d).
template <bool OUT>
__global__ void __launch_bounds__(256) pair_sweep_kernel(const float *__restrict__ P, const float *__restrict__ Pp,
                                                         int64_t nr, const float *__restrict__ Qm,
                                                         const float *__restrict__ Qp, int64_t nc, int D, int d,
                                                         int64_t cs, double *__restrict__ lossp,
                                                         float *__restrict__ Out) {
    __shared__ __align__(16) float As[PK][PT + 4];
    __shared__ __align__(16) float Bs[PK][PT + 4];
    __shared__ float Rs[PT][PT + 1];
    __shared__ double red[256];
    const int64_t r0 = (int64_t)blockIdx.x * PT;
    // Out tile accumulators: thread owns rows (threadIdx.x / 16) * 4 + u, cols (threadIdx.x % 16) + 16 w
    const int orow = (threadIdx.x >> 4) * 4, ocol = threadIdx.x & 15;
    constexpr int OW = OUT ? DMAX / 16 : 1;  // the loss-only sweep keeps no output accumulators
    float o[4][OW];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < OW; ++w) o[u][w] = 0.f;
    double ls = 0.0;
    const int64_t cbeg = (int64_t)blockIdx.y * cs, cend = min(nc, cbeg + cs);
    for (int64_t c0 = cbeg; c0 < cend; c0 += PT) {
        residual_tile(P, Pp, r0, nr, Qm, Qp, c0, nc, D, d, As, Bs, Rs);
        if (lossp) {
            for (int t = threadIdx.x; t < PT * PT; t += 256) {
                const float r = Rs[t / PT][t % PT];
                ls += (double)r * (double)r;
            }
        }
        if (OUT) {
            // Out[r][c] += sum_k Rs[r][k] * Qp[c0 + k][c]
            for (int k = 0; k < PT; ++k) {
                const int64_t ck = c0 + k;
                if (ck >= cend) break;
                const float *qrow = Qp + ck * d;
                float rv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) rv[u] = Rs[orow + u][k];
#pragma unroll
                for (int w = 0; w < OW; ++w) {
                    const int c = ocol + 16 * w;
                    if (c < d) {
                        const float q = qrow[c];
#pragma unroll
                        for (int u = 0; u < 4; ++u) o[u][w] = fmaf(rv[u], q, o[u][w]);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (OUT) {
        float *const Oy = Out + (int64_t)blockIdx.y * nr * d;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t r = r0 + orow + u;
            if (r >= nr) continue;
#pragma unroll
            for (int w = 0; w < OW; ++w) {
                const int c = ocol + 16 * w;
                if (c < d) Oy[r * d + c] = o[u][w];
            }
        }
    }
    if (lossp) {
        red[threadIdx.x] = ls;
        __syncthreads();
        for (int s = 128; s; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) lossp[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
    }
}

// out_y (d x D) = scale * M^T Y over the rows [y rs, (y + 1) rs) of M (rows x d) and Y (rows x D),
// y = blockIdx.y (split y's partial at out + y * d * D): column blocks of D, rows looped
__global__ void __launch_bounds__(256) tgemm_kernel(const float *__restrict__ M, const float *__restrict__ Y,
                                                    int64_t rows_total, int64_t rs, int d, int D, float scale,
                                                    float *__restrict__ out) {
    const int64_t rbeg = (int64_t)blockIdx.y * rs;
    const int64_t rows = max((int64_t)0, min(rows_total - rbeg, rs));
    M += rbeg * d;
    Y += rbeg * D;
    out += (int64_t)blockIdx.y * d * D;
    const int c = blockIdx.x * 64 + (threadIdx.x & 63);
    const int r0 = (threadIdx.x >> 6);  // 4 row groups of d
    __shared__ float Ms[32][DMAX];
    __shared__ float Ys[32][64];
    float acc[DMAX / 4];
#pragma unroll
    for (int i = 0; i < DMAX / 4; ++i) acc[i] = 0.f;
    for (int64_t k0 = 0; k0 < rows; k0 += 32) {
        for (int t = threadIdx.x; t < 32 * d; t += 256) {
            const int kk = t / d, i = t % d;
            Ms[kk][i] = (k0 + kk < rows) ? M[(k0 + kk) * d + i] : 0.f;
        }
        for (int t = threadIdx.x; t < 32 * 64; t += 256) {
            const int kk = t / 64, j = t % 64;
            const int cc = blockIdx.x * 64 + j;
            Ys[kk][j] = (k0 + kk < rows && cc < D) ? Y[(k0 + kk) * D + cc] : 0.f;
        }
        __syncthreads();
        for (int kk = 0; kk < 32; ++kk) {
            const float y = Ys[kk][threadIdx.x & 63];
#pragma unroll
            for (int i = 0; i < DMAX / 4; ++i) {
                const int row = r0 + 4 * i;
                if (row < d) acc[i] = fmaf(Ms[kk][row], y, acc[i]);
            }
        }
        __syncthreads();
    }
    if (c < D) {
#pragma unroll
        for (int i = 0; i < DMAX / 4; ++i) {
            const int row = r0 + 4 * i;
            if (row < d) out[(int64_t)row * D + c] = scale * acc[i];
        }
    }
}

int pair_sq_tf32(const float *Qh, const float *Ql, int64_t m, const float *Xh, const float *Xl, int64_t n, int K,
                 double *partial, int *nparts, int *status, cudaStream_t st);
int launch_tf32_split(const float *v, int64_t len, float *hi, float *lo, cudaStream_t st);
int launch_transpose_tf32_split(const float *Y, int64_t rows, int cols, float *hi, float *lo, int64_t ldt,
                                cudaStream_t st);
int launch_bf16_split(const float *v, int64_t len, __nv_bfloat16 *hi, __nv_bfloat16 *lo, cudaStream_t st);
int pair_flash_splits(int64_t M, int64_t N, int grid, int max_splits, int *cbps);
int pair_flash(const __nv_bfloat16 *Rh, const __nv_bfloat16 *Rl, int64_t M, const __nv_bfloat16 *Ch,
               const __nv_bfloat16 *Cl, int64_t N, int K, const float *Th, const float *Tl, int64_t ldt, int d,
               int splits, int cbps, float *out, int *status, cudaStream_t st);
int gemm_t_tf32_splits(int64_t M, int64_t N, int64_t K);
bool project_bf16_fused_ok(const float *X, int D, int d);
size_t project_tc_ws_bytes(int prec, int64_t n, int D, int d, const float *X);
int project_tf32x3(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, void **ws,
                   size_t *ws_bytes, int *status, cudaStream_t st);
int gemm_t_tf32(const float *Ah, const float *Al, int64_t M, int64_t lda, const float *Bh, const float *Bl, int64_t N,
                int64_t ldb, int64_t K, float *out, int64_t ldo, int64_t split_stride, int accumulate, int splits,
                int *status, cudaStream_t st);

// Bt (D x d) = B^T for B (d x D)
__global__ void transpose_kernel(const float *__restrict__ B, int d, int D, float *__restrict__ Bt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)d * D) return;
    const int i = (int)(t / D), k = (int)(t % D);
    Bt[(int64_t)k * d + i] = B[t];
}

// Y -= Z elementwise (float32)
__global__ void sub_inplace_kernel(float *__restrict__ Y, const float *__restrict__ Z, int64_t len) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < len) Y[t] = Y[t] - Z[t];
}

// out[i] = scale * sum_y part[y * len + i] for y = 0 .. splits - 1, in that order
__global__ void split_sum_kernel(const float *__restrict__ part, int splits, int64_t len, float *__restrict__ out,
                                 float scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    float v = 0.f;
    for (int y = 0; y < splits; ++y) v += part[(int64_t)y * len + i];
    out[i] = scale * v;
}

// splits of a sweep with `tiles` row tiles over `ncols` columns: about 4 blocks per SM in all,
// each split at least one column tile
static int sweep_splits(int64_t tiles, int64_t ncols) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (4 * (int64_t)sms + tiles - 1) / tiles;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (ncols + PT - 1) / PT));
}

static int64_t split_len(int64_t total, int splits, int64_t align) {
    return ((total + splits - 1) / splits + align - 1) / align * align;
}

struct PairWork {
    float *Qp = nullptr, *Xp = nullptr, *U = nullptr, *V = nullptr;
    float *Up = nullptr, *Gp = nullptr;  // split partials of U and of the gradient GEMMs
    double *part = nullptr;
};

static int pair_prepare(const float *A, const float *B, const float *Q, int64_t m, const float *X, int64_t n, int D,
                        int d, PairWork &w, bool grads, cudaStream_t st) {
    const int64_t tiles = (m + PT - 1) / PT;
    if (tmp_alloc((void **)&w.Qp, sizeof(float) * (size_t)m * d, st) ||
        tmp_alloc((void **)&w.Xp, sizeof(float) * (size_t)n * d, st) ||
        tmp_alloc((void **)&w.part, sizeof(double) * (size_t)(tiles * sweep_splits(tiles, n)), st))
        return fail(LV_ERR_OOM, "ood_loss: allocation failed");
    if (grads && (tmp_alloc((void **)&w.U, sizeof(float) * (size_t)m * d, st) ||
                  tmp_alloc((void **)&w.V, sizeof(float) * (size_t)n * d, st)))
        return fail(LV_ERR_OOM, "ood_loss: allocation failed");
    int rc = launch_project_fp32(Q, m, D, A, d, w.Qp, d, st);
    if (rc) return rc;
    return launch_project_fp32(X, n, D, B, d, w.Xp, d, st);
}

static void pair_free(PairWork &w, cudaStream_t st) {
    tmp_free(w.Up, st);
    tmp_free(w.Gp, st);
    tmp_free(w.Qp, st);
    tmp_free(w.Xp, st);
    tmp_free(w.U, st);
    tmp_free(w.V, st);
    tmp_free(w.part, st);
}

// Gradients on the tensor cores (D % 8 == 0, d <= 128):
//   Q' = Q A^T, Qt = Q - Q' B (so that r_ij = qt_j^T x_i carries no cancellation), X' = X B^T;
//   U = R X' and V = R^T Q' by pair_flash: every residual tile is recomputed from Qt and X
//   (bf16x3 products in TMEM) and contracted there with X' or Q' (tf32x3), never stored -- the
//   scratch is O((m + n) D + splits (m + n) d), with no m x n term; the column ranges' partial
//   slots are summed in order;
//   dL/dA = c U^T Q, dL/dB = c V^T X (tf32x3 GEMMs, the D-wide side as M, K = m or n split over
//   the SMs), c = -2 scale / (n m).
static int ood_loss_bwd_tc(const float *A, const float *B, const float *Q, int64_t m, const float *X, int64_t n, int D,
                           int d, float scale, float *gA, float *gB, cudaStream_t st) {
    const int64_t ldm = round_up(m, 4), ldn = round_up(n, 4);
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // column splits of the two passes, their partial slots capped at 512 MB each
    const int64_t cap = (int64_t)512 << 20;
    int cu = 0, cv = 0;
    const int su = pair_flash_splits(m, n, sms, (int)std::max<int64_t>(1, cap / (4 * m * d)), &cu);
    const int sv = pair_flash_splits(n, m, sms, (int)std::max<int64_t>(1, cap / (4 * n * d)), &cv);
    const int sa = gemm_t_tf32_splits(D, d, m), sb = gemm_t_tf32_splits(D, d, n);
    const bool proj_tc = project_bf16_fused_ok(X, D, d);
    float *Qp = nullptr, *Bt = nullptr, *QB = nullptr, *Qt = nullptr, *Xp = nullptr, *XpTh = nullptr,
          *XpTl = nullptr, *QpTh = nullptr, *QpTl = nullptr, *Up = nullptr, *Vp = nullptr, *U = nullptr, *V = nullptr,
          *Pw = nullptr, *Gp = nullptr;
    __nv_bfloat16 *Qbh = nullptr, *Qbl = nullptr, *Xbh = nullptr, *Xbl = nullptr;
    int *status = nullptr, h = 0;
    int rc = LV_OK;
    auto grab = [&](float **p, int64_t count) {
        if (rc == LV_OK && tmp_alloc((void **)p, sizeof(float) * (size_t)count, st))
            rc = fail(LV_ERR_OOM, "ood_loss_bwd: allocation failed");
    };
    auto grab16 = [&](__nv_bfloat16 **p, int64_t count) {
        if (rc == LV_OK && tmp_alloc((void **)p, sizeof(__nv_bfloat16) * (size_t)count, st))
            rc = fail(LV_ERR_OOM, "ood_loss_bwd: allocation failed");
    };
    const size_t pw_bytes = proj_tc ? project_tc_ws_bytes(LV_PREC_TF32X3, n, D, d, X) : 0;
    grab(&Qp, m * d);
    grab(&Bt, (int64_t)d * D);
    grab(&QB, m * D);
    grab(&Qt, m * D);
    grab16(&Qbh, m * D);
    grab16(&Qbl, m * D);
    grab16(&Xbh, n * D);
    grab16(&Xbl, n * D);
    grab(&Xp, n * d);
    grab(&XpTh, d * ldn);
    grab(&XpTl, d * ldn);
    grab(&QpTh, d * ldm);
    grab(&QpTl, d * ldm);
    grab(&Up, su * m * d);
    grab(&Vp, sv * n * d);
    grab(&U, m * d);
    grab(&V, n * d);
    grab(&Pw, (int64_t)(pw_bytes + 3) / 4);
    if (rc == LV_OK && tmp_alloc((void **)&status, sizeof(int), st))
        rc = fail(LV_ERR_OOM, "ood_loss_bwd: allocation failed");
    if (rc == LV_OK && cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
        rc = fail(LV_ERR_CUDA, "ood_loss_bwd: memset failed");
    if (rc == LV_OK) rc = launch_project_fp32(Q, m, D, A, d, Qp, d, st);  // Q'
    if (rc == LV_OK) {
        transpose_kernel<<<(unsigned)(((int64_t)d * D + 255) / 256), 256, 0, st>>>(B, d, D, Bt);
        rc = launch_project_fp32(Qp, m, d, Bt, D, QB, D, st);  // Q' B
    }
    if (rc == LV_OK &&
        cudaMemcpyAsync(Qt, Q, sizeof(float) * (size_t)m * D, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        rc = fail(LV_ERR_CUDA, "ood_loss_bwd: copy failed");
    if (rc == LV_OK) {
        sub_inplace_kernel<<<(unsigned)(((int64_t)m * D + 255) / 256), 256, 0, st>>>(Qt, QB, (int64_t)m * D);
        rc = launch_bf16_split(Qt, m * D, Qbh, Qbl, st);
    }
    if (rc == LV_OK) rc = launch_bf16_split(X, n * D, Xbh, Xbl, st);
    if (rc == LV_OK) {  // X'
        if (proj_tc) {
            void *ws = Pw;
            size_t have = pw_bytes;
            rc = project_tf32x3(X, n, D, B, d, Xp, d, &ws, &have, status, st);
        } else {
            rc = launch_project_fp32(X, n, D, B, d, Xp, d, st);
        }
    }
    if (rc == LV_OK) rc = launch_transpose_tf32_split(Xp, n, d, XpTh, XpTl, ldn, st);
    if (rc == LV_OK) rc = launch_transpose_tf32_split(Qp, m, d, QpTh, QpTl, ldm, st);
    // U (m x d) = R X': rows Qt, columns X; V (n x d) = R^T Q': rows X, columns Qt
    if (rc == LV_OK) rc = pair_flash(Qbh, Qbl, m, Xbh, Xbl, n, D, XpTh, XpTl, ldn, d, su, cu, Up, status, st);
    if (rc == LV_OK) rc = pair_flash(Xbh, Xbl, n, Qbh, Qbl, m, D, QpTh, QpTl, ldm, d, sv, cv, Vp, status, st);
    auto sum = [&](const float *part, int splits, int64_t len, float *out, float sc) {
        split_sum_kernel<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(part, splits, len, out, sc);
    };
    if (rc == LV_OK) {
        sum(Up, su, m * d, U, 1.f);
        sum(Vp, sv, n * d, V, 1.f);
    }
    // the gradient products reuse the passes' memory: Q^T, U^T, X^T, V^T as tf32 pairs
    for (float *p : {Up, Vp}) tmp_free(p, st);
    for (__nv_bfloat16 *p : {Qbh, Qbl, Xbh, Xbl}) tmp_free(p, st);
    Up = Vp = nullptr;
    Qbh = Qbl = Xbh = Xbl = nullptr;
    float *QTh = nullptr, *QTl = nullptr, *UTh = nullptr, *UTl = nullptr, *XTh = nullptr, *XTl = nullptr,
          *VTh = nullptr, *VTl = nullptr;
    grab(&QTh, D * ldm);
    grab(&QTl, D * ldm);
    grab(&UTh, d * ldm);
    grab(&UTl, d * ldm);
    grab(&XTh, D * ldn);
    grab(&XTl, D * ldn);
    grab(&VTh, d * ldn);
    grab(&VTl, d * ldn);
    grab(&Gp, (int64_t)std::max(sa, sb) * d * D);
    const float c = (float)(-2.0 * (double)scale / ((double)n * (double)m));
    if (rc == LV_OK) rc = launch_transpose_tf32_split(Q, m, D, QTh, QTl, ldm, st);
    if (rc == LV_OK) rc = launch_transpose_tf32_split(U, m, d, UTh, UTl, ldm, st);
    if (rc == LV_OK)  // (Q^T U)^T = U^T Q: M = D, N = d, K = m
        rc = gemm_t_tf32(QTh, QTl, D, ldm, UTh, UTl, d, ldm, m, Gp, D, (int64_t)d * D, 0, sa, status, st);
    if (rc == LV_OK) sum(Gp, sa, (int64_t)d * D, gA, c);
    if (rc == LV_OK) rc = launch_transpose_tf32_split(X, n, D, XTh, XTl, ldn, st);
    if (rc == LV_OK) rc = launch_transpose_tf32_split(V, n, d, VTh, VTl, ldn, st);
    if (rc == LV_OK)  // V^T X: M = D, N = d, K = n
        rc = gemm_t_tf32(XTh, XTl, D, ldn, VTh, VTl, d, ldn, n, Gp, D, (int64_t)d * D, 0, sb, status, st);
    if (rc == LV_OK) sum(Gp, sb, (int64_t)d * D, gB, c);
    if (rc == LV_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "ood_loss_bwd kernels");
    }
    if (rc == LV_OK && (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
        rc = fail(LV_ERR_CUDA, "ood_loss_bwd: sync failed");
    if (rc == LV_OK && h) rc = fail(LV_ERR_TIMEOUT, "ood_loss_bwd: a tensor-core pipeline wait timed out");
    for (float *p : {Qp, Bt, QB, Qt, Xp, XpTh, XpTl, QpTh, QpTl, U, V, Pw, Gp, QTh, QTl, UTh, UTl, XTh, XTl, VTh,
                     VTl})
        tmp_free(p, st);
    tmp_free(status, st);
    return rc;
}

}  // namespace lv

using namespace lv;

extern "C" {

int leanvec_ood_loss_fwd(const float *A, const float *B, const float *Q, int64_t m, const float *X, int64_t n, int D,
                         int d, double *loss, lv_stream_t stream) {
    if (!A || !B || !Q || !X || !loss || m <= 0 || n <= 0 || D <= 0 || d <= 0)
        return fail(LV_ERR_ARG, "ood_loss_fwd: invalid sizes or null pointer");
    if (d > DMAX) return fail(LV_ERR_ARG, "ood_loss_fwd: d <= 256 is supported");
    cudaStream_t st = (cudaStream_t)stream;
    if (D % 4 == 0 && m < (1ll << 31) && n < (1ll << 31)) {
        // tensor-core form: r_ij = qt_j^T x_i with qt_j = q_j - B^T (A q_j) (float32); the tile
        // products (three tf32 MMAs on hi / lo splits) and their squares summed by tcgen05 MMAs and
        // the epilogue; FP64 partials summed in order
        float *Qp = nullptr, *Bt = nullptr, *Qt = nullptr, *QB = nullptr, *Qh = nullptr, *Xh = nullptr,
              *Xl = nullptr;
        double *part = nullptr;
        int *status = nullptr, h = 0, np = 0;
        int rc = pair_sq_tf32(nullptr, nullptr, m, nullptr, nullptr, n, D, nullptr, &np, nullptr, st);  // count
        const int64_t np_alloc = std::max(np, 1);
        if (rc == LV_OK &&
            (tmp_alloc((void **)&Qp, sizeof(float) * (size_t)m * d, st) ||
             tmp_alloc((void **)&Bt, sizeof(float) * (size_t)d * D, st) ||
             tmp_alloc((void **)&Qt, sizeof(float) * (size_t)m * D, st) ||
             tmp_alloc((void **)&QB, sizeof(float) * (size_t)m * D, st) ||
             tmp_alloc((void **)&Qh, sizeof(float) * (size_t)m * D, st) ||
             tmp_alloc((void **)&Xh, sizeof(float) * (size_t)n * D, st) ||
             tmp_alloc((void **)&Xl, sizeof(float) * (size_t)n * D, st) ||
             tmp_alloc((void **)&part, sizeof(double) * (size_t)np_alloc, st) ||
             tmp_alloc((void **)&status, sizeof(int), st)))
            rc = fail(LV_ERR_OOM, "ood_loss_fwd: allocation failed");
        if (rc == LV_OK) rc = launch_project_fp32(Q, m, D, A, d, Qp, d, st);  // A q
        if (rc == LV_OK) {
            transpose_kernel<<<(unsigned)(((int64_t)d * D + 255) / 256), 256, 0, st>>>(B, d, D, Bt);
            rc = launch_project_fp32(Qp, m, d, Bt, D, QB, D, st);  // B^T A q
        }
        if (rc == LV_OK && cudaMemcpyAsync(Qt, Q, sizeof(float) * (size_t)m * D, cudaMemcpyDeviceToDevice, st) !=
                               cudaSuccess)
            rc = fail(LV_ERR_CUDA, "ood_loss_fwd: copy failed");
        if (rc == LV_OK) {
            sub_inplace_kernel<<<(unsigned)(((int64_t)m * D + 255) / 256), 256, 0, st>>>(Qt, QB, (int64_t)m * D);
            if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) rc = fail(LV_ERR_CUDA, "memset failed");
        }
        if (rc == LV_OK) rc = launch_tf32_split(Qt, (int64_t)m * D, Qh, QB, st);  // QB now holds the lo part
        if (rc == LV_OK) rc = launch_tf32_split(X, (int64_t)n * D, Xh, Xl, st);
        if (rc == LV_OK) rc = pair_sq_tf32(Qh, QB, m, Xh, Xl, n, D, part, &np, status, st);
        std::vector<double> hp(np_alloc, 0.0);
        if (rc == LV_OK && (cudaMemcpyAsync(hp.data(), part, sizeof(double) * np, cudaMemcpyDeviceToHost, st) !=
                                cudaSuccess ||
                            cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                            cudaStreamSynchronize(st) != cudaSuccess))
            rc = fail(LV_ERR_CUDA, "ood_loss_fwd: reduction copy failed");
        if (rc == LV_OK && h) rc = fail(LV_ERR_TIMEOUT, "ood_loss_fwd: a tensor-core pipeline wait timed out");
        if (rc == LV_OK) {
            double s = 0.0;
            for (double v : hp) s += v;  // fixed order
            *loss = s / ((double)n * (double)m);
        }
        for (void *p : {(void *)Qp, (void *)Bt, (void *)Qt, (void *)QB, (void *)Qh, (void *)Xh, (void *)Xl, (void *)part,
                        (void *)status})
            tmp_free(p, st);
        return rc;
    }
    PairWork w;
    int rc = pair_prepare(A, B, Q, m, X, n, D, d, w, false, st);
    const int nb = (int)((m + PT - 1) / PT);
    const int sp = sweep_splits(nb, n);  // column splits of the database
    std::vector<double> part((size_t)nb * sp);
    if (rc == LV_OK) {
        pair_sweep_kernel<false><<<dim3(nb, sp), 256, 0, st>>>(Q, w.Qp, m, X, w.Xp, n, D, d, split_len(n, sp, PT),
                                                               w.part, nullptr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "pair_sweep_kernel");
    }
    if (rc == LV_OK && (cudaMemcpyAsync(part.data(), w.part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
        rc = fail(LV_ERR_CUDA, "ood_loss_fwd: reduction copy failed");
    if (rc == LV_OK) {
        double s = 0.0;
        for (double v : part) s += v;  // fixed order
        *loss = s / ((double)n * (double)m);
    }
    pair_free(w, st);
    return rc;
}

int leanvec_ood_loss_bwd(const float *A, const float *B, const float *Q, int64_t m, const float *X, int64_t n, int D,
                         int d, float scale, float *gA, float *gB, lv_stream_t stream) {
    if (!A || !B || !Q || !X || !gA || !gB || m <= 0 || n <= 0 || D <= 0 || d <= 0)
        return fail(LV_ERR_ARG, "ood_loss_bwd: invalid sizes or null pointer");
    if (d > DMAX) return fail(LV_ERR_ARG, "ood_loss_bwd: d <= 256 is supported");
    cudaStream_t st = (cudaStream_t)stream;
    if (D % 8 == 0 && d <= 128 && m < (1ll << 31) && n < (1ll << 31))
        return ood_loss_bwd_tc(A, B, Q, m, X, n, D, d, scale, gA, gB, st);
    PairWork w;
    int rc = pair_prepare(A, B, Q, m, X, n, D, d, w, true, st);
    // U = R X' (query tiles, the database split in column ranges whose partials are summed in
    // order), V = R^T Q' (database tiles: rows X, cols Q, residual sign unchanged); the gradient
    // GEMMs split their rows the same way
    const int64_t tq = (m + PT - 1) / PT, tx = (n + PT - 1) / PT;
    const int su = sweep_splits(tq, n), sv = sweep_splits(tx, m);
    const int cb = (D + 63) / 64;
    const int sa = sweep_splits(cb, m), sb = sweep_splits(cb, n);
    if (rc == LV_OK && (tmp_alloc((void **)&w.Up, sizeof(float) * (size_t)std::max(su, sv) * std::max(m, n) * d, st) ||
                        tmp_alloc((void **)&w.Gp, sizeof(float) * (size_t)std::max(sa, sb) * d * D, st)))
        rc = fail(LV_ERR_OOM, "ood_loss_bwd: allocation failed");
    if (rc == LV_OK) {
        const float c = (float)(-2.0 * (double)scale / ((double)n * (double)m));
        auto sum = [&](const float *part, int splits, int64_t len, float *out) {
            split_sum_kernel<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(part, splits, len, out, 1.f);
        };
        pair_sweep_kernel<true><<<dim3((unsigned)tq, su), 256, 0, st>>>(Q, w.Qp, m, X, w.Xp, n, D, d,
                                                                        split_len(n, su, PT), nullptr, w.Up);
        sum(w.Up, su, m * d, w.U);
        pair_sweep_kernel<true><<<dim3((unsigned)tx, sv), 256, 0, st>>>(X, w.Xp, n, Q, w.Qp, m, D, d,
                                                                        split_len(m, sv, PT), nullptr, w.Up);
        sum(w.Up, sv, n * d, w.V);
        tgemm_kernel<<<dim3(cb, sa), 256, 0, st>>>(w.U, Q, m, split_len(m, sa, 32), d, D, c, w.Gp);
        sum(w.Gp, sa, (int64_t)d * D, gA);
        tgemm_kernel<<<dim3(cb, sb), 256, 0, st>>>(w.V, X, n, split_len(n, sb, 32), d, D, c, w.Gp);
        sum(w.Gp, sb, (int64_t)d * D, gB);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "ood_loss_bwd kernels");
    }
    if (rc == LV_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(LV_ERR_CUDA, "ood_loss_bwd: sync failed");
    pair_free(w, st);
    return rc;
}

}  // extern "C"
