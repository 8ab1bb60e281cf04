// The nout leading eigenpairs of a symmetric FP64 matrix.  LeanVec-ID (Sec. 2.1) and the
// eigenvector search (Algorithm 2) use only the d leading eigenvectors of a D x D second moment,
// so instead of diagonalising the whole matrix (cyclic Jacobi, fit.cu) this path
//   1. reduces K to tridiagonal form T = Q^T K Q by D - 2 Householder reflections (one persistent
//      kernel, all SMs, one grid barrier per reflection);
//   2. finds the nout largest eigenvalues of T by multisection on Sturm counts (one warp each);
//   3. finds their eigenvectors of T by inverse iteration on the pivoted tridiagonal factorisation
//      of T - lambda I, with Gram-Schmidt inside clusters of close eigenvalues (one block per
//      cluster);
//   4. maps them back through the reflections (x = Q z, one warp per eigenvector) and fixes the
//      sign (largest-magnitude entry positive, first index on ties).
// FP64 throughout.  Every grid-wide wait is bounded: a block that waits too long records
// ST_TIMEOUT and returns.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace lv {

constexpr int TRI_THREADS = 256, TRI_WARPS = TRI_THREADS / 32;
constexpr long long TRI_SPIN = 1ll << 25;  // with a 64 ns sleep per try: a give-up within seconds
constexpr int EIGH_TOP_MAX_D = 4096;

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// sum over the block in a fixed order (the same in every block for the same data)
__device__ double block_sum_d(double x, double *red) {
    x = warp_sum_d(x);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    double t = 0.0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) t += red[i];
    __syncthreads();
    return t;
}

// Grid barrier on a cumulative arrival counter: barrier number `target` completes when
// gridDim.x * target blocks have arrived.  False when this block gave up waiting.
__device__ bool grid_barrier(unsigned *count, volatile unsigned *gen, unsigned &target) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        ++target;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u) + 1u;
        if (arrived == gridDim.x * target) {
            __threadfence();
            atomicExch(const_cast<unsigned *>(gen), target);
        } else {
            long long it = 0;
            while (*gen < target) {
                if (++it > TRI_SPIN) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// Householder tridiagonalisation of the symmetric D x D matrix A (device, full storage).  Reflection
// k (k = 0 .. D - 3) maps the column below the diagonal, x = A^(k)[k + 1 .., k], to (beta, 0, ..):
// H_k = I - tau_k v_k v_k^T with v_k[0] = 1, stored as Hv[k][k + 1 ..].  The trailing matrix
// changes by A^(k+1) = A^(k) - v w^T - w v^T with p = tau A^(k) v, w = p - (tau / 2)(p . v) v.
// That update is applied one step late, inside the next step's pass over the rows, so that a
// step needs one grid barrier: step k rebuilds row k of A^(k) from the stored row and the pending
// (v, w) of step k - 1, forms v_k, then each block updates its rows (owner = row % gridDim.x, one
// warp per row), writes them back and forms their entries of p = tau_k A^(k) v_k; after the barrier
// every block forms w_k.  Outputs: diagonal dg (D), off-diagonal ofd (D - 1), Hv, tau.  Everything
// that crosses blocks goes through L2 (ld.cg / st.cg).
__global__ void __launch_bounds__(TRI_THREADS) tridiag_kernel(double *A, int D, double *dg, double *ofd,
                                                               double *Hv, double *tau, double *pbuf,
                                                               unsigned *bar_count, unsigned *bar_gen, int *status) {
    extern __shared__ double sh[];
    double *vp = sh, *wp = sh + D, *vc = sh + 2 * D, *red = sh + 3 * D;  // global row indices
    const int G = (int)gridDim.x, c = (int)blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned target = 0;
    for (int g = tid; g < D; g += TRI_THREADS) vp[g] = wp[g] = 0.0;
    __syncthreads();
    for (int k = 0; k + 2 < D; ++k) {
        const double *rowk = A + (int64_t)k * D;
        const double vk = vp[k], wk = wp[k];
        // x_j = A^(k)[k][j], j > k: the stored row k with step k - 1's update
        double s = 0.0;
        for (int j = k + 2 + tid; j < D; j += TRI_THREADS) {
            const double xj = __ldcg(rowk + j) - vk * wp[j] - wk * vp[j];
            vc[j] = xj;
            s = fma(xj, xj, s);
        }
        const double xn2 = block_sum_d(s, red);
        const double x0 = __ldcg(rowk + k + 1) - vk * wp[k + 1] - wk * vp[k + 1];
        double beta = x0, t = 0.0, scal = 0.0;
        if (xn2 > 0.0) {
            beta = -copysign(sqrt(fma(x0, x0, xn2)), x0);
            t = (beta - x0) / beta;
            scal = 1.0 / (x0 - beta);
        }
        for (int j = k + 1 + tid; j < D; j += TRI_THREADS) vc[j] = j == k + 1 ? 1.0 : vc[j] * scal;
        __syncthreads();
        if (c == 0) {
            for (int j = k + 1 + tid; j < D; j += TRI_THREADS) Hv[(int64_t)k * D + j] = vc[j];
            if (tid == 0) {
                tau[k] = t;
                ofd[k] = beta;
                dg[k] = __ldcg(rowk + k) - 2.0 * vk * wk;
            }
        }
        // rows i > k of this block: apply step k - 1's update, store, p_i = t (row_i . v_k)
        const int first = k + 1 + (((c - (k + 1)) % G) + G) % G;
        for (int i = first + wid * G; i < D; i += TRI_WARPS * G) {
            double *ar = A + (int64_t)i * D;
            const double vi = vp[i], wi = wp[i];
            double acc = 0.0;
            for (int j = k + 1 + lane; j < D; j += 32) {
                const double a = __ldcg(ar + j) - vi * wp[j] - wi * vp[j];
                __stcg(ar + j, a);
                acc = fma(a, vc[j], acc);
            }
            acc = warp_sum_d(acc);
            if (lane == 0) __stcg(pbuf + i, t * acc);
        }
        if (!grid_barrier(bar_count, bar_gen, target)) {
            if (tid == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        // w_k = p - (t / 2)(p . v_k) v_k, pending for the next step
        double pv = 0.0;
        for (int j = k + 1 + tid; j < D; j += TRI_THREADS) pv = fma(__ldcg(pbuf + j), vc[j], pv);
        pv = block_sum_d(pv, red);
        const double gam = 0.5 * t * pv;
        for (int j = k + 1 + tid; j < D; j += TRI_THREADS) {
            wp[j] = fma(-gam, vc[j], __ldcg(pbuf + j));
            vp[j] = vc[j];
        }
        __syncthreads();
    }
    if (c == 0 && tid == 0) {
        const int a = D - 2, b2 = D - 1;
        dg[a] = __ldcg(A + (int64_t)a * D + a) - 2.0 * vp[a] * wp[a];
        ofd[a] = __ldcg(A + (int64_t)a * D + b2) - vp[a] * wp[b2] - wp[a] * vp[b2];
        dg[b2] = __ldcg(A + (int64_t)b2 * D + b2) - 2.0 * vp[b2] * wp[b2];
        tau[a] = 0.0;
    }
}

// number of eigenvalues of T below x (Sturm count of the LDL^T pivots of T - x I)
__device__ int sturm_below(const double *dg, const double *ofd, int D, double x, double pivmin) {
    double q = dg[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    int neg = q < 0.0;
    for (int j = 1; j < D; ++j) {
        q = dg[j] - x - ofd[j - 1] * ofd[j - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        neg += q < 0.0;
    }
    return neg;
}

// lam[i] = the (i + 1)-th largest eigenvalue of T, i < nout; one warp per eigenvalue.  Each round
// lanes 0 .. 30 count at 31 interior points of [lo, hi] (a point at or below lo counts as holding
// the invariant, one at or above hi as not), and the interval shrinks to the two neighbouring points
// around the change, until it no longer shrinks.
__global__ void bisect_kernel(const double *dg, const double *ofd, int D, int nout, double lo0, double hi0,
                              double pivmin, double *lam) {
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= nout) return;  // whole warps
    double lo = lo0, hi = hi0;
    for (int round = 0; round < 64; ++round) {
        const double x = lo + (hi - lo) * ((double)(lane + 1) / 32.0);
        bool pred;
        if (lane == 31 || x >= hi)
            pred = false;
        else if (x <= lo)
            pred = true;
        else
            pred = D - sturm_below(dg, ofd, D, x, pivmin) >= i + 1;
        const unsigned bal = __ballot_sync(FULL, pred);
        const int nt = __popc(bal);  // the true lanes are a prefix (counts fall as x grows)
        const double xl = __shfl_sync(FULL, x, max(nt - 1, 0)), xh = __shfl_sync(FULL, x, min(nt, 31));
        const double nlo = nt > 0 ? fmax(lo, xl) : lo, nhi = nt < 31 ? fmin(hi, xh) : hi;
        if (nlo == lo && nhi == hi) break;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) lam[i] = 0.5 * (lo + hi);
}

// a deterministic start vector entry in [-1, 1)
__device__ __forceinline__ double start_entry(int i, int e) {
    unsigned h = (unsigned)i * 0x9E3779B1u ^ ((unsigned)e + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    return (double)(h >> 8) * (2.0 / 16777216.0) - 1.0;
}

// Inverse iteration, one block per cluster [cb[c], ce[c]) of eigenvalues (descending, close ones
// together).  For eigenvalue e: T - lam I = P L U by Gaussian elimination with partial pivoting
// (thread 0; pivots below tol replaced by +-tol, stored as reciprocals), then: solve, orthogonalise
// against the cluster's earlier vectors (modified Gram-Schmidt), normalise -- three rounds (the
// eigenvalue is accurate to the last bits, so one solve already nearly converges).  Z: nout x D.
// scratch: 5 D doubles and D ints per cluster.
__global__ void __launch_bounds__(128) inviter_kernel(const double *dg, const double *ofd, int D, const double *lam,
                                                      const int *cb, const int *ce, double tol, double *Z,
                                                      double *scratch, int *piv_all) {
    __shared__ double red[4];
    const int c = blockIdx.x, tid = threadIdx.x;
    double *dl = scratch + (size_t)c * 5 * D, *dd = dl + D, *du = dd + D, *du2 = du + D, *x = du2 + D;
    int *piv = piv_all + (size_t)c * D;
    for (int e = cb[c]; e < ce[c]; ++e) {
        // distinct shifts inside a cluster (equal eigenvalues would give the same vector)
        double le = lam[e];
        if (e > cb[c]) le = fmin(le, lam[e - 1] - 4.0 * DBL_EPSILON * fabs(lam[e - 1]) - tol * 1e-3);
        if (tid == 0) {
            for (int j = 0; j < D; ++j) {
                dd[j] = dg[j] - le;
                if (j + 1 < D) dl[j] = du[j] = ofd[j];
                du2[j] = 0.0;
            }
            for (int j = 0; j + 1 < D; ++j) {
                if (fabs(dd[j]) >= fabs(dl[j])) {
                    if (fabs(dd[j]) < tol) dd[j] = dd[j] < 0.0 ? -tol : tol;
                    const double mult = dl[j] / dd[j];
                    dl[j] = mult;
                    dd[j + 1] -= mult * du[j];
                    piv[j] = 0;
                } else {
                    const double mult = dd[j] / dl[j];
                    dd[j] = dl[j];
                    const double tmp = dd[j + 1];
                    dd[j + 1] = du[j] - mult * tmp;
                    if (j + 2 < D) {
                        du2[j] = du[j + 1];
                        du[j + 1] = -mult * du2[j];
                    }
                    du[j] = tmp;
                    dl[j] = mult;
                    piv[j] = 1;
                }
            }
            if (fabs(dd[D - 1]) < tol) dd[D - 1] = dd[D - 1] < 0.0 ? -tol : tol;
            for (int j = 0; j < D; ++j) dd[j] = 1.0 / dd[j];  // the solves multiply
        }
        for (int i = tid; i < D; i += blockDim.x) x[i] = start_entry(i, e);
        __syncthreads();
        for (int round = 0; round < 3; ++round) {
            if (tid == 0) {
                for (int j = 0; j + 1 < D; ++j) {
                    if (piv[j]) {
                        const double tmp = x[j];
                        x[j] = x[j + 1];
                        x[j + 1] = tmp - dl[j] * x[j];
                    } else {
                        x[j + 1] -= dl[j] * x[j];
                    }
                }
                x[D - 1] *= dd[D - 1];
                x[D - 2] = (x[D - 2] - du[D - 2] * x[D - 1]) * dd[D - 2];
                for (int j = D - 3; j >= 0; --j) x[j] = (x[j] - du[j] * x[j + 1] - du2[j] * x[j + 2]) * dd[j];
            }
            __syncthreads();
            for (int f = cb[c]; f < e; ++f) {
                const double *zf = Z + (size_t)f * D;
                double s = 0.0;
                for (int i = tid; i < D; i += blockDim.x) s = fma(zf[i], x[i], s);
                s = block_sum_d(s, red);
                for (int i = tid; i < D; i += blockDim.x) x[i] = fma(-s, zf[i], x[i]);
                __syncthreads();
            }
            double s = 0.0;
            for (int i = tid; i < D; i += blockDim.x) s = fma(x[i], x[i], s);
            s = block_sum_d(s, red);
            const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
            for (int i = tid; i < D; i += blockDim.x) x[i] *= inv;
            __syncthreads();
        }
        double *ze = Z + (size_t)e * D;
        for (int i = tid; i < D; i += blockDim.x) ze[i] = x[i];
        __syncthreads();
    }
}

// evecs[r] = Q z_r = H_0 H_1 .. H_{D-3} z_r, unit norm, largest-magnitude entry positive (first
// index on ties); evals[r] = lam[r] (evals nullable).  One warp per eigenvector.
__global__ void __launch_bounds__(32) backtrans_kernel(const double *Z, const double *Hv, const double *tau, int D,
                                                       const double *lam, double *evals, double *evecs) {
    extern __shared__ double sx[];
    const int r = blockIdx.x, lane = threadIdx.x;
    for (int i = lane; i < D; i += 32) sx[i] = Z[(size_t)r * D + i];
    __syncwarp();
    for (int k = D - 3; k >= 0; --k) {
        const double t = tau[k];
        if (t == 0.0) continue;
        const double *vk = Hv + (int64_t)k * D;
        double s = 0.0;
        for (int i = k + 1 + lane; i < D; i += 32) s = fma(vk[i], sx[i], s);
        s = warp_sum_d(s) * t;
        for (int i = k + 1 + lane; i < D; i += 32) sx[i] = fma(-s, vk[i], sx[i]);
        __syncwarp();
    }
    double s = 0.0, best = -1.0;
    int bi = D;
    for (int i = lane; i < D; i += 32) {
        s = fma(sx[i], sx[i], s);
        const double a = fabs(sx[i]);
        if (a > best) {
            best = a;
            bi = i;
        }
    }
    s = warp_sum_d(s);
    // largest |x_i|, first index on ties
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_xor_sync(FULL, best, o);
        const int oi = __shfl_xor_sync(FULL, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    const double scale = (s > 0.0 ? 1.0 / sqrt(s) : 0.0) * (bi < D && sx[bi] < 0.0 ? -1.0 : 1.0);
    for (int i = lane; i < D; i += 32) evecs[(size_t)r * D + i] = sx[i] * scale;
    if (lane == 0 && evals) evals[r] = lam[r];
}

// the path applies: 8 <= D <= 4096, 1 <= nout <= D
bool eigh_top_ok(int D, int nout) { return D >= 8 && D <= EIGH_TOP_MAX_D && nout >= 1 && nout <= D; }

int eigh_top(const double *K, int D, int nout, double *evals, double *evecs, cudaStream_t st) {
    if (!eigh_top_ok(D, nout)) return fail(LV_ERR_ARG, "eigh_top: need 8 <= D <= 4096 and 1 <= nout <= D");
    double *A = nullptr, *Hv = nullptr, *tau = nullptr, *dg = nullptr, *ofd = nullptr, *pbuf = nullptr;
    double *lam = nullptr, *Z = nullptr, *scr = nullptr;
    unsigned *bar = nullptr;
    int *status = nullptr, *cl = nullptr, *piv = nullptr;
    int rc = LV_OK;
    const size_t DD = (size_t)D * D;
    std::vector<double> hd(D), he(D), hl(nout);
    std::vector<int> hcb, hce;
    int dev = 0, sms = 0, per_sm = 0, nclus = 0, hstatus = 0;
    const size_t tsm = sizeof(double) * (3 * (size_t)D + TRI_WARPS);
    if (tmp_alloc((void **)&A, sizeof(double) * DD, st) || tmp_alloc((void **)&Hv, sizeof(double) * DD, st) ||
        tmp_alloc((void **)&tau, sizeof(double) * D, st) || tmp_alloc((void **)&dg, sizeof(double) * D, st) ||
        tmp_alloc((void **)&ofd, sizeof(double) * D, st) || tmp_alloc((void **)&pbuf, sizeof(double) * D, st) ||
        tmp_alloc((void **)&lam, sizeof(double) * nout, st) || tmp_alloc((void **)&Z, sizeof(double) * nout * (size_t)D, st) ||
        tmp_alloc((void **)&bar, 2 * sizeof(unsigned), st) || tmp_alloc((void **)&status, sizeof(int), st)) {
        rc = fail(LV_ERR_OOM, "eigh_top: allocation failed");
        goto done;
    }
    if (cudaMemcpyAsync(A, K, sizeof(double) * DD, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) {
        rc = fail(LV_ERR_CUDA, "eigh_top: copy failed");
        goto done;
    }
    // 1. tridiagonal form: one block per SM, all co-resident (cooperative launch)
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_kernel, TRI_THREADS, tsm) != cudaSuccess ||
        per_sm < 1) {
        rc = fail(LV_ERR_CUDA, "eigh_top: cannot size the tridiagonalisation");
        goto done;
    }
    {
        int Dv = D;
        unsigned *bar_gen = bar + 1;
        void *args[] = {&A, &Dv, &dg, &ofd, &Hv, &tau, &pbuf, &bar, &bar_gen, &status};
        if (cudaLaunchCooperativeKernel((const void *)tridiag_kernel, dim3((unsigned)sms), dim3(TRI_THREADS), args, tsm,
                                        st) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(LV_ERR_CUDA, "eigh_top: tridiagonalisation launch failed");
            goto done;
        }
    }
    if (cudaMemcpyAsync(hd.data(), dg, sizeof(double) * D, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(he.data(), ofd, sizeof(double) * (D - 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        rc = fail(LV_ERR_CUDA, "eigh_top: tridiagonalisation failed");
        goto done;
    }
    if (hstatus) {
        rc = fail(LV_ERR_TIMEOUT, "eigh_top: a grid barrier of the tridiagonalisation timed out");
        goto done;
    }
    {
        // 2. eigenvalues: Gershgorin interval, pivot floor as in the usual Sturm-count bisection
        double lo = hd[0], hi = hd[0], e2max = 0.0;
        for (int j = 0; j < D; ++j) {
            const double r = (j > 0 ? fabs(he[j - 1]) : 0.0) + (j + 1 < D ? fabs(he[j]) : 0.0);
            lo = std::min(lo, hd[j] - r);
            hi = std::max(hi, hd[j] + r);
            if (j + 1 < D) e2max = std::max(e2max, he[j] * he[j]);
        }
        const double tnorm = std::max(fabs(lo), fabs(hi));
        const double pad = 4.0 * DBL_EPSILON * tnorm + DBL_MIN;
        lo -= pad;
        hi += pad;
        const double pivmin = DBL_MIN * std::max(1.0, e2max);
        // one warp per block, so that the eigenvalues' warps spread over all SMs
        bisect_kernel<<<nout, 32, 0, st>>>(dg, ofd, D, nout, lo, hi, pivmin, lam);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(hl.data(), lam, sizeof(double) * nout, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "eigh_top: bisection failed");
            goto done;
        }
        // 3. clusters: consecutive eigenvalues closer than 1e-5 ||T||
        const double ctol = 1e-5 * tnorm;
        for (int i = 0; i < nout; ++i) {
            if (i == 0 || hl[i - 1] - hl[i] > ctol) {
                hcb.push_back(i);
                hce.push_back(i + 1);
            } else {
                hce.back() = i + 1;
            }
        }
        nclus = (int)hcb.size();
        if (tmp_alloc((void **)&cl, sizeof(int) * 2 * nclus, st) ||
            tmp_alloc((void **)&scr, sizeof(double) * 5 * (size_t)D * nclus, st) ||
            tmp_alloc((void **)&piv, sizeof(int) * (size_t)D * nclus, st)) {
            rc = fail(LV_ERR_OOM, "eigh_top: allocation failed");
            goto done;
        }
        if (cudaMemcpyAsync(cl, hcb.data(), sizeof(int) * nclus, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(cl + nclus, hce.data(), sizeof(int) * nclus, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "eigh_top: cluster copy failed");
            goto done;
        }
        const double tol = std::max(DBL_EPSILON * tnorm, DBL_MIN);
        inviter_kernel<<<nclus, 128, 0, st>>>(dg, ofd, D, lam, cl, cl + nclus, tol, Z, scr, piv);
        if (cudaGetLastError() != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "eigh_top: inverse iteration launch failed");
            goto done;
        }
        // 4. back to K's basis
        const size_t bsm = sizeof(double) * (size_t)D;
        if (bsm > 48 * 1024 &&
            cudaFuncSetAttribute(backtrans_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm) != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "eigh_top: shared-memory attribute failed");
            goto done;
        }
        backtrans_kernel<<<nout, 32, bsm, st>>>(Z, Hv, tau, D, lam, evals, evecs);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(LV_ERR_CUDA, "eigh_top: back-transformation failed");
            goto done;
        }
    }
done:
    tmp_free(A, st);
    tmp_free(Hv, st);
    tmp_free(tau, st);
    tmp_free(dg, st);
    tmp_free(ofd, st);
    tmp_free(pbuf, st);
    tmp_free(lam, st);
    tmp_free(Z, st);
    tmp_free(bar, st);
    tmp_free(status, st);
    tmp_free(cl, st);
    tmp_free(scr, st);
    tmp_free(piv, st);
    return rc;
}

}  // namespace lv

extern "C" int leanvec_eigh_top(const double *K, int D, int nout, double *evals, double *evecs, lv_stream_t stream) {
    if (!K || !evecs) return lv::fail(LV_ERR_ARG, "eigh_top: null pointer");
    return lv::eigh_top(K, D, nout, evals, evecs, (cudaStream_t)stream);
}
