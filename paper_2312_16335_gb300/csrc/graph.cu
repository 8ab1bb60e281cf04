// Graph construction on the primary vectors (App. A: search + prune for every node;
// App. D: Vamana with R, L, alpha), batch-synchronous and bit-reproducible:
//   1. beam search of every batch node on the graph as it was at the batch start
//      (beam_kernel in build mode, exact integer-core pair scores);
//   2. RobustPrune of pool = beam u old out-list (one CTA per node, pool records
//      staged in shared memory);
//   3. the batch's out-lists are replaced;
//   4. reverse edges grouped by target with a count / scan / scatter pass, each
//      target's sources sorted ascending, appended, and the target pruned if it
//      exceeds R.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "beam.cuh"
#include "common.cuh"
#include "index.cuh"

namespace lv {

// -------------------------------------------------------------------- helpers
static inline float host_fsub(float a, float b) { return a - b; }  // IEEE float32 (host SSE/NEON)
__host__ __device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t a, uint64_t b) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL * (1ULL + (a << 32) + b);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool entry_better(float ga, int ia, float gb, int ib) {
    if (isnan(ga)) return false;
    if (isnan(gb)) return true;
    return ga > gb || (ga == gb && ia < ib);
}

// Remove out-of-range and repeated ids of every row (first occurrence kept).
__global__ void graph_sanitize_kernel(int32_t *g, int64_t n, int R, int *status) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t *row = g + v * R;
    for (int s = 0; s < R; ++s) {
        int32_t u = row[s];
        if (u < -1 || u >= n) {
            atomicOr(status, ST_CORRUPT);
            row[s] = -1;
            continue;
        }
        if (u < 0) continue;
        for (int t = 0; t < s; ++t)
            if (row[t] == u) {
                row[s] = -1;
                break;
            }
    }
}

// argmax_i G_i (ties -> smaller id): G is the third float of the record constants; with the L2
// metric argmax_i 2 G_i - N_i (the primary nearest the mean; N = first float of the second chunk).
__global__ void entry_partial_kernel(const uint8_t *rec, int64_t n, int64_t stride, int cb, int metric, float *bg,
                                     int *bi) {
    __shared__ float sg[256];
    __shared__ int si[256];
    float best = -INFINITY;
    int bid = 0x7fffffff;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float gv = *reinterpret_cast<const float *>(rec + i * stride + cb + 8);
        if (metric) gv = __fsub_rn(__fmul_rn(2.0f, gv), *reinterpret_cast<const float *>(rec + i * stride + cb + 16));
        if (entry_better(gv, (int)i, best, bid) || bid == 0x7fffffff) {
            if (!isnan(gv) || bid == 0x7fffffff) {
                best = isnan(gv) ? -INFINITY : gv;
                bid = (int)i;
            }
        }
    }
    sg[threadIdx.x] = best;
    si[threadIdx.x] = bid;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o && entry_better(sg[threadIdx.x + o], si[threadIdx.x + o], sg[threadIdx.x], si[threadIdx.x])) {
            sg[threadIdx.x] = sg[threadIdx.x + o];
            si[threadIdx.x] = si[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bg[blockIdx.x] = sg[0];
        bi[blockIdx.x] = si[0];
    }
}

__global__ void entry_final_kernel(const float *bg, const int *bi, int nb, int32_t *out) {
    __shared__ float sg[256];
    __shared__ int si[256];
    float best = -INFINITY;
    int bid = 0x7fffffff;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        if (entry_better(bg[t], bi[t], best, bid)) {
            best = bg[t];
            bid = bi[t];
        }
    sg[threadIdx.x] = best;
    si[threadIdx.x] = bid;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o && entry_better(sg[threadIdx.x + o], si[threadIdx.x + o], sg[threadIdx.x], si[threadIdx.x])) {
            sg[threadIdx.x] = sg[threadIdx.x + o];
            si[threadIdx.x] = si[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = si[0] == 0x7fffffff ? 0 : si[0];
}

// Initial graph: node v keeps the first min(R, n-1) draws splitmix(seed, v, j) mod n
// that are neither v nor repeated.
__global__ void random_graph_kernel(int32_t *g, int64_t n, int R, uint64_t seed, int *status) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t *row = g + v * R;
    const int want = (int)((n - 1) < R ? (n - 1) : R);
    int cnt = 0;
    uint64_t j = 0;
    const uint64_t limit = 1ull << 24;
    while (cnt < want) {
        if (j >= limit) {
            atomicOr(status, ST_TIMEOUT);
            break;
        }
        int32_t u = (int32_t)(splitmix(seed, (uint64_t)v, j) % (uint64_t)n);
        ++j;
        if (u == v) continue;
        bool dup = false;
        for (int t = 0; t < cnt; ++t)
            if (row[t] == u) {
                dup = true;
                break;
            }
        if (dup) continue;
        row[cnt++] = u;
    }
    for (int t = cnt; t < R; ++t) row[t] = -1;
}

// --------------------------------------------------------------- RobustPrune
// Pair score of two records held in shared memory (exact build score; L2: -||y_a - y_b||^2).
template <int BITS, bool L2>
__device__ __forceinline__ float smem_pair_score(const uint8_t *ra, const uint8_t *rb, int CH, int cb, float mu2,
                                                 float fdim) {
    int P = 0;
    for (int c = 0; c < CH; ++c)
        P += code_dot<BITS>(*reinterpret_cast<const uint4 *>(ra + 16 * c), *reinterpret_cast<const uint4 *>(rb + 16 * c));
    const float4 ka = *reinterpret_cast<const float4 *>(ra + cb);
    const float4 kb = *reinterpret_cast<const float4 *>(rb + cb);
    const float ip = build_pair_score(mu2, fdim, ka.x, ka.y, ka.z, ka.w, kb.x, kb.y, kb.z, kb.w, P);
    if (!L2) return ip;
    return l2_from_ip(ip, *reinterpret_cast<const float *>(ra + cb + 16), *reinterpret_cast<const float *>(rb + cb + 16));
}

struct PruneParams {
    const uint8_t *prim;
    int64_t stride;  // record stride (multiple of 32)
    int CH, cb, dim;
    float mu2, alpha, shift;
    int metric;  // 1: L2 pair scores -||y_a - y_b||^2
    int R, PMAX;
    int64_t n;
    int32_t *graph;        // n x R
    // mode 0: batch nodes
    const int32_t *nodes;  // perm + b0
    const int32_t *beams;  // nb x Lb
    int Lb;
    int32_t *newl;         // nb x R
    // mode 1: reverse edges
    const int64_t *offs;   // n + 1 exclusive scan (hi: sources, lo: touched count)
    const int32_t *srcs;
    const int32_t *touched;
    const int64_t *total;  // lo 32 bits: number of touched targets
    int *status;
};

// MODE 0: pool = beam (minus p) u old out-list of p; output to newl[t].
// MODE 1: pool = current out-list of u + its new sources (ascending, not present);
//         pruned only when it exceeds R; output to graph[u].
template <int BITS, int MODE, bool L2>
__global__ void __launch_bounds__(128) prune_kernel(const PruneParams pp) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int stride = (int)pp.stride;
    uint8_t *recs = sm;                                              // PMAX records
    uint8_t *prec = recs + (size_t)pp.PMAX * stride;                 // own record
    int *pid = reinterpret_cast<int *>(prec + stride);               // PMAX ids
    float *psc = reinterpret_cast<float *>(pid + pp.PMAX);           // PMAX scores
    int *ord = reinterpret_cast<int *>(psc + pp.PMAX);               // PMAX order
    int *aux = ord + pp.PMAX;                                        // PMAX scratch
    unsigned char *dead = reinterpret_cast<unsigned char *>(aux + pp.PMAX);
    __shared__ int s_np, s_nsel, s_nl, s_out[RMAX];
    const int tid = threadIdx.x;

    int64_t p;
    int32_t *dst;
    if (MODE == 0) {
        p = pp.nodes[blockIdx.x];
        dst = pp.newl + (int64_t)blockIdx.x * pp.R;
    } else {
        if ((int64_t)blockIdx.x >= (*pp.total & 0xffffffff)) return;
        p = pp.touched[blockIdx.x];
        dst = pp.graph + p * pp.R;
    }
    const int32_t *old = pp.graph + p * pp.R;

    // ---- gather the pool (ordered: first list, then additions) ----
    if (MODE == 0) {
        // beam members except p (distinct), then old neighbours not in the beam
        const int32_t *beam = pp.beams + (int64_t)blockIdx.x * pp.Lb;
        if (tid == 0) {
            int np = 0;
            for (int t = 0; t < pp.Lb; ++t) {
                int u = beam[t];
                if (u < 0) break;
                if (u != p) pid[np++] = u;
            }
            s_np = np;
        }
        __syncthreads();
        const int nbeam = s_np;
        // old neighbours: flag those already in the beam (parallel), then append in order
        for (int s = tid; s < pp.R; s += blockDim.x) {
            int u = old[s];
            int keep = (u >= 0 && u != p) ? 1 : 0;
            if (keep)
                for (int t = 0; t < nbeam; ++t)
                    if (pid[t] == u) {
                        keep = 0;
                        break;
                    }
            aux[s] = keep ? u : -1;
        }
        __syncthreads();
        if (tid == 0) {
            int np = nbeam;
            for (int s = 0; s < pp.R; ++s)
                if (aux[s] >= 0 && np < pp.PMAX) pid[np++] = aux[s];
            s_np = np;
        }
        __syncthreads();
    } else {
        const int64_t o0 = pp.offs[p] >> 32, o1 = pp.offs[p + 1] >> 32;
        const int nsrc = (int)(o1 - o0);
        // current list (compacted)
        if (tid == 0) {
            int nl = 0;
            for (int s = 0; s < pp.R; ++s)
                if (old[s] >= 0) pid[nl++] = old[s];
            s_nl = nl;
        }
        __syncthreads();
        const int nl = s_nl;
        // sort the sources ascending (ranks; sources are distinct) and drop present ones
        if (nsrc > pp.PMAX && tid == 0) atomicOr(pp.status, ST_CAPACITY);
        for (int t = tid; t < nsrc; t += blockDim.x) {
            const int s = pp.srcs[o0 + t];
            int rank = 0;
            for (int w = 0; w < nsrc; ++w) rank += pp.srcs[o0 + w] < s ? 1 : 0;
            int keep = s != p;
            if (keep)
                for (int w = 0; w < nl; ++w)
                    if (pid[w] == s) {
                        keep = 0;
                        break;
                    }
            if (rank < pp.PMAX) ord[rank] = keep ? s : -1;
        }
        __syncthreads();
        if (tid == 0) {
            int np = nl;
            for (int t = 0; t < nsrc && t < pp.PMAX; ++t)
                if (ord[t] >= 0) {
                    if (np < pp.PMAX)
                        pid[np++] = ord[t];
                    else
                        atomicOr(pp.status, ST_CAPACITY);
                }
            s_np = np;
        }
        __syncthreads();
        if (s_np <= pp.R) {
            for (int s = tid; s < pp.R; s += blockDim.x) dst[s] = s < s_np ? pid[s] : -1;
            return;
        }
    }
    const int np = s_np;

    // ---- stage records (16-byte chunks) ----
    const int chunks = stride / 16;
    for (int t = tid; t < (np + 1) * chunks; t += blockDim.x) {
        const int r = t / chunks, c = t % chunks;
        const int64_t id = r < np ? pid[r] : p;
        uint8_t *dstr = r < np ? recs + (size_t)r * stride : prec;
        *reinterpret_cast<uint4 *>(dstr + 16 * c) = *reinterpret_cast<const uint4 *>(pp.prim + id * pp.stride + 16 * c);
    }
    __syncthreads();
    const float fdim = (float)pp.dim;
    for (int i = tid; i < np; i += blockDim.x) {
        psc[i] = smem_pair_score<BITS, L2>(prec, recs + (size_t)i * stride, pp.CH, pp.cb, pp.mu2, fdim);
        dead[i] = 0;
    }
    __syncthreads();
    // ---- order by (score desc, id asc) ----
    for (int i = tid; i < np; i += blockDim.x) {
        const float s = psc[i];
        const int id = pid[i];
        int rank = 0;
        for (int t = 0; t < np; ++t) rank += key_better(psc[t], pid[t], s, id) ? 1 : 0;
        ord[rank] = i;
    }
    if (tid == 0) s_nsel = 0;
    __syncthreads();
    // ---- greedy selection ----
    for (int pos = 0; pos < np; ++pos) {
        const int i = ord[pos];
        if (dead[i]) continue;  // uniform: dead[] only changes between barriers
        const int nsel = s_nsel;
        if (nsel >= pp.R) break;
        __syncthreads();
        if (tid == 0) {
            s_out[nsel] = pid[i];
            s_nsel = nsel + 1;
        }
        if (nsel + 1 < pp.R) {
            const uint8_t *ri = recs + (size_t)i * stride;
            for (int q = pos + 1 + tid; q < np; q += blockDim.x) {
                const int j = ord[q];
                if (dead[j]) continue;
                const float s = smem_pair_score<BITS, L2>(ri, recs + (size_t)j * stride, pp.CH, pp.cb, pp.mu2, fdim);
                if (__fmul_rn(pp.alpha, s) >= __fadd_rn(psc[j], pp.shift)) dead[j] = 1;
            }
        }
        __syncthreads();
    }
    __syncthreads();
    const int nsel = s_nsel;
    for (int s = tid; s < pp.R; s += blockDim.x) dst[s] = s < nsel ? s_out[s] : -1;
}

__global__ void scatter_rows_kernel(const int32_t *newl, const int32_t *nodes, int nb, int R, int32_t *graph) {
    const int t = blockIdx.x;
    if (t >= nb) return;
    const int64_t p = nodes[t];
    for (int s = threadIdx.x; s < R; s += blockDim.x) graph[p * R + s] = newl[(int64_t)t * R + s];
}

__global__ void count_pairs_kernel(const int32_t *newl, int64_t total, int *cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int u = newl[i];
    if (u >= 0) atomicAdd(cnt + u, 1);
}

__global__ void scatter_pairs_kernel(const int32_t *newl, const int32_t *nodes, int nb, int R, const int64_t *offs,
                                     int *cnt, int32_t *srcs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nb * R) return;
    int u = newl[i];
    if (u < 0) return;
    const int t = (int)(i / R);
    const int64_t pos = (offs[u] >> 32) + atomicSub(cnt + u, 1) - 1;
    srcs[pos] = nodes[t];
}

// Exclusive scan of packed (count << 32 | (count > 0)) over n nodes: 8192 per block.
constexpr int SCAN_T = 1024, SCAN_E = 8;
__global__ void scan_local_kernel(const int *cnt, int64_t n, int64_t *offs, int64_t *bsum) {
    __shared__ int64_t sh[SCAN_T];
    const int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_E + (int64_t)threadIdx.x * SCAN_E;
    int64_t v[SCAN_E];
    int64_t s = 0;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e) {
        const int64_t i = base + e;
        const int c = i < n ? cnt[i] : 0;
        v[e] = ((int64_t)c << 32) | (c > 0 ? 1 : 0);
        s += v[e];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {
        int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int64_t run = sh[threadIdx.x] - s;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e) {
        const int64_t i = base + e;
        if (i < n) offs[i] = run;
        run += v[e];
    }
    if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = sh[SCAN_T - 1];
}

__global__ void scan_blocks_kernel(int64_t *bsum, int nb, int64_t *total) {
    __shared__ int64_t sh[SCAN_T];
    int64_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SCAN_T) {
        const int i = b0 + threadIdx.x;
        const int64_t v = i < nb ? bsum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < SCAN_T; o <<= 1) {
            int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
        const int64_t tot = sh[SCAN_T - 1];
        __syncthreads();
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_add_kernel(int64_t *offs, int64_t n, const int64_t *bsum, const int64_t *total,
                                const int *cnt, int32_t *touched) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) {
        offs[n] = *total;
        return;
    }
    const int64_t v = offs[i] + bsum[i / (SCAN_T * SCAN_E)];
    offs[i] = v;
    if (cnt[i] > 0) touched[(int)(v & 0xffffffff)] = (int32_t)i;
}

// ---------------------------------------------------------------- launchers
int launch_graph_sanitize(int32_t *graph, int64_t n, int R, int *status, cudaStream_t st) {
    graph_sanitize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(graph, n, R, status);
    LV_CHECK_LAUNCH("graph_sanitize_kernel");
    return LV_OK;
}

int launch_entry_argmax(const uint8_t *rec, int64_t n, int64_t stride, int code_bytes, int metric, int32_t *out,
                        cudaStream_t st) {
    const int nb = 256;
    float *bg = nullptr;
    int *bi = nullptr;
    int rc = tmp_alloc((void **)&bg, sizeof(float) * nb, st);
    if (rc == LV_OK) rc = tmp_alloc((void **)&bi, sizeof(int) * nb, st);
    if (rc) {
        tmp_free(bg, st);
        return rc;
    }
    entry_partial_kernel<<<nb, 256, 0, st>>>(rec, n, stride, code_bytes, metric, bg, bi);
    entry_final_kernel<<<1, 256, 0, st>>>(bg, bi, nb, out);
    cudaError_t e = cudaGetLastError();
    tmp_free(bg, st);
    tmp_free(bi, st);
    if (e != cudaSuccess) return cuda_fail(e, "entry kernels");
    return LV_OK;
}

// ------------------------------------------------------------------ driver
static int prune_smem(int PMAX, int64_t stride) { return (int)(PMAX * (stride + 17) + stride + 16); }

template <int BITS, bool L2>
static int launch_prune_m(const PruneParams &pp, int mode, unsigned grid, cudaStream_t st) {
    const int sm = prune_smem(pp.PMAX, pp.stride);
    if (grid == 0) return LV_OK;
    if (mode == 0) {
        auto k = prune_kernel<BITS, 0, L2>;
        LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        k<<<grid, 128, sm, st>>>(pp);
    } else {
        auto k = prune_kernel<BITS, 1, L2>;
        LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        k<<<grid, 128, sm, st>>>(pp);
    }
    LV_CHECK_LAUNCH("prune_kernel");
    return LV_OK;
}

template <int BITS>
static int launch_prune(const PruneParams &pp, int mode, unsigned grid, cudaStream_t st) {
    return pp.metric ? launch_prune_m<BITS, true>(pp, mode, grid, st) : launch_prune_m<BITS, false>(pp, mode, grid, st);
}

int build_graph_impl(lv_index *idx, int R, int Lb, float alpha, int passes, int batch, uint64_t seed, int rule,
                     cudaStream_t st) {
    const int64_t n = idx->n;
    batch = (int)std::min<int64_t>(batch, n);
    const int PMAX = Lb + R;
    if (prune_smem(PMAX, idx->pg.stride) > 227 * 1024) return fail(LV_ERR_CAPACITY, "build: L_build + R too large");
    // reverse-edge pool: the target's list plus its new sources of one batch
    int PMAX1 = std::max(PMAX, 4 * R + 256);
    // (two prune blocks per SM for short records; long records may take most of an SM's shared memory)
    const int cap1 = idx->pg.stride > 256 ? 200 * 1024 : 120 * 1024;
    while (PMAX1 > PMAX && prune_smem(PMAX1, idx->pg.stride) > cap1) PMAX1 -= 32;
    cudaFree(idx->graph);
    idx->graph = nullptr;
    idx->R = 0;
    idx->entry = -1;
    LV_CUDA(cudaMalloc(&idx->graph, sizeof(int32_t) * (size_t)n * R));

    // workspace layout
    const int64_t nblk = (n + SCAN_T * SCAN_E - 1) / (SCAN_T * SCAN_E);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += round_up((int64_t)bytes, 256);
        return o;
    };
    const size_t o_perm = take(sizeof(int32_t) * n);
    const size_t o_bid = take(sizeof(int32_t) * (size_t)batch * Lb);
    const size_t o_bsc = take(sizeof(float) * (size_t)batch * Lb);
    const size_t o_newl = take(sizeof(int32_t) * (size_t)batch * R);
    const size_t o_cnt = take(sizeof(int) * n);
    const size_t o_offs = take(sizeof(int64_t) * (n + 1));
    const size_t o_bsum = take(sizeof(int64_t) * (nblk + 1));
    const size_t o_tot = take(sizeof(int64_t));
    const size_t o_touch = take(sizeof(int32_t) * (size_t)std::min<int64_t>(n, (int64_t)batch * R));
    const size_t o_srcs = take(sizeof(int32_t) * (size_t)batch * R);
    const size_t o_ent = take(sizeof(int32_t));
    int rc = ensure_ws(&idx->bws, &idx->bws_bytes, off);
    if (rc) return rc;
    uint8_t *ws = reinterpret_cast<uint8_t *>(idx->bws);
    int32_t *perm_d = reinterpret_cast<int32_t *>(ws + o_perm);
    int32_t *bid = reinterpret_cast<int32_t *>(ws + o_bid);
    float *bsc = reinterpret_cast<float *>(ws + o_bsc);
    int32_t *newl = reinterpret_cast<int32_t *>(ws + o_newl);
    int *cnt = reinterpret_cast<int *>(ws + o_cnt);
    int64_t *offs = reinterpret_cast<int64_t *>(ws + o_offs);
    int64_t *bsum = reinterpret_cast<int64_t *>(ws + o_bsum);
    int64_t *tot = reinterpret_cast<int64_t *>(ws + o_tot);
    int32_t *touched = reinterpret_cast<int32_t *>(ws + o_touch);
    int32_t *srcs = reinterpret_cast<int32_t *>(ws + o_srcs);
    int32_t *ent_d = reinterpret_cast<int32_t *>(ws + o_ent);

    // initial graph, entry point, order
    random_graph_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(idx->graph, n, R, seed, idx->status);
    LV_CHECK_LAUNCH("random_graph_kernel");
    rc = launch_entry_argmax(idx->prim, n, idx->pg.stride, idx->pg.code_bytes, idx->metric, ent_d, st);
    if (rc) return rc;
    int32_t entry = 0;
    LV_CUDA(cudaMemcpyAsync(&entry, ent_d, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    std::vector<int32_t> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i >= 1; --i) {
        int64_t j = (int64_t)(splitmix(seed + 1, (uint64_t)i, 0) % (uint64_t)(i + 1));
        std::swap(perm[i], perm[j]);
    }
    LV_CUDA(cudaMemcpyAsync(perm_d, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    LV_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * n, st));
    LV_CUDA(cudaStreamSynchronize(st));

    // search in build mode
    BeamParams bp;
    memset(&bp, 0, sizeof(bp));
    bp.prim = idx->prim;
    bp.prim_stride = idx->pg.stride;
    bp.prim_chunks = idx->pg.code_chunks;
    bp.prim_dim = idx->d;
    bp.graph = idx->graph;
    bp.R = R;
    bp.n = n;
    bp.entry = entry;
    bp.uni = make_int4(Lb, Lb, 0, 0);
    bp.mu2 = idx->mu2;
    bp.metric = idx->metric;
    bp.ids = bid;
    bp.scores = bsc;
    bp.ldo = Lb;
    bp.status = idx->status;
    bp.work = idx->status + 1;
    bp.Lcap = (int)round_up(Lb, 32);
    int hs = 1024;
    while (hs < 8 * Lb && hs < 8192) hs <<= 1;
    while (hs < 2 * bp.Lcap) hs <<= 1;
    bp.Hcap = hs;
    bp.hbits = 0;
    while ((1 << bp.hbits) < hs) bp.hbits++;
    bp.W = 1;
    bp.T = 1;
    bp.Rcap = beam_rcap(1, 1, R);
    bp.vbits = 32;
    bp.warp_smem = beam_warp_smem(bp.Lcap, bp.Hcap, 32, bp.Rcap, 0);  // the build scorer keeps its query in registers
    int warps = 8;
    while (warps > 1 && (size_t)warps * bp.warp_smem > 227 * 1024) warps >>= 1;
    const size_t bsmem = (size_t)warps * bp.warp_smem;
    const int nc = (idx->pg.code_chunks + 1 + idx->metric + 3) / 4;

    PruneParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.prim = idx->prim;
    pp.stride = idx->pg.stride;
    pp.CH = idx->pg.code_chunks;
    pp.cb = idx->pg.code_bytes;
    pp.dim = idx->d;
    pp.mu2 = idx->mu2;
    pp.metric = idx->metric;
    pp.R = R;
    pp.PMAX = PMAX;
    pp.n = n;
    pp.graph = idx->graph;
    pp.beams = bid;
    pp.Lb = Lb;
    pp.newl = newl;
    pp.offs = offs;
    pp.srcs = srcs;
    pp.touched = touched;
    pp.total = tot;
    pp.status = idx->status;

    for (int pass = 0; pass < passes; ++pass) {
        pp.alpha = pass < passes - 1 ? 1.0f : alpha;
        pp.shift = rule ? host_fsub(pp.alpha, 1.0f) : 0.0f;
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int nb = (int)std::min<int64_t>(batch, n - b0);
            bp.qnodes = perm_d + b0;
            bp.m = nb;
            LV_CUDA(cudaMemsetAsync(bp.work, 0, sizeof(int), st));
            rc = launch_build_search(bp, idx->pbits, nc, warps * 32, bsmem, idx->num_sms, st);
            if (rc) return rc;
            pp.nodes = perm_d + b0;
            rc = idx->pbits == 8 ? launch_prune<8>(pp, 0, nb, st) : launch_prune<4>(pp, 0, nb, st);
            if (rc) return rc;
            scatter_rows_kernel<<<nb, 64, 0, st>>>(newl, perm_d + b0, nb, R, idx->graph);
            const int64_t tp = (int64_t)nb * R;
            count_pairs_kernel<<<(unsigned)((tp + 255) / 256), 256, 0, st>>>(newl, tp, cnt);
            scan_local_kernel<<<(unsigned)nblk, SCAN_T, 0, st>>>(cnt, n, offs, bsum);
            scan_blocks_kernel<<<1, SCAN_T, 0, st>>>(bsum, (int)nblk, tot);
            scan_add_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(offs, n, bsum, tot, cnt, touched);
            scatter_pairs_kernel<<<(unsigned)((tp + 255) / 256), 256, 0, st>>>(newl, perm_d + b0, nb, R, offs, cnt, srcs);
            LV_CHECK_LAUNCH("reverse-edge kernels");
            const unsigned g1 = (unsigned)std::min<int64_t>(n, tp);
            PruneParams pr = pp;
            pr.PMAX = PMAX1;  // a target may receive many reverse edges in one batch
            rc = idx->pbits == 8 ? launch_prune<8>(pr, 1, g1, st) : launch_prune<4>(pr, 1, g1, st);
            if (rc) return rc;
        }
    }
    LV_CUDA(cudaStreamSynchronize(st));
    idx->R = R;
    idx->entry = entry;
    return LV_OK;
}

}  // namespace lv
