// Host side of the C ABI declared in include/leanvec.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "beam.cuh"
#include "common.cuh"
#include "index.cuh"

namespace lv {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LV_ERR_OOM : LV_ERR_CUDA;
}

// kernels of other translation units
int launch_column_mean(const float *X, int64_t n, int dim, float *mean, cudaStream_t st);
int launch_lvq_self_norms(uint8_t *rec, int64_t n, int dim, int bits, int64_t stride, int code_bytes, float mu2,
                          cudaStream_t st);
int launch_set_sqnorms(uint8_t *rec, int64_t n, int64_t stride, int off, const float *X, int D, cudaStream_t st);
int launch_lvq_encode(const float *V, int64_t n, int dim, const float *mean, int bits, uint8_t *rec,
                      cudaStream_t st, int metric = 0);
int launch_fp32_records(const float *X, int64_t n, int dim, uint8_t *rec, int64_t stride, cudaStream_t st);
int launch_fp16_records(const float *X, int64_t n, int dim, int64_t stride, uint8_t *out, cudaStream_t st);
int launch_mu2(const float *mean, int dim, float *out, cudaStream_t st);
int launch_project_fp32(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy,
                        cudaStream_t st);
int launch_pad_rows(const float *X, int64_t n, int D, float *Y, int ldy, cudaStream_t st);
int launch_graph_sanitize(int32_t *graph, int64_t n, int R, int *status, cudaStream_t st);
int launch_entry_argmax(const uint8_t *rec, int64_t n, int64_t stride, int code_bytes, int metric, int32_t *out,
                        cudaStream_t st);
int build_graph_impl(lv_index *idx, int R, int L_build, float alpha, int passes, int batch, uint64_t seed,
                     int rule, cudaStream_t st);
int project_bf16(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, void **ws,
                 size_t *ws_bytes, int *status, cudaStream_t st);
int project_fp8(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, void **ws,
                size_t *ws_bytes, int *status, cudaStream_t st);
size_t project_tc_ws_bytes(int prec, int64_t n, int D, int d, const float *X);
bool project_bf16_fused_ok(const float *X, int D, int d);
// tensor-core projection with bf16 or e4m3 (per-row scaled) operands
int project_tf32x3(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, void **ws,
                   size_t *ws_bytes, int *status, cudaStream_t st);
static int project_tc(int prec, const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, void **ws,
                      size_t *ws_bytes, int *status, cudaStream_t st) {
    if (prec == LV_PREC_TF32X3) return project_tf32x3(X, n, D, P, d, Y, ldy, ws, ws_bytes, status, st);
    return prec == LV_PREC_FP8 ? project_fp8(X, n, D, P, d, Y, ldy, ws, ws_bytes, status, st)
                               : project_bf16(X, n, D, P, d, Y, ldy, ws, ws_bytes, status, st);
}

}  // namespace lv

using namespace lv;


namespace lv {
void index_free_stores(lv_index *idx) {
    cudaFree(idx->prim);
    cudaFree(idx->pmean);
    cudaFree(idx->sec);
    cudaFree(idx->smean);
    cudaFree(idx->graph);
    idx->prim = nullptr;
    idx->pmean = nullptr;
    idx->sec = nullptr;
    idx->smean = nullptr;
    idx->graph = nullptr;
    idx->n = 0;
    idx->R = 0;
    idx->entry = -1;
    idx->pbits = idx->sbits = 0;
}

int ensure_ws(void **p, size_t *have, size_t want) {
    if (*have >= want) return LV_OK;
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
    if (cudaMalloc(p, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(LV_ERR_OOM, "workspace allocation failed");
    }
    *have = want;
    return LV_OK;
}

int *index_status(lv_index *idx) { return idx->status; }
int index_num_sms(lv_index *idx) { return idx->num_sms; }

static int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

int search_shape(const lv_index *idx, const lv_search_params *params, BeamParams &p, int *block, size_t *smem,
                 const char *who) {
    const std::string w(who);
    const lv_query_desc &u = params->uniform;
    p.Lcap = (int)round_up(u.L, 32);
    const int hs32 = std::min(8192, std::max(1024, next_pow2(4 * u.L)));  // default slots of 32-bit ids
    int hs = params->hash_slots > 0 ? params->hash_slots : hs32;
    if (hs & (hs - 1)) return fail(LV_ERR_ARG, w + ": hash_slots must be a power of two");
    hs = std::max(hs, next_pow2(2 * p.Lcap));
    // visited-cache slots of one query per warp: 32-bit ids, or on request 16-bit tags (by default
    // twice the slots of 32-bit ids, in the same bytes); two queries per warp always hold tags, in
    // buckets of 4
    const int vb = params->visited_bits;
    if (vb != 0 && vb != 16 && vb != 32) return fail(LV_ERR_ARG, w + ": visited_bits must be 0, 16 or 32");
    p.vbits = 32;
    if (vb == 16 && params->queries_per_warp != 2) {
        const int hs16 = params->hash_slots > 0 ? hs : std::max(hs, 2 * hs32);
        if (!tags_fit(idx->n, hs16)) return fail(LV_ERR_ARG, w + ": visited_bits 16 needs n <= 65535 * hash_slots / 8");
        p.vbits = 16;
        hs = hs16;
    }
    p.Hcap = hs;
    p.hbits = 0;
    while ((1 << p.hbits) < hs) p.hbits++;
    p.W = params->width > 0 ? params->width : 1;
    if (p.W > WMAX || p.W * idx->R > CMAX) return fail(LV_ERR_ARG, w + ": need width <= 4 and width * R <= 256");
    p.T = params->warps_per_query > 0 ? params->warps_per_query : 1;
    if ((p.T != 1 && p.T != 2 && p.T != 4) || p.W % p.T)
        return fail(LV_ERR_ARG, w + ": warps_per_query must be 1, 2 or 4 and divide width");
    const int qpw = params->queries_per_warp;
    if (qpw < 0 || qpw > 2) return fail(LV_ERR_ARG, w + ": queries_per_warp must be 0, 1 or 2");
    const bool half_ok = idx->pbits != 32 && p.T == 1 && p.W <= 2 && p.W * idx->R <= 16 * HALF_IDS &&
                         half_tags_fit(idx->n, hs);
    if (qpw == 2 && !half_ok)
        return fail(LV_ERR_ARG, w + ": two queries per warp need LVQ primaries, warps_per_query 1, width <= 2, "
                                    "width * R <= 128 and n <= 65535 * hash_slots / 4");
    p.qpw = qpw == 2 ? 2 : 1;
    const int nc_q = idx->pbits == 32 ? 0 : (idx->pg.code_chunks + 1 + idx->metric + 3) / 4;
    const int qbytes = lvq_query_bytes(idx->pbits, nc_q);
    int warps = params->warps_per_block;
    if (warps > 32) return fail(LV_ERR_ARG, w + ": warps_per_block must be <= 32");
    if (p.qpw == 2) {
        p.Rcap = half_rcap(p.W, idx->R);
        p.warp_smem = half_query_smem(p.Lcap, p.Hcap, p.Rcap, qbytes);
        if (warps <= 0) warps = 10;
        while (warps > 1 && (size_t)2 * warps * p.warp_smem > 227 * 1024) warps >>= 1;
        *smem = (size_t)2 * warps * p.warp_smem;
    } else {
        p.Rcap = beam_rcap(p.W, p.T, idx->R);
        p.warp_smem = beam_warp_smem(p.Lcap, p.Hcap, p.vbits, p.Rcap, qbytes);
        if (warps <= 0) warps = 8;
        if (warps % p.T) return fail(LV_ERR_ARG, w + ": warps_per_block must be a multiple of warps_per_query");
        while (warps > p.T && (size_t)(warps / p.T) * p.warp_smem > 227 * 1024) warps >>= 1;
        *smem = (size_t)(warps / p.T) * p.warp_smem;
    }
    if (*smem > 227 * 1024) return fail(LV_ERR_CAPACITY, w + ": L / hash_slots too large for shared memory");
    *block = warps * 32;
    return LV_OK;
}

int launch_beam_search(const lv_index *idx, const BeamParams &p, int block, size_t smem, cudaStream_t st) {
    if (idx->pbits == 32) return launch_search_fp32(p, (idx->pg.code_chunks + 31) / 32, block, smem, idx->num_sms, st);
    const int nc = (idx->pg.code_chunks + 1 + idx->metric + 3) / 4;  // codes + constants chunks over 4 lanes
    if (p.qpw == 2)
        return idx->pbits == 8 ? launch_search_half8(p, nc, block, smem, idx->num_sms, st)
                               : launch_search_half4(p, nc, block, smem, idx->num_sms, st);
    return idx->pbits == 8 ? launch_search_lvq8(p, nc, block, smem, idx->num_sms, st)
                           : launch_search_lvq4(p, nc, block, smem, idx->num_sms, st);
}
}  // namespace lv

extern "C" {

const char *leanvec_last_error(void) { return g_last_error.c_str(); }

int64_t leanvec_record_stride(int dim, int bits) {
    RecGeom g;
    if (!rec_geom(dim, bits, g)) return fail(LV_ERR_ARG, "record_stride: dim must be > 0 and bits in {4, 8, 32}");
    return g.stride;
}

int leanvec_column_mean(const float *X, int64_t n, int dim, float *mean, lv_stream_t stream) {
    if (!X || !mean || n <= 0 || dim <= 0) return fail(LV_ERR_ARG, "column_mean: empty input or null pointer");
    return launch_column_mean(X, n, dim, mean, (cudaStream_t)stream);
}

int leanvec_lvq_encode(const float *V, int64_t n, int dim, const float *mean, int bits, uint8_t *records,
                       lv_stream_t stream) {
    if (n < 0 || dim <= 0 || (n > 0 && (!V || !mean || !records)))
        return fail(LV_ERR_ARG, "lvq_encode: invalid sizes or null pointer");
    if (bits != 4 && bits != 8) return fail(LV_ERR_ARG, "lvq_encode: bits must be 4 or 8");
    return launch_lvq_encode(V, n, dim, mean, bits, records, (cudaStream_t)stream);
}

int leanvec_project(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, int precision,
                    lv_stream_t stream) {
    if (n < 0 || D <= 0 || d <= 0 || ldy < d || (n > 0 && (!X || !P || !Y)))
        return fail(LV_ERR_ARG, "project: invalid sizes or null pointer");
    if (precision == LV_PREC_FP32) return launch_project_fp32(X, n, D, P, d, Y, ldy, (cudaStream_t)stream);
    if (precision != LV_PREC_BF16 && precision != LV_PREC_FP8 && precision != LV_PREC_TF32X3)
        return fail(LV_ERR_ARG, "project: precision must be LV_PREC_FP32, LV_PREC_BF16, LV_PREC_FP8 or LV_PREC_TF32X3");
    if (n == 0) return LV_OK;
    cudaStream_t st = (cudaStream_t)stream;
    void *ws = nullptr;
    size_t wsb = project_tc_ws_bytes(precision, n, D, d, X);
    int *status = nullptr;
    int h_status = 0;
    int rc = tmp_alloc((void **)&status, sizeof(int), st);
    if (rc == LV_OK) rc = tmp_alloc(&ws, wsb, st);
    if (rc == LV_OK && cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
        rc = fail(LV_ERR_CUDA, "project: memset failed");
    if (rc == LV_OK) rc = project_tc(precision, X, n, D, P, d, Y, ldy, &ws, &wsb, status, st);
    if (rc == LV_OK && cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = fail(LV_ERR_CUDA, "project: status copy failed");
    if (rc == LV_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(LV_ERR_CUDA, "project: sync failed");
    if (rc == LV_OK && h_status) rc = fail(LV_ERR_TIMEOUT, "project: a tensor-core pipeline wait timed out");
    tmp_free(ws, st);
    tmp_free(status, st);
    return rc;
}

int leanvec_index_create(lv_index **out, int device) {
    if (!out) return fail(LV_ERR_ARG, "index_create: null output");
    *out = nullptr;
    int ndev = 0;
    LV_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(LV_ERR_ARG, "index_create: no such CUDA device");
    DeviceGuard g(device);
    if (!g.ok) return fail(LV_ERR_CUDA, "index_create: cannot select device");
    lv_index *idx = new lv_index();
    idx->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete idx;
        return fail(LV_ERR_CUDA, "index_create: cudaGetDeviceProperties failed");
    }
    idx->num_sms = prop.multiProcessorCount;
    if (cudaMalloc(&idx->status, 4 * sizeof(int)) != cudaSuccess || cudaMemset(idx->status, 0, 4 * sizeof(int)) != cudaSuccess) {
        cudaFree(idx->status);
        delete idx;
        return fail(LV_ERR_OOM, "index_create: status allocation failed");
    }
    *out = idx;
    return LV_OK;
}

int leanvec_index_free(lv_index *idx) {
    if (!idx) return LV_OK;
    DeviceGuard g(idx->device);
    index_free_stores(idx);
    cudaFree(idx->status);
    cudaFree(idx->ws_q);
    cudaFree(idx->ws_cand);
    cudaFree(idx->bws);
    if (idx->aux) cudaStreamDestroy(idx->aux);
    if (idx->ev_fork) cudaEventDestroy(idx->ev_fork);
    if (idx->ev_join) cudaEventDestroy(idx->ev_join);
    host_slots_free(idx);
    delete idx;
    return LV_OK;
}

int leanvec_set_metric(lv_index *idx, int metric) {
    if (!idx) return fail(LV_ERR_ARG, "set_metric: null index");
    if (metric != LV_METRIC_IP && metric != LV_METRIC_L2)
        return fail(LV_ERR_ARG, "set_metric: metric must be LV_METRIC_IP or LV_METRIC_L2");
    if (idx->n != 0 && metric != idx->metric)
        return fail(LV_ERR_STATE, "set_metric: set the metric before the index holds a store");
    idx->metric = metric;
    return LV_OK;
}

int leanvec_index_info(const lv_index *idx, lv_index_info *out) {
    if (!idx || !out) return fail(LV_ERR_ARG, "index_info: null pointer");
    memset(out, 0, sizeof(*out));
    out->n = idx->n;
    out->D = idx->D;
    out->d = idx->d;
    out->primary_bits = idx->pbits;
    out->secondary_bits = idx->sbits;
    out->primary_stride = idx->pg.stride;
    out->secondary_stride = idx->sbits ? idx->sg.stride : 0;
    out->R = idx->R;
    out->entry = idx->entry;
    out->mu2 = idx->mu2;
    out->last_search_kernels = idx->last_kernels;
    return LV_OK;
}

int leanvec_index_buffers(const lv_index *idx, const uint8_t **primary, const float **primary_mean,
                          const uint8_t **secondary, const float **secondary_mean, const int32_t **graph) {
    if (!idx) return fail(LV_ERR_ARG, "index_buffers: null index");
    if (primary) *primary = idx->prim;
    if (primary_mean) *primary_mean = idx->pmean;
    if (secondary) *secondary = idx->sec;
    if (secondary_mean) *secondary_mean = idx->smean;
    if (graph) *graph = idx->graph;
    return LV_OK;
}

#define LV_TRY(x)                      \
    do {                               \
        rc = (x);                      \
        if (rc != LV_OK) goto cleanup; \
    } while (0)
#define LV_TRYC(x)                      \
    do {                                \
        cudaError_t _e = (x);           \
        if (_e != cudaSuccess) {        \
            rc = cuda_fail(_e, #x);     \
            goto cleanup;               \
        }                               \
    } while (0)

static void drop_primary(lv_index *idx) {
    cudaFree(idx->prim);
    cudaFree(idx->pmean);
    cudaFree(idx->graph);
    idx->prim = nullptr;
    idx->pmean = nullptr;
    idx->graph = nullptr;
    idx->R = 0;
    idx->entry = -1;
    idx->pbits = 0;
}

static void drop_secondary(lv_index *idx) {
    cudaFree(idx->sec);
    cudaFree(idx->smean);
    idx->sec = nullptr;
    idx->smean = nullptr;
    idx->sbits = 0;
}

static int set_primary_impl(lv_index *idx, const float *Y, int64_t n, int d, const float *mean, int bits, int D,
                            cudaStream_t st) {
    RecGeom pg;
    rec_geom(d, bits, pg, idx->metric);
    float *mu2d = nullptr;
    int rc = LV_OK;
    drop_primary(idx);
    if (idx->n != n) drop_secondary(idx);
    LV_TRY(tmp_alloc((void **)&mu2d, sizeof(float), st));
    LV_TRYC(cudaMalloc(&idx->prim, (size_t)n * pg.stride));
    LV_TRYC(cudaMalloc(&idx->pmean, sizeof(float) * d));
    if (mean)
        LV_TRYC(cudaMemcpyAsync(idx->pmean, mean, sizeof(float) * d, cudaMemcpyDeviceToDevice, st));
    else
        LV_TRY(launch_column_mean(Y, n, d, idx->pmean, st));
    LV_TRY(launch_lvq_encode(Y, n, d, idx->pmean, bits, idx->prim, st, idx->metric));
    LV_TRY(launch_mu2(idx->pmean, d, mu2d, st));
    LV_TRYC(cudaMemcpyAsync(&idx->mu2, mu2d, sizeof(float), cudaMemcpyDeviceToHost, st));
    LV_TRYC(cudaStreamSynchronize(st));
    // L2: self scores N (and ||x||^2 := N until the original vectors are known)
    if (idx->metric) LV_TRY(launch_lvq_self_norms(idx->prim, n, d, bits, pg.stride, pg.code_bytes, idx->mu2, st));
    idx->n = n;
    idx->d = d;
    idx->D = D;
    idx->pbits = bits;
    idx->pg = pg;
cleanup:
    tmp_free(mu2d, st);
    if (rc != LV_OK) {
        drop_primary(idx);
        drop_secondary(idx);
        idx->n = 0;
    }
    return rc;
}

// bits 8: LVQ-8 records of x - mean; bits 16: x rounded to IEEE half (no mean, no constants)
static int set_secondary_impl(lv_index *idx, const float *X, int64_t n, int D, const float *mean, int bits,
                              cudaStream_t st) {
    RecGeom sg;
    rec_geom(D, bits, sg, idx->metric);
    int rc = LV_OK;
    drop_secondary(idx);
    LV_TRYC(cudaMalloc(&idx->sec, (size_t)n * sg.stride));
    if (bits == 16) {
        LV_TRY(launch_fp16_records(X, n, D, sg.stride, idx->sec, st));
    } else {
        LV_TRYC(cudaMalloc(&idx->smean, sizeof(float) * D));
        if (mean)
            LV_TRYC(cudaMemcpyAsync(idx->smean, mean, sizeof(float) * D, cudaMemcpyDeviceToDevice, st));
        else
            LV_TRY(launch_column_mean(X, n, D, idx->smean, st));
        LV_TRY(launch_lvq_encode(X, n, D, idx->smean, 8, idx->sec, st, idx->metric));
        if (idx->metric) LV_TRY(launch_set_sqnorms(idx->sec, n, sg.stride, sg.code_bytes + 20, X, D, st));
    }
    // L2: the primaries' ||x||^2 from the original vectors too
    if (idx->metric && idx->prim && idx->pbits != 32)
        LV_TRY(launch_set_sqnorms(idx->prim, n, idx->pg.stride, idx->pg.code_bytes + 20, X, D, st));
    LV_TRYC(cudaStreamSynchronize(st));
    idx->sbits = bits;
    idx->sg = sg;
cleanup:
    if (rc != LV_OK) drop_secondary(idx);
    return rc;
}

int leanvec_set_primary(lv_index *idx, const float *Y, int64_t n, int d, const float *mean, int bits, int D,
                        lv_stream_t stream) {
    if (!idx || !Y) return fail(LV_ERR_ARG, "set_primary: null pointer");
    if (n <= 0 || n >= (int64_t)0x7fffffff) return fail(LV_ERR_ARG, "set_primary: n must be in [1, 2^31 - 1)");
    if (d <= 0 || D < d) return fail(LV_ERR_ARG, "set_primary: need 0 < d <= D");
    if (bits != 4 && bits != 8) return fail(LV_ERR_ARG, "set_primary: bits must be 4 or 8");
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "set_primary: cannot select device");
    return set_primary_impl(idx, Y, n, d, mean, bits, D, (cudaStream_t)stream);
}

int leanvec_set_secondary(lv_index *idx, const float *X, int64_t n, int D, const float *mean, lv_stream_t stream) {
    if (!idx || !X) return fail(LV_ERR_ARG, "set_secondary: null pointer");
    if (idx->n == 0 || idx->pbits == 32) return fail(LV_ERR_STATE, "set_secondary: set an LVQ primary store first");
    if (n != idx->n || D != idx->D) return fail(LV_ERR_ARG, "set_secondary: n and D must match the primary store");
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "set_secondary: cannot select device");
    return set_secondary_impl(idx, X, n, D, mean, 8, (cudaStream_t)stream);
}

int leanvec_encode(lv_index *idx, const float *X, int64_t n, int D, const float *B, int d, int primary_bits,
                   int secondary_bits, int projection_precision, lv_stream_t stream) {
    if (!idx || !X || !B) return fail(LV_ERR_ARG, "encode: null pointer");
    if (n <= 0 || n >= (int64_t)0x7fffffff) return fail(LV_ERR_ARG, "encode: n must be in [1, 2^31 - 1)");
    if (D <= 0 || d <= 0 || d > D) return fail(LV_ERR_ARG, "encode: need 0 < d <= D");
    if (primary_bits != 4 && primary_bits != 8) return fail(LV_ERR_ARG, "encode: primary_bits must be 4 or 8");
    if (secondary_bits != 0 && secondary_bits != 8 && secondary_bits != 16)
        return fail(LV_ERR_ARG, "encode: secondary_bits must be 0, 8 (LVQ-8) or 16 (FP16)");
    if (projection_precision < LV_PREC_FP32 || projection_precision > LV_PREC_TF32X3)
        return fail(LV_ERR_ARG, "encode: projection precision must be an lv_precision value");
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "encode: cannot select device");
    cudaStream_t st = (cudaStream_t)stream;
    float *Y = nullptr;
    int rc = LV_OK;
    index_free_stores(idx);
    LV_TRY(tmp_alloc((void **)&Y, sizeof(float) * (size_t)n * d, st));
    if (projection_precision != LV_PREC_FP32) {
        LV_TRY(project_tc(projection_precision, X, n, D, B, d, Y, d, &idx->bws, &idx->bws_bytes, idx->status, st));
    } else {
        LV_TRY(launch_project_fp32(X, n, D, B, d, Y, d, st));
    }
    LV_TRY(set_primary_impl(idx, Y, n, d, nullptr, primary_bits, D, st));
    if (secondary_bits) LV_TRY(set_secondary_impl(idx, X, n, D, nullptr, secondary_bits, st));
    if (idx->metric) {  // the primaries' ||x||^2 from X (also without a secondary store)
        LV_TRY(launch_set_sqnorms(idx->prim, n, idx->pg.stride, idx->pg.code_bytes + 20, X, D, st));
        LV_TRYC(cudaStreamSynchronize(st));
    }
cleanup:
    tmp_free(Y, st);
    if (rc != LV_OK) index_free_stores(idx);
    return rc;
}

int leanvec_encode_fp32(lv_index *idx, const float *X, int64_t n, int D, lv_stream_t stream) {
    if (!idx || !X) return fail(LV_ERR_ARG, "encode_fp32: null pointer");
    if (n <= 0 || n >= (int64_t)0x7fffffff || D <= 0) return fail(LV_ERR_ARG, "encode_fp32: invalid sizes");
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "encode_fp32: cannot select device");
    cudaStream_t st = (cudaStream_t)stream;
    index_free_stores(idx);
    RecGeom pg;
    rec_geom(D, 32, pg);
    int rc = LV_OK;
    LV_TRYC(cudaMalloc(&idx->prim, (size_t)n * pg.stride));
    LV_TRY(launch_fp32_records(X, n, D, idx->prim, pg.stride, st));
    LV_TRYC(cudaStreamSynchronize(st));
    idx->n = n;
    idx->D = D;
    idx->d = D;
    idx->pbits = 32;
    idx->sbits = 0;
    idx->pg = pg;
    idx->mu2 = 0.f;
cleanup:
    if (rc != LV_OK) index_free_stores(idx);
    return rc;
}

int leanvec_set_graph(lv_index *idx, const int32_t *adj, int R, int32_t entry, lv_stream_t stream) {
    if (!idx || !adj) return fail(LV_ERR_ARG, "set_graph: null pointer");
    if (idx->n == 0) return fail(LV_ERR_STATE, "set_graph: the index has no store");
    if (R < 1 || R > RMAX) return fail(LV_ERR_ARG, "set_graph: R must be in [1, 128]");
    if (entry >= idx->n) return fail(LV_ERR_ARG, "set_graph: entry out of range");
    if (entry < 0 && idx->pbits == 32)
        return fail(LV_ERR_ARG, "set_graph: a float32 index needs an explicit entry point");
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "set_graph: cannot select device");
    cudaStream_t st = (cudaStream_t)stream;
    cudaFree(idx->graph);
    idx->graph = nullptr;
    idx->R = 0;
    idx->entry = -1;
    LV_CUDA(cudaMalloc(&idx->graph, sizeof(int32_t) * (size_t)idx->n * R));
    LV_CUDA(cudaMemcpyAsync(idx->graph, adj, sizeof(int32_t) * (size_t)idx->n * R, cudaMemcpyDeviceToDevice, st));
    int rc = launch_graph_sanitize(idx->graph, idx->n, R, idx->status, st);
    if (rc != LV_OK) return rc;
    if (entry < 0) {
        int32_t *e = nullptr;
        rc = tmp_alloc((void **)&e, sizeof(int32_t), st);
        if (rc != LV_OK) return rc;
        rc = launch_entry_argmax(idx->prim, idx->n, idx->pg.stride, idx->pg.code_bytes, idx->metric, e, st);
        if (rc == LV_OK && cudaMemcpyAsync(&entry, e, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = fail(LV_ERR_CUDA, "set_graph: entry copy failed");
        if (rc == LV_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(LV_ERR_CUDA, "set_graph: sync failed");
        tmp_free(e, st);
        if (rc != LV_OK) return rc;
    }
    idx->R = R;
    idx->entry = entry;
    return LV_OK;
}

int leanvec_get_graph(const lv_index *idx, int32_t *adj, int32_t *entry, lv_stream_t stream) {
    if (!idx || !adj) return fail(LV_ERR_ARG, "get_graph: null pointer");
    if (!idx->graph) return fail(LV_ERR_STATE, "get_graph: the index has no graph");
    DeviceGuard g(idx->device);
    LV_CUDA(cudaMemcpyAsync(adj, idx->graph, sizeof(int32_t) * (size_t)idx->n * idx->R, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    if (entry) *entry = idx->entry;
    return LV_OK;
}

int leanvec_build_graph(lv_index *idx, int R, int L_build, float alpha, int passes, int batch, uint64_t seed,
                        int prune_rule, lv_stream_t stream) {
    if (!idx) return fail(LV_ERR_ARG, "build_graph: null index");
    if (idx->n == 0 || (idx->pbits != 8 && idx->pbits != 4))
        return fail(LV_ERR_STATE, "build_graph: the index has no LVQ primary store");
    if (R < 1 || R > RMAX || L_build < 1 || L_build > LCAP_MAX || passes < 1 || batch < 1 || !(alpha > 0.f))
        return fail(LV_ERR_ARG, "build_graph: need 1 <= R <= 128, 1 <= L_build <= 512, passes >= 1, batch >= 1, alpha > 0");
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "build_graph: cannot select device");
    if (prune_rule != LV_PRUNE_SCALED && prune_rule != LV_PRUNE_UNIT_L2)
        return fail(LV_ERR_ARG, "build_graph: unknown prune rule");
    return build_graph_impl(idx, R, L_build, alpha, passes, batch, seed, prune_rule, (cudaStream_t)stream);
}

int leanvec_search(lv_index *idx, const float *Q, int64_t m, const float *A, const lv_search_params *params,
                   const lv_query_desc *desc, int32_t *ids, float *scores, int ldo, lv_search_stats *stats,
                   lv_stream_t stream) {
    if (!idx || !params) return fail(LV_ERR_ARG, "search: null index or params");
    if (m < 0 || m >= (int64_t)0x7fffffff) return fail(LV_ERR_ARG, "search: invalid m");
    if (m == 0) return LV_OK;
    if (!Q || !ids || !scores) return fail(LV_ERR_ARG, "search: null query or output pointer");
    if (idx->n == 0) return fail(LV_ERR_STATE, "search: the index has no store");
    if (!idx->graph) return fail(LV_ERR_STATE, "search: the index has no graph");
    if (idx->pbits != 32 && !A) return fail(LV_ERR_ARG, "search: an LVQ index needs the projection A");
    const lv_query_desc &u = params->uniform;
    if (u.L < 1 || u.L > LCAP_MAX) return fail(LV_ERR_ARG, "search: L must be in [1, 512]");
    if (!desc && (u.k < 1 || u.k > u.L || u.k > ldo || u.rerank < 0 || u.rerank > u.L || u.max_hops < 0))
        return fail(LV_ERR_ARG, "search: need 1 <= k <= min(L, ldo), 0 <= rerank <= L, max_hops >= 0");
    if (u.rerank > 0 && !desc && !idx->sec) return fail(LV_ERR_STATE, "search: rerank needs a secondary store");
    if (params->projection < LV_PREC_FP32 || params->projection > LV_PREC_TF32X3)
        return fail(LV_ERR_ARG, "search: projection precision must be an lv_precision value");
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "search: cannot select device");
    cudaStream_t st = (cudaStream_t)stream;

    // padded queries in the primary space + per-query constants
    int cpc = idx->pbits == 8 ? 16 : idx->pbits == 4 ? 32 : 4;
    int ldq = idx->pg.code_chunks * cpc;
    int rc = ensure_ws((void **)&idx->ws_q, &idx->ws_q_bytes, sizeof(float) * (size_t)m * ldq);
    if (rc) return rc;
    idx->last_kernels = 0;
    // kernels of the projection: padding copy / float32 GEMM: 1; bf16 with float32 X converted in
    // the GEMM: cast of A + GEMM; otherwise casts of Q and A + GEMM
    // (tf32x3: split of A + GEMM)
    const int proj_kernels = idx->pbits == 32 || params->projection == LV_PREC_FP32 ? 1
                             : params->projection == LV_PREC_TF32X3 ? 2
                             : params->projection == LV_PREC_BF16 && project_bf16_fused_ok(Q, idx->D, idx->d) ? 2
                                                                                                                : 3;
    if (idx->pbits == 32) {
        rc = launch_pad_rows(Q, m, idx->D, idx->ws_q, ldq, st);
    } else if (params->projection != LV_PREC_FP32) {
        rc = project_tc(params->projection, Q, m, idx->D, A, idx->d, idx->ws_q, ldq, &idx->bws, &idx->bws_bytes,
                        idx->status, st);
    } else {
        rc = launch_project_fp32(Q, m, idx->D, A, idx->d, idx->ws_q, ldq, st);
    }
    if (rc) return rc;

    BeamParams p;
    memset(&p, 0, sizeof(p));
    p.prim = idx->prim;
    p.prim_stride = idx->pg.stride;
    p.prim_chunks = idx->pg.code_chunks;
    p.prim_dim = idx->d;
    p.graph = idx->graph;
    p.R = idx->R;
    p.n = idx->n;
    p.entry = idx->entry;
    p.qp = idx->ws_q;
    p.ldq = ldq;
    p.pmean = idx->pbits == 32 ? nullptr : idx->pmean;
    p.smean = idx->smean;
    p.desc = reinterpret_cast<const int4 *>(desc);
    p.uni = make_int4(u.k, u.L, idx->sec ? u.rerank : 0, u.max_hops);
    p.m = m;
    p.sec = idx->sec;
    p.sec_stride = idx->sbits ? idx->sg.stride : 0;
    p.sec_chunks = idx->sbits ? idx->sg.code_chunks : 0;
    p.sec_bits = idx->sbits;
    p.metric = idx->metric;
    p.Q = Q;
    p.D = idx->D;
    p.ids = ids;
    p.scores = scores;
    p.ldo = ldo;
    p.stats = reinterpret_cast<int2 *>(stats);
    p.status = idx->status;
    p.work = idx->status + 1;
    p.slots = nullptr;
    int block = 0;
    size_t smem = 0;
    rc = search_shape(idx, params, p, &block, &smem, "search");
    if (rc) return rc;
    if (idx->sbits == 8 && idx->sg.code_chunks + 1 + idx->metric > 64)
        return fail(LV_ERR_ARG, "search: D > 1008 (992 with L2) is not supported by the rerank");
    if (idx->sbits == 16 && idx->sg.code_chunks > 128) return fail(LV_ERR_ARG, "search: D > 1024 is not supported by the FP16 rerank");
    const bool rerank = idx->sbits && idx->pbits != 32 && (desc || u.rerank > 0);
    if (rerank) {
        p.ldc = p.Lcap;  // r <= L <= Lcap
        rc = ensure_ws((void **)&idx->ws_cand, &idx->ws_cand_bytes, sizeof(int32_t) * (size_t)m * (p.ldc + 1));
        if (rc) return rc;
        p.cand = idx->ws_cand;
        p.cand_n = idx->ws_cand + (size_t)m * p.ldc;
    }
    LV_CUDA(cudaMemsetAsync(p.work, 0, 2 * sizeof(int), st));  // the work counters of both sub-batches
    auto beam = [&](const BeamParams &q, cudaStream_t s) -> int { return launch_beam_search(idx, q, block, smem, s); };
    // Sub-batches: with rerank and m above one wave of resident query slots (slots = blocks per SM
    // x SMs x queries per block) and not a multiple of it, the first batch takes the whole waves
    // but the last 10 % of the last one, the rest forms a second batch launched on a second stream:
    // the second batch's blocks start as the first one's finish, and the first batch's rerank runs
    // beside the second batch's partial wave instead of after it.  Every query is computed exactly
    // as in one launch.
    int64_t mA = m;
    if (rerank) {
        int64_t slots = 0;
        BeamParams q = p;
        q.slots = &slots;
        rc = beam(q, st);
        if (rc) return rc;
        if (slots > 0 && m > slots && m % slots) mA = (m / slots - 1) * slots + slots * 9 / 10;
    }
    if (mA < m && !idx->aux) {
        LV_CUDA(cudaStreamCreateWithFlags(&idx->aux, cudaStreamNonBlocking));
        LV_CUDA(cudaEventCreateWithFlags(&idx->ev_fork, cudaEventDisableTiming));
        LV_CUDA(cudaEventCreateWithFlags(&idx->ev_join, cudaEventDisableTiming));
    }
    idx->last_kernels = proj_kernels + (mA == m ? 1 : 2) * (rerank ? 2 : 1);
    if (params->event_begin) LV_CUDA(cudaEventRecord((cudaEvent_t)params->event_begin, st));
    if (mA == m) {
        rc = beam(p, st);
        if (!rc && rerank) rc = launch_rerank(p, idx->num_sms, st);
        if (rc) return rc;
    } else {
        BeamParams pa = p, pb = p;
        pa.m = mA;
        pb.m = m - mA;
        pb.qp = p.qp + mA * ldq;
        if (p.desc) pb.desc = p.desc + mA;
        pb.Q = p.Q + mA * p.D;
        pb.ids = p.ids + mA * ldo;
        pb.scores = p.scores + mA * ldo;
        if (p.stats) pb.stats = p.stats + mA;
        pb.cand = p.cand + mA * p.ldc;
        pb.cand_n = p.cand_n + mA;
        pb.work = p.work + 1;
        LV_CUDA(cudaEventRecord(idx->ev_fork, st));
        LV_CUDA(cudaStreamWaitEvent(idx->aux, idx->ev_fork, 0));
        rc = beam(pa, st);
        if (!rc) rc = beam(pb, idx->aux);
        if (!rc) rc = launch_rerank(pa, idx->num_sms, st);
        if (!rc) rc = launch_rerank(pb, idx->num_sms, idx->aux);
        // join even after a failed launch, so that the caller's stream orders after the second one
        LV_CUDA(cudaEventRecord(idx->ev_join, idx->aux));
        LV_CUDA(cudaStreamWaitEvent(st, idx->ev_join, 0));
        if (rc) return rc;
    }
    if (params->event_end) LV_CUDA(cudaEventRecord((cudaEvent_t)params->event_end, st));
    return LV_OK;
}

int leanvec_sync_status(lv_index *idx, lv_stream_t stream) {
    if (!idx) return fail(LV_ERR_ARG, "sync_status: null index");
    DeviceGuard g(idx->device);
    int s = 0;
    LV_CUDA(cudaMemcpyAsync(&s, idx->status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    LV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    LV_CUDA(cudaMemsetAsync(idx->status, 0, sizeof(int), (cudaStream_t)stream));
    LV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (s & ST_CORRUPT) return fail(LV_ERR_CORRUPT, "a graph id was out of range");
    if (s & ST_CAPACITY) return fail(LV_ERR_CAPACITY, "a per-query size exceeded the launch capacity and was clamped");
    if (s & ST_TIMEOUT) return fail(LV_ERR_TIMEOUT, "a bounded device wait gave up");
    return LV_OK;
}

}  // extern "C"
