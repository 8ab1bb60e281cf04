// leanvec_search_noalloc: the search of leanvec_search for callers that must not
// allocate device memory.  Its scratch (the work counter, the projected queries, the bf16
// copy of A for the tensor-core projection and the rerank hand-off) lives in one file-scope
// __device__ array instead of a workspace obtained with cudaMalloc.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "beam.cuh"
#include "common.cuh"
#include "index.cuh"

namespace lv {

int launch_project_fp32(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy,
                        cudaStream_t st);
int launch_pad_rows(const float *X, int64_t n, int D, float *Y, int ldy, cudaStream_t st);
bool project_bf16_fused_ok(const float *X, int D, int d);
size_t project_tc_ws_bytes(int prec, int64_t n, int D, int d, const float *X);
int project_bf16(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, void **ws,
                 size_t *ws_bytes, int *status, cudaStream_t st);

// 16 MiB, held by every GPU that loads this library until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;
constexpr size_t NOALLOC_HEADER_BYTES = 256;  // work counter, padded
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch for each device ordinal, looked up once per
// device with that device current.  In host code the array's name only stands for
// the symbol; it is never dereferenced or passed to a kernel.
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[128] = {};

static int noalloc_scratch(int device, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (device < 0 || device >= 128) return fail(LV_ERR_ARG, "search_noalloc: unsupported device ordinal");
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "search_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_addr[device]);
    return LV_OK;
}

}  // namespace lv

using namespace lv;

extern "C" int leanvec_search_noalloc(lv_index *idx, const float *Q, int64_t m, const float *A,
                                      const lv_search_params *params, const lv_query_desc *desc, int32_t *ids,
                                      float *scores, int ldo, lv_search_stats *stats, lv_stream_t stream) {
    if (!idx || !params) return fail(LV_ERR_ARG, "search_noalloc: null index or params");
    if (m < 0 || m >= (int64_t)0x7fffffff) return fail(LV_ERR_ARG, "search_noalloc: invalid m");
    if (m == 0) return LV_OK;
    if (!Q || !ids || !scores) return fail(LV_ERR_ARG, "search_noalloc: null query or output pointer");
    if (idx->n == 0) return fail(LV_ERR_STATE, "search_noalloc: the index has no store");
    if (!idx->graph) return fail(LV_ERR_STATE, "search_noalloc: the index has no graph");
    if (idx->pbits != 32 && !A) return fail(LV_ERR_ARG, "search_noalloc: an LVQ index needs the projection A");
    const lv_query_desc &u = params->uniform;
    if (u.L < 1 || u.L > LCAP_MAX) return fail(LV_ERR_ARG, "search_noalloc: L must be in [1, 512]");
    if (!desc && (u.k < 1 || u.k > u.L || u.k > ldo || u.rerank < 0 || u.rerank > u.L || u.max_hops < 0))
        return fail(LV_ERR_ARG, "search_noalloc: need 1 <= k <= min(L, ldo), 0 <= rerank <= L, max_hops >= 0");
    if (u.rerank > 0 && !desc && !idx->sec) return fail(LV_ERR_STATE, "search_noalloc: rerank needs a secondary store");
    // the bf16 projection converts Q inside the GEMM and needs only a bf16 copy of A (in the
    // scratch); the other tensor-core paths would need a converted copy of Q
    // (a float32 index ignores the projection, as leanvec_search does)
    const bool bf16 = params->projection == LV_PREC_BF16 && idx->pbits != 32;
    if (params->projection < LV_PREC_FP32 || params->projection > LV_PREC_TF32X3)
        return fail(LV_ERR_ARG, "search_noalloc: projection precision must be an lv_precision value");
    if (idx->pbits != 32 && params->projection != LV_PREC_FP32 && !(bf16 && project_bf16_fused_ok(Q, idx->D, idx->d)))
        return fail(LV_ERR_ARG, "search_noalloc: the projection must be LV_PREC_FP32, or LV_PREC_BF16 with 16-byte "
                                "aligned query rows (D a multiple of 4)");
    if (idx->sbits == 8 && idx->sg.code_chunks + 1 + idx->metric > 64)
        return fail(LV_ERR_ARG, "search_noalloc: D > 1008 is not supported by the rerank");
    if (idx->sbits == 16 && idx->sg.code_chunks > 128)
        return fail(LV_ERR_ARG, "search_noalloc: D > 1024 is not supported by the FP16 rerank");

    const int cpc = idx->pbits == 8 ? 16 : idx->pbits == 4 ? 32 : 4;
    const int ldq = idx->pg.code_chunks * cpc;
    const size_t q_bytes = round_up((int64_t)sizeof(float) * m * ldq, 256);
    // rerank hand-off (beam kernel -> rerank kernel): m x Lcap ids + m counts
    const bool rerank = idx->sbits && idx->pbits != 32 && (desc || u.rerank > 0);
    const int Lcap = (int)round_up(u.L, 32);
    const size_t r_bytes = rerank ? (size_t)round_up((int64_t)sizeof(int32_t) * m * (Lcap + 1), 256) : 0;
    const size_t a_bytes = bf16 ? round_up((int64_t)project_tc_ws_bytes(LV_PREC_BF16, m, idx->D, idx->d, Q), 256) : 0;
    const size_t need = NOALLOC_HEADER_BYTES + q_bytes + r_bytes + a_bytes;
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(LV_ERR_CAPACITY, "search_noalloc: m * (4 * padded primary dimension [+ 4 * (L rounded up to "
                                     "32) + 4 with rerank]) + 256 [+ 2 d (D rounded up to 8) for a bf16 "
                                     "projection] bytes (each part rounded up to 256) exceed the 16 MiB static "
                                     "scratch; split the batch");

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return fail(LV_ERR_CUDA, "search_noalloc: cudaGetDevice failed");
    if (prev != idx->device && cudaSetDevice(idx->device) != cudaSuccess)
        return fail(LV_ERR_CUDA, "search_noalloc: cannot select the index's device");
    int rc = LV_OK;
    unsigned char *scratch = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    do {
        rc = noalloc_scratch(idx->device, &scratch);
        if (rc) break;
        int *work = reinterpret_cast<int *>(scratch);
        float *qp = reinterpret_cast<float *>(scratch + NOALLOC_HEADER_BYTES);
        int32_t *cand = reinterpret_cast<int32_t *>(scratch + NOALLOC_HEADER_BYTES + q_bytes);
        if (idx->pbits == 32) {
            rc = launch_pad_rows(Q, m, idx->D, qp, ldq, st);
        } else if (bf16) {
            void *ws = scratch + NOALLOC_HEADER_BYTES + q_bytes + r_bytes;
            size_t wsb = a_bytes;  // large enough: project_bf16 does not grow it
            rc = project_bf16(Q, m, idx->D, A, idx->d, qp, ldq, &ws, &wsb, idx->status, st);
        } else {
            rc = launch_project_fp32(Q, m, idx->D, A, idx->d, qp, ldq, st);
        }
        if (rc) break;

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
        p.qp = qp;
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
        p.work = work;
        int block = 0;
        size_t smem = 0;
        rc = search_shape(idx, params, p, &block, &smem, "search_noalloc");
        if (rc) break;
        if (rerank) {
            p.ldc = p.Lcap;
            p.cand = cand;
            p.cand_n = cand + (size_t)m * p.ldc;
        }
        // the scratch keeps the previous call's contents: the work counter must restart at 0
        cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int), st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "search_noalloc: cudaMemsetAsync");
            break;
        }
        if (params->event_begin && (e = cudaEventRecord((cudaEvent_t)params->event_begin, st)) != cudaSuccess) {
            rc = cuda_fail(e, "search_noalloc: cudaEventRecord(event_begin)");
            break;
        }
        rc = launch_beam_search(idx, p, block, smem, st);
        if (!rc && rerank) rc = launch_rerank(p, idx->num_sms, st);
        if (rc) break;
        if (params->event_end && (e = cudaEventRecord((cudaEvent_t)params->event_end, st)) != cudaSuccess) {
            rc = cuda_fail(e, "search_noalloc: cudaEventRecord(event_end)");
            break;
        }
    } while (0);
    if (prev >= 0 && prev != idx->device) cudaSetDevice(prev);
    return rc;
}
