// Search of query batches held in host memory (leanvec_search_host): the batches are copied in,
// searched and copied out by the library, with the copies of neighbouring batches on two copy
// streams of the index's own so that they overlap the searches (Sec. 2 "Search" is the search
// itself; the staging is this library's).  Each batch is searched exactly as one leanvec_search
// call on device buffers.
#include "index.cuh"

namespace lv {

void host_slots_free(lv_index *idx) {
    auto &h = idx->hs;
    for (int b = 0; b < 2; ++b) {
        cudaFree(h.q[b]);
        cudaFree(h.desc[b]);
        cudaFree(h.ids[b]);
        cudaFree(h.sc[b]);
        h.q[b] = nullptr;
        h.desc[b] = nullptr;
        h.ids[b] = nullptr;
        h.sc[b] = nullptr;
        h.qb[b] = h.db[b] = h.ib[b] = h.sb[b] = 0;
        if (h.copied[b]) cudaEventDestroy(h.copied[b]);
        if (h.searched[b]) cudaEventDestroy(h.searched[b]);
        if (h.drained[b]) cudaEventDestroy(h.drained[b]);
        h.copied[b] = h.searched[b] = h.drained[b] = nullptr;
    }
    if (h.start) cudaEventDestroy(h.start);
    if (h.done) cudaEventDestroy(h.done);
    if (h.s_in) cudaStreamDestroy(h.s_in);
    if (h.s_out) cudaStreamDestroy(h.s_out);
    h.start = h.done = nullptr;
    h.s_in = h.s_out = nullptr;
}

// LV_OK, or the library's status for a failed CUDA call
static int ck(cudaError_t e, const char *what) { return e == cudaSuccess ? LV_OK : cuda_fail(e, what); }

static int host_slots_setup(lv_index *idx) {
    auto &h = idx->hs;
    if (h.s_in) return LV_OK;
    LV_CUDA(cudaStreamCreateWithFlags(&h.s_in, cudaStreamNonBlocking));
    LV_CUDA(cudaStreamCreateWithFlags(&h.s_out, cudaStreamNonBlocking));
    LV_CUDA(cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming));
    LV_CUDA(cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming));
    for (int b = 0; b < 2; ++b) {
        LV_CUDA(cudaEventCreateWithFlags(&h.copied[b], cudaEventDisableTiming));
        LV_CUDA(cudaEventCreateWithFlags(&h.searched[b], cudaEventDisableTiming));
        LV_CUDA(cudaEventCreateWithFlags(&h.drained[b], cudaEventDisableTiming));
    }
    return LV_OK;
}

}  // namespace lv

using namespace lv;

extern "C" {

int leanvec_search_host(lv_index *idx, const float *Q, int64_t m, const float *A, const lv_search_params *params,
                        const lv_query_desc *desc, int32_t *ids, float *scores, int ldo, int64_t batch,
                        lv_stream_t stream) {
    if (!idx || !params) return fail(LV_ERR_ARG, "search_host: null index or params");
    if (m < 0 || m >= (int64_t)0x7fffffff) return fail(LV_ERR_ARG, "search_host: invalid m");
    if (m == 0) return LV_OK;
    if (!Q || !ids || !scores) return fail(LV_ERR_ARG, "search_host: null query or output pointer");
    if (idx->n == 0) return fail(LV_ERR_STATE, "search_host: the index has no store");
    if (ldo < 1) return fail(LV_ERR_ARG, "search_host: ldo must be >= 1");
    const int64_t bt = batch > 0 ? std::min(batch, m) : m;
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "search_host: cannot select device");
    int rc = host_slots_setup(idx);
    if (rc) return rc;
    auto &h = idx->hs;
    const int D = idx->D;
    const int nslot = m > bt ? 2 : 1;
    for (int b = 0; b < nslot; ++b) {
        if ((rc = ensure_ws((void **)&h.q[b], &h.qb[b], sizeof(float) * (size_t)bt * D))) return rc;
        if ((rc = ensure_ws((void **)&h.ids[b], &h.ib[b], sizeof(int32_t) * (size_t)bt * ldo))) return rc;
        if ((rc = ensure_ws((void **)&h.sc[b], &h.sb[b], sizeof(float) * (size_t)bt * ldo))) return rc;
        if (desc && (rc = ensure_ws((void **)&h.desc[b], &h.db[b], sizeof(lv_query_desc) * (size_t)bt))) return rc;
    }
    lv_search_params prm = *params;
    prm.event_begin = prm.event_end = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    // the copies start after the caller's earlier work on `stream`
    LV_CUDA(cudaEventRecord(h.start, st));
    LV_CUDA(cudaStreamWaitEvent(h.s_in, h.start, 0));
    LV_CUDA(cudaStreamWaitEvent(h.s_out, h.start, 0));
    int64_t nb = (m + bt - 1) / bt;
    for (int64_t i = 0; i < nb && rc == LV_OK; ++i) {
        const int s = (int)(i & 1);
        const int64_t q0 = i * bt, mb = std::min(bt, m - q0);
        // slot s: its queries are overwritten once the search two batches back has read them
        if (i >= 2 && (rc = ck(cudaStreamWaitEvent(h.s_in, h.searched[s], 0), "search_host: wait"))) break;
        if ((rc = ck(cudaMemcpyAsync(h.q[s], Q + q0 * D, sizeof(float) * (size_t)mb * D,
                                            cudaMemcpyHostToDevice, h.s_in), "search_host: query copy")))
            break;
        if (desc && (rc = ck(cudaMemcpyAsync(h.desc[s], desc + q0, sizeof(lv_query_desc) * (size_t)mb,
                                                    cudaMemcpyHostToDevice, h.s_in), "search_host: desc copy")))
            break;
        if ((rc = ck(cudaEventRecord(h.copied[s], h.s_in), "search_host: event"))) break;
        if ((rc = ck(cudaStreamWaitEvent(st, h.copied[s], 0), "search_host: wait"))) break;
        // and its results are overwritten once they have left the device
        if (i >= 2 && (rc = ck(cudaStreamWaitEvent(st, h.drained[s], 0), "search_host: wait"))) break;
        rc = leanvec_search(idx, h.q[s], mb, A, &prm, desc ? h.desc[s] : nullptr, h.ids[s], h.sc[s], ldo, nullptr,
                            stream);
        if (rc) break;
        if ((rc = ck(cudaEventRecord(h.searched[s], st), "search_host: event"))) break;
        if ((rc = ck(cudaStreamWaitEvent(h.s_out, h.searched[s], 0), "search_host: wait"))) break;
        if ((rc = ck(cudaMemcpyAsync(ids + q0 * ldo, h.ids[s], sizeof(int32_t) * (size_t)mb * ldo,
                                            cudaMemcpyDeviceToHost, h.s_out), "search_host: id copy")))
            break;
        if ((rc = ck(cudaMemcpyAsync(scores + q0 * ldo, h.sc[s], sizeof(float) * (size_t)mb * ldo,
                                            cudaMemcpyDeviceToHost, h.s_out), "search_host: score copy")))
            break;
        rc = ck(cudaEventRecord(h.drained[s], h.s_out), "search_host: event");
    }
    // `stream`'s later work waits for every copy issued (also after a failure)
    cudaError_t e1 = cudaEventRecord(h.done, h.s_in);
    cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(st, h.done, 0) : e1;
    cudaError_t e3 = cudaEventRecord(h.done, h.s_out);
    cudaError_t e4 = e3 == cudaSuccess ? cudaStreamWaitEvent(st, h.done, 0) : e3;
    if (rc) return rc;
    if (e2 != cudaSuccess) return cuda_fail(e2, "search_host: join");
    if (e4 != cudaSuccess) return cuda_fail(e4, "search_host: join");
    return LV_OK;
}

}  // extern "C"
