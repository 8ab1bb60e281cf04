// Internal definition of the opaque lv_index (shared by the host-side sources).
#pragma once

#include "common.cuh"

struct lv_index {
    int device = 0;
    int num_sms = 0;
    int metric = 0;  // LV_METRIC_IP or LV_METRIC_L2
    int64_t n = 0;
    int D = 0, d = 0;
    int pbits = 0, sbits = 0;
    lv::RecGeom pg, sg;
    uint8_t *prim = nullptr;
    float *pmean = nullptr;
    uint8_t *sec = nullptr;
    float *smean = nullptr;
    float mu2 = 0.f;
    int R = 0;
    int32_t *graph = nullptr;
    int32_t entry = -1;
    int *status = nullptr;  // device: [0] status bits, [1] work counter
    // search workspace
    float *ws_q = nullptr;
    size_t ws_q_bytes = 0;
    int32_t *ws_cand = nullptr;  // rerank hand-off: m x Lcap ids + m counts
    size_t ws_cand_bytes = 0;
    // build workspace
    void *bws = nullptr;
    size_t bws_bytes = 0;
    // second stream of the search's sub-batch, and its fork / join events (created on first use)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int last_kernels = 0;  // kernels launched by the last search call
    // leanvec_search_host: two device staging slots (queries, descriptors, results), the copy
    // streams and the events that order them (created on first use)
    struct HostSlots {
        float *q[2] = {nullptr, nullptr};
        lv_query_desc *desc[2] = {nullptr, nullptr};
        int32_t *ids[2] = {nullptr, nullptr};
        float *sc[2] = {nullptr, nullptr};
        size_t qb[2] = {0, 0}, db[2] = {0, 0}, ib[2] = {0, 0}, sb[2] = {0, 0};
        cudaStream_t s_in = nullptr, s_out = nullptr;
        cudaEvent_t start = nullptr, done = nullptr;
        cudaEvent_t copied[2] = {nullptr, nullptr}, searched[2] = {nullptr, nullptr}, drained[2] = {nullptr, nullptr};
    } hs;
};

namespace lv {
// Makes the index's device current for the scope of an API call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && (prev == dev || cudaSetDevice(dev) == cudaSuccess)) ok = true;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void index_free_stores(lv_index *idx);
void host_slots_free(lv_index *idx);
int ensure_ws(void **p, size_t *have, size_t want);
}  // namespace lv
