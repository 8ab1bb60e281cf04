// Stream-ordered scratch allocator of the library.  The temporaries of the offline calls
// (bf16 / e4m3 operand copies, split-K partials, the FP64 eigen-solver matrices, fit and
// loss buffers) come from one memory pool per device that keeps freed blocks mapped
// (release threshold unlimited): a repeated call reuses device memory instead of mapping
// and unmapping it, and no call pays the device-wide synchronisation of cudaFree.
// The stores of an index (records, graph, search workspaces) are not scratch and keep
// their own allocations.
#include <mutex>

#include "common.cuh"

namespace lv {

constexpr int MAX_DEVICES = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[MAX_DEVICES];
static bool g_have_pool[MAX_DEVICES];

static int pool_of(int dev, bool create, cudaMemPool_t *out) {
    if (dev < 0 || dev >= MAX_DEVICES) return fail(LV_ERR_ARG, "scratch pool: device ordinal out of range");
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (!g_have_pool[dev]) {
        if (!create) {
            *out = nullptr;
            return LV_OK;
        }
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        LV_CUDA(cudaMemPoolCreate(&g_pools[dev], &props));
        uint64_t keep = ~0ull;
        LV_CUDA(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
        g_have_pool[dev] = true;
    }
    *out = g_pools[dev];
    return LV_OK;
}

// bytes of scratch on the current device, ordered on `st`; *p = nullptr for 0 bytes
int tmp_alloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) return LV_OK;
    int dev = -1;
    LV_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    int rc = pool_of(dev, true, &pool);
    if (rc) return rc;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(LV_ERR_OOM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return LV_OK;
}

void tmp_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

}  // namespace lv

using namespace lv;

extern "C" int leanvec_trim_scratch(int device) {
    cudaMemPool_t pool = nullptr;
    int rc = pool_of(device, false, &pool);
    if (rc || !pool) return rc;
    LV_CUDA(cudaMemPoolTrimTo(pool, 0));
    return LV_OK;
}
