// Full-dimensional float32 graph search (the baseline the paper compares against):
// the same beam kernel with whole-warp float32 record scoring and no rerank.
#include "beam.cuh"

namespace lv {

template <int NCW, int WT, bool L2>
static int go_w(const BeamParams &p, int block, size_t smem, int num_sms, cudaStream_t st) {
    auto k = beam_kernel<WarpScorer<NCW, 0, L2>, false, false, WT>;
    LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    LV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem));
    if (per_sm < 1) return fail(LV_ERR_CAPACITY, "search: beam/visited capacity does not fit in shared memory");
    const int teams = block / 32 / p.T;  // queries served at once by one block
    if (p.slots) {
        *p.slots = (int64_t)per_sm * num_sms * teams;
        return LV_OK;
    }
    int64_t want = (p.m + teams - 1) / teams;
    int64_t grid = std::min<int64_t>((int64_t)per_sm * num_sms, want);
    k<<<(unsigned)std::max<int64_t>(grid, 1), block, smem, st>>>(p);
    LV_CHECK_LAUNCH("beam_kernel<fp32>");
    return LV_OK;
}

template <int NCW>
static int go(const BeamParams &p, int block, size_t smem, int num_sms, cudaStream_t st) {
    // widths 1 and 2 get their own instantiations (fixed-trip parent loops); 3 and 4 the generic one
    if (p.metric) {
        if (p.W == 1) return go_w<NCW, 1, true>(p, block, smem, num_sms, st);
        if (p.W == 2) return go_w<NCW, 2, true>(p, block, smem, num_sms, st);
        return go_w<NCW, 0, true>(p, block, smem, num_sms, st);
    }
    if (p.W == 1) return go_w<NCW, 1, false>(p, block, smem, num_sms, st);
    if (p.W == 2) return go_w<NCW, 2, false>(p, block, smem, num_sms, st);
    return go_w<NCW, 0, false>(p, block, smem, num_sms, st);
}

int launch_search_fp32(const BeamParams &p, int ncw, int block, size_t smem, int num_sms, cudaStream_t st) {
    if (ncw <= 1) return go<1>(p, block, smem, num_sms, st);
    if (ncw <= 2) return go<2>(p, block, smem, num_sms, st);
    if (ncw <= 4) return go<4>(p, block, smem, num_sms, st);
    if (ncw <= 6) return go<6>(p, block, smem, num_sms, st);
    if (ncw <= 8) return go<8>(p, block, smem, num_sms, st);
    return fail(LV_ERR_ARG, "search: float32 records longer than 1024 floats are not supported");
}

}  // namespace lv
