// Beam search in build mode: the queries are database nodes and the scores are the
// exact build score, so that graph construction is reproducible bit for bit.
#include "beam.cuh"

namespace lv {

template <int NC, int BITS, bool L2>
static int go(const BeamParams &p, int block, size_t smem, int num_sms, cudaStream_t st) {
    auto k = beam_kernel<BuildScorer<NC, BITS, L2>, true, false, 1>;
    LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    LV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem));
    if (per_sm < 1) return fail(LV_ERR_CAPACITY, "build: beam/visited capacity does not fit in shared memory");
    const int teams = block / 32 / p.T;  // queries served at once by one block
    int64_t want = (p.m + teams - 1) / teams;
    int64_t grid = std::min<int64_t>((int64_t)per_sm * num_sms, want);
    k<<<(unsigned)std::max<int64_t>(grid, 1), block, smem, st>>>(p);
    LV_CHECK_LAUNCH("beam_kernel<build>");
    return LV_OK;
}

template <int BITS, bool L2>
static int go_warp(const BeamParams &p, int block, size_t smem, int num_sms, cudaStream_t st) {
    auto k = beam_kernel<BuildWarpScorer<BITS, L2>, true, false, 1>;
    LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    LV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem));
    if (per_sm < 1) return fail(LV_ERR_CAPACITY, "build: beam/visited capacity does not fit in shared memory");
    const int teams = block / 32;
    int64_t want = (p.m + teams - 1) / teams;
    int64_t grid = std::min<int64_t>((int64_t)per_sm * num_sms, want);
    k<<<(unsigned)std::max<int64_t>(grid, 1), block, smem, st>>>(p);
    LV_CHECK_LAUNCH("beam_kernel<build, whole warp>");
    return LV_OK;
}

template <bool L2>
static int build_search_m(const BeamParams &p, int bits, int nc, int block, size_t smem, int num_sms,
                          cudaStream_t st) {
    // records longer than 4 lanes x 4 (LVQ-8) or 3 (LVQ-4) chunks: a whole warp per record
    if (p.prim_chunks + 1 + (L2 ? 1 : 0) <= 64 && ((bits == 8 && nc > 4) || (bits == 4 && nc > 3)))
        return bits == 8 ? go_warp<8, L2>(p, block, smem, num_sms, st) : go_warp<4, L2>(p, block, smem, num_sms, st);
    if (bits == 8) {
        switch (nc) {
            case 1: return go<1, 8, L2>(p, block, smem, num_sms, st);
            case 2: return go<2, 8, L2>(p, block, smem, num_sms, st);
            case 3: return go<3, 8, L2>(p, block, smem, num_sms, st);
            case 4: return go<4, 8, L2>(p, block, smem, num_sms, st);
        }
    } else if (bits == 4) {
        switch (nc) {
            case 1: return go<1, 4, L2>(p, block, smem, num_sms, st);
            case 2: return go<2, 4, L2>(p, block, smem, num_sms, st);
            case 3: return go<3, 4, L2>(p, block, smem, num_sms, st);
        }
    }
    return fail(LV_ERR_ARG, "build: unsupported primary record size");
}

int launch_build_search(const BeamParams &p, int bits, int nc, int block, size_t smem, int num_sms,
                        cudaStream_t st) {
    return p.metric ? build_search_m<true>(p, bits, nc, block, smem, num_sms, st)
                    : build_search_m<false>(p, bits, nc, block, smem, num_sms, st);
}

}  // namespace lv
