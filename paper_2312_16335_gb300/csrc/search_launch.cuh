// Launchers of the search instantiations of the beam kernel (beam.cuh): a persistent grid of
// as many blocks as stay resident, each warp (or team of warps) pulling queries from the
// batch's counter.  The instantiations are spread over several translation units so that
// they compile in parallel: one unit per primary encoding and visited-cache slot width.
#pragma once

#include "beam.cuh"

namespace lv {

// the scorers as templates of the metric alone (L2 = true: Euclidean scores)
template <int NC, int BITS>
struct LvqAt {
    template <bool L2>
    using S = LvqIntScorer<NC, BITS, L2>;
};
template <int NCW>
struct WarpAt {
    template <bool L2>
    using S = WarpScorer<NCW, 0, L2>;
};

template <class K>
int launch_persistent(K k, const BeamParams &p, int block, size_t smem, int num_sms, cudaStream_t st,
                      const char *name) {
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
    LV_CHECK_LAUNCH(name);
    return LV_OK;
}

// widths 1 and 2 get their own instantiations (fixed-trip parent loops); 3 and 4 the generic one
template <template <bool> class PS, bool RERANK, bool TAGS>
int launch_by_width(const BeamParams &p, int block, size_t smem, int num_sms, cudaStream_t st, const char *name) {
    if (p.metric) {
        if (p.W == 1) return launch_persistent(beam_kernel<PS<true>, false, RERANK, 1, TAGS>, p, block, smem, num_sms, st, name);
        if (p.W == 2) return launch_persistent(beam_kernel<PS<true>, false, RERANK, 2, TAGS>, p, block, smem, num_sms, st, name);
        return launch_persistent(beam_kernel<PS<true>, false, RERANK, 0, TAGS>, p, block, smem, num_sms, st, name);
    }
    if (p.W == 1) return launch_persistent(beam_kernel<PS<false>, false, RERANK, 1, TAGS>, p, block, smem, num_sms, st, name);
    if (p.W == 2) return launch_persistent(beam_kernel<PS<false>, false, RERANK, 2, TAGS>, p, block, smem, num_sms, st, name);
    return launch_persistent(beam_kernel<PS<false>, false, RERANK, 0, TAGS>, p, block, smem, num_sms, st, name);
}

// LVQ primaries (BITS 8: chunks per lane 1..4; BITS 4: 1..3), search + rerank hand-off
template <int BITS, bool TAGS>
int launch_search_lvq(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st) {
    const char *name = BITS == 8 ? "beam_kernel<lvq8>" : "beam_kernel<lvq4>";
    switch (nc) {
        case 1: return launch_by_width<LvqAt<1, BITS>::template S, true, TAGS>(p, block, smem, num_sms, st, name);
        case 2: return launch_by_width<LvqAt<2, BITS>::template S, true, TAGS>(p, block, smem, num_sms, st, name);
        case 3: return launch_by_width<LvqAt<3, BITS>::template S, true, TAGS>(p, block, smem, num_sms, st, name);
        case 4:
            if constexpr (BITS == 8) return launch_by_width<LvqAt<4, BITS>::template S, true, TAGS>(p, block, smem, num_sms, st, name);
            [[fallthrough]];
        default:
            return fail(LV_ERR_ARG, BITS == 8 ? "search: primary dimension too large for LVQ-8 (d <= 240)"
                                              : "search: primary dimension too large for LVQ-4 (d <= 352)");
    }
}

// full-dimensional float32 records (the baseline the paper compares against), no rerank
template <bool TAGS>
int launch_search_f32(const BeamParams &p, int ncw, int block, size_t smem, int num_sms, cudaStream_t st) {
    const char *name = "beam_kernel<fp32>";
    if (ncw <= 1) return launch_by_width<WarpAt<1>::template S, false, TAGS>(p, block, smem, num_sms, st, name);
    if (ncw <= 2) return launch_by_width<WarpAt<2>::template S, false, TAGS>(p, block, smem, num_sms, st, name);
    if (ncw <= 4) return launch_by_width<WarpAt<4>::template S, false, TAGS>(p, block, smem, num_sms, st, name);
    if (ncw <= 6) return launch_by_width<WarpAt<6>::template S, false, TAGS>(p, block, smem, num_sms, st, name);
    if (ncw <= 8) return launch_by_width<WarpAt<8>::template S, false, TAGS>(p, block, smem, num_sms, st, name);
    return fail(LV_ERR_ARG, "search: float32 records longer than 1024 floats are not supported");
}

}  // namespace lv
