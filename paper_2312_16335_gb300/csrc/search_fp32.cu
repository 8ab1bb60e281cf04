// Full-dimensional float32 graph search (the baseline the paper compares against): the same
// beam kernel with whole-warp float32 record scoring and no rerank; visited cache of 32-bit ids.
#include "search_launch.cuh"

namespace lv {

int launch_search_fp32(const BeamParams &p, int ncw, int block, size_t smem, int num_sms, cudaStream_t st) {
    if (p.vbits == 16) return launch_search_fp32_tags(p, ncw, block, smem, num_sms, st);
    return launch_search_f32<false>(p, ncw, block, smem, num_sms, st);
}

}  // namespace lv
