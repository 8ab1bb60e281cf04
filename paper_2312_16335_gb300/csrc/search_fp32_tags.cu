// Full-dimensional float32 graph search, visited cache of 16-bit tags.
#include "search_launch.cuh"

namespace lv {

int launch_search_fp32_tags(const BeamParams &p, int ncw, int block, size_t smem, int num_sms, cudaStream_t st) {
    return launch_search_f32<true>(p, ncw, block, smem, num_sms, st);
}

}  // namespace lv
