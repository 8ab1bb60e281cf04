// Search + rerank instantiations for LVQ-4 primaries, visited cache of 16-bit tags.
#include "search_launch.cuh"

namespace lv {

int launch_search_lvq4_tags(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st) {
    return launch_search_lvq<4, true>(p, nc, block, smem, num_sms, st);
}

}  // namespace lv
