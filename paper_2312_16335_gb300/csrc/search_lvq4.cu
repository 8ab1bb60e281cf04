// Search + rerank instantiations for LVQ-4 primaries, visited cache of 32-bit ids.
#include "search_launch.cuh"

namespace lv {

int launch_search_lvq4(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st) {
    if (p.vbits == 16) return launch_search_lvq4_tags(p, nc, block, smem, num_sms, st);
    return launch_search_lvq<4, false>(p, nc, block, smem, num_sms, st);
}

}  // namespace lv
