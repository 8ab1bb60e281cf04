// Search + rerank instantiations for LVQ-8 primaries, visited cache of 32-bit ids.
#include "search_launch.cuh"

namespace lv {

int launch_search_lvq8(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st) {
    if (p.vbits == 16) return launch_search_lvq8_tags(p, nc, block, smem, num_sms, st);
    return launch_search_lvq<8, false>(p, nc, block, smem, num_sms, st);
}

}  // namespace lv
