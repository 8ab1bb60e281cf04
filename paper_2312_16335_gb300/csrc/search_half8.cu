// Two-queries-per-warp search instantiations for LVQ-8 primaries (chunks per lane 1..4).
#include "beam_half.cuh"

namespace lv {

int launch_search_half8(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st) {
    switch (nc) {
        case 1: return half_go_nc<1, 8>(p, block, smem, num_sms, st);
        case 2: return half_go_nc<2, 8>(p, block, smem, num_sms, st);
        case 3: return half_go_nc<3, 8>(p, block, smem, num_sms, st);
        case 4: return half_go_nc<4, 8>(p, block, smem, num_sms, st);
        default: return fail(LV_ERR_ARG, "search: primary dimension too large for LVQ-8 (d <= 240)");
    }
}

}  // namespace lv
