// Two-queries-per-warp search instantiations for LVQ-4 primaries (chunks per lane 1..3).
#include "beam_half.cuh"

namespace lv {

int launch_search_half4(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st) {
    switch (nc) {
        case 1: return half_go_nc<1, 4>(p, block, smem, num_sms, st);
        case 2: return half_go_nc<2, 4>(p, block, smem, num_sms, st);
        case 3: return half_go_nc<3, 4>(p, block, smem, num_sms, st);
        default: return fail(LV_ERR_ARG, "search: primary dimension too large for LVQ-4 (d <= 320)");
    }
}

}  // namespace lv
