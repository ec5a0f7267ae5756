// RAAR frame pass for 256x256 frames, all flag variants and both row chunks
// of the batch tuner (single scan and batch share the kernel).
#include "frame256.cuh"

namespace sharp {

template <int RCH>
static cudaError_t launch_big_raar_c(int flags, const FrameArgs& a, const BatchTable* bt, int grid, float2* slab,
                                    cudaStream_t s) {
    switch (flags & (RF_FORM_B | RF_METRIC)) {
        case 0: return big_launch<MODE_RAAR, 0, RCH>(a, bt, grid, slab, s);
        case RF_FORM_B: return big_launch<MODE_RAAR, RF_FORM_B, RCH>(a, bt, grid, slab, s);
        case RF_METRIC: return big_launch<MODE_RAAR, RF_METRIC, RCH>(a, bt, grid, slab, s);
        default: return big_launch<MODE_RAAR, RF_FORM_B | RF_METRIC, RCH>(a, bt, grid, slab, s);
    }
}

cudaError_t launch_big_raar(int flags, const FrameArgs& a, const BatchTable* bt, int grid, float2* slab,
                            cudaStream_t s, int ch) {
    if (ch == 4) return launch_big_raar_c<4>(flags, a, bt, grid, slab, s);
    if (ch == 8) return launch_big_raar_c<8>(flags, a, bt, grid, slab, s);
    return cudaErrorInvalidValue;
}

}  // namespace sharp
