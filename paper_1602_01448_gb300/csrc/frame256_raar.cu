// RAAR frame pass for 256x256 frames, all flag variants (single scan and
// batch share the kernel).
#include "frame256.cuh"

namespace sharp {

cudaError_t launch_big_raar(int flags, const FrameArgs& a, const BatchTable* bt, int grid, float2* slab,
                            cudaStream_t s) {
    switch (flags & (RF_FORM_B | RF_METRIC)) {
        case 0: return big_launch<MODE_RAAR, 0>(a, bt, grid, slab, s);
        case RF_FORM_B: return big_launch<MODE_RAAR, RF_FORM_B>(a, bt, grid, slab, s);
        case RF_METRIC: return big_launch<MODE_RAAR, RF_METRIC>(a, bt, grid, slab, s);
        default: return big_launch<MODE_RAAR, RF_FORM_B | RF_METRIC>(a, bt, grid, slab, s);
    }
}

}  // namespace sharp
