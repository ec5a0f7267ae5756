// FP32 RAAR frame pass for 256^2 frames through four 128^2 register-resident
// transforms (raar_split256.cuh): the batch variants (scans of a batch, wrap
// read per scan), both row chunks of the batch tuner.
#include "raar_split256.cuh"

namespace sharp {

template <int LCH>
static cudaError_t launch_split256_batch_c(int flags, const BatchTable& bt, int grid, float2* slab, cudaStream_t s) {
    FrameArgs none;
    memset(&none, 0, sizeof(none));
    switch (flags & (RF_FORM_B | RF_METRIC)) {
        case 0: return launch_split256_one<0, -1, LCH>(none, &bt, grid, slab, s);
        case RF_FORM_B: return launch_split256_one<RF_FORM_B, -1, LCH>(none, &bt, grid, slab, s);
        case RF_METRIC: return launch_split256_one<RF_METRIC, -1, LCH>(none, &bt, grid, slab, s);
        default: return launch_split256_one<RF_FORM_B | RF_METRIC, -1, LCH>(none, &bt, grid, slab, s);
    }
}

cudaError_t launch_split256_batch(int flags, const BatchTable& bt, int grid, float2* slab, cudaStream_t s, int ch) {
    if (ch == 2) return launch_split256_batch_c<2>(flags, bt, grid, slab, s);
    if (ch == 4) return launch_split256_batch_c<4>(flags, bt, grid, slab, s);
    return cudaErrorInvalidValue;
}

}  // namespace sharp
