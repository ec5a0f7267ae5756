// FP32 RAAR frame pass for 256^2 frames through four 128^2 register-resident
// transforms (raar_split256.cuh): the single-scan variants.
#include "raar_split256.cuh"

namespace sharp {

cudaError_t launch_split256(int flags, const FrameArgs& a, float2* slab, cudaStream_t s) {
    if (a.K <= 0) return cudaSuccess;
    const int f = flags & (RF_FORM_B | RF_METRIC);
    if (a.wrap) {
        switch (f) {
            case 0: return launch_split256_one<0, 1, 4>(a, nullptr, 0, slab, s);
            case RF_FORM_B: return launch_split256_one<RF_FORM_B, 1, 4>(a, nullptr, 0, slab, s);
            case RF_METRIC: return launch_split256_one<RF_METRIC, 1, 4>(a, nullptr, 0, slab, s);
            default: return launch_split256_one<RF_FORM_B | RF_METRIC, 1, 4>(a, nullptr, 0, slab, s);
        }
    }
    switch (f) {
        case 0: return launch_split256_one<0, 0, 4>(a, nullptr, 0, slab, s);
        case RF_FORM_B: return launch_split256_one<RF_FORM_B, 0, 4>(a, nullptr, 0, slab, s);
        case RF_METRIC: return launch_split256_one<RF_METRIC, 0, 4>(a, nullptr, 0, slab, s);
        default: return launch_split256_one<RF_FORM_B | RF_METRIC, 0, 4>(a, nullptr, 0, slab, s);
    }
}

}  // namespace sharp
