// Standalone frame operators for 256x256 frames: P_a of explicit frames
// (Eq. 7), the forward model (Eq. 1), the amplitude loss and its adjoint, and
// the Fourier mask of the illumination constraint (Sec. 2.2, step 7).
#include "frame256.cuh"

namespace sharp {

cudaError_t launch_big_ops(int mode, const FrameArgs& a, cudaStream_t s) {
    switch (mode) {
        case MODE_PROJECT: return big_launch<MODE_PROJECT>(a, a.scratch, s);
        case MODE_AMPS: return big_launch<MODE_AMPS>(a, a.scratch, s);
        case MODE_LOSS: return big_launch<MODE_LOSS>(a, a.scratch, s);
        case MODE_GRAD: return big_launch<MODE_GRAD>(a, a.scratch, s);
        case MODE_MASK: return big_launch<MODE_MASK>(a, a.scratch, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sharp
