// Fused RAAR frame pass for 128 x 128 frames, periodic object indexing
// (one translation unit per variant so the build compiles them in parallel).
#include "raar_kernel.cuh"

namespace sharp {
template cudaError_t launch_raar_w<128, 1>(int, const FrameArgs&, cudaStream_t);
}  // namespace sharp
