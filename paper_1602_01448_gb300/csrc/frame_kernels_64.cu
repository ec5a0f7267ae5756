// Frame kernels for 64 x 64 frames (one translation unit per frame size so
// the build compiles them in parallel).
#include "frame_kernel.cuh"

namespace sharp {
template cudaError_t launch_frames_m<64>(int, int, const FrameArgs&, cudaStream_t);
}  // namespace sharp
