// Batched RAAR frame pass, 64x64 frames: all flag variants (a translation
// unit of its own so the build compiles it in parallel with the others).
#include "raar_kernel.cuh"

namespace sharp {
template cudaError_t launch_raar_batch_m<64>(int, const BatchTable&, int, cudaStream_t);
template cudaError_t raar_batch_max_grid<64>(int*);
}  // namespace sharp
