// Batched RAAR frame pass, 128x128 frames: all flag variants (a translation
// unit of its own so the build compiles it in parallel with the others).
#include "raar_kernel.cuh"

namespace sharp {
template cudaError_t launch_raar_batch_m<128>(int, const BatchTable&, int, cudaStream_t);
template cudaError_t raar_batch_max_grid<128>(int*);
}  // namespace sharp
