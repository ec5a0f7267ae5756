// Batched RAAR frame pass, 64x64 frames, 8 rows per load / epilogue round
// trip: all flag variants (a translation unit of its own so the build compiles
// the tile shapes of the batch tuner in parallel).
#include "raar_kernel.cuh"

namespace sharp {
template cudaError_t launch_raar_batch_mc<64, 8>(int, const BatchTable&, int, cudaStream_t);
template cudaError_t raar_batch_max_grid<64>(int*);
}  // namespace sharp
