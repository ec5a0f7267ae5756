// Batched RAAR frame pass, 64x64 frames, 4 rows per load / epilogue round
// trip: all flag variants (a translation unit of its own so the build compiles
// the tile shapes of the batch tuner in parallel).
#include "raar_kernel.cuh"

namespace sharp {
template cudaError_t launch_raar_batch_mc<64, 4>(int, const BatchTable&, int, cudaStream_t);
}  // namespace sharp
