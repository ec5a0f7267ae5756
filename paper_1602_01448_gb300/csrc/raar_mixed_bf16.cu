// Tensor-core RAAR frame pass and data projection, BF16 three-term split
// operands (raar_mixed.cuh).
#include "raar_mixed.cuh"

namespace sharp {
template cudaError_t launch_mixed_prec<SHARP_PREC_BF16X3>(int, int, const FrameArgs&, cudaStream_t);
}
