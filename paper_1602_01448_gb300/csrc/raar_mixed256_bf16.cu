// Tensor-core RAAR frame pass and data projection for 256^2 frames,
// BF16 three-term split operands (raar_mixed256.cuh).
#include "raar_mixed256.cuh"

namespace sharp {
template cudaError_t launch_mixed256_prec<SHARP_PREC_BF16X3>(int, int, const FrameArgs&, float2*, cudaStream_t);
}
