// Tensor-core RAAR frame pass and data projection for 256^2 frames,
// FP16 operands with per-frame power-of-two scaling (raar_mixed256.cuh).
#include "raar_mixed256.cuh"

namespace sharp {
template cudaError_t launch_mixed256_prec<SHARP_PREC_FP16S>(int, int, const FrameArgs&, float2*, cudaStream_t);
}
