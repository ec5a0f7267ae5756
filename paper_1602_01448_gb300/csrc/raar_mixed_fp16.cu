// Tensor-core RAAR frame pass and data projection, FP16 operands with per-frame
// power-of-two scaling (raar_mixed.cuh).
#include "raar_mixed.cuh"

namespace sharp {
template cudaError_t launch_mixed_prec<SHARP_PREC_FP16S>(int, int, const FrameArgs&, cudaStream_t);
}
