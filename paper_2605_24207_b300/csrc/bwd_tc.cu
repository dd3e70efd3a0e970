// Backward of the BF16 form (placeholder until the tensor-core backward lands): the FP32 CUDA-core
// backward on the device.
#include "bwd.cuh"

namespace relnn {

relnn_status backward_tc(Plan& p, const CallIO& io, const GradIO& g, cudaStream_t st) {
    return backward_fp32(p, io, g, st);
}

}  // namespace relnn
