// Backward of a planned rule (the fit of paper Sec. 2.3 optimises both the Linear weights and the
// per-tuple embeddings, Sec. 3.6): SUM backward broadcasts dOut[key] to the key's tuples, ReLU masks
// by the pre-activation, Linear gives dW = dY^T X, db = sum dY, dX = dY W, and the Concat backward
// adds each slice of dX to the embedding row it was gathered from (reusing the plan's join index).
#pragma once

#include "fwd.cuh"

namespace relnn {

struct GradIO {
    const float* dout = nullptr;          // [n_out, d_out]
    std::vector<float*> dW, db, dr;       // per branch (entries may be null)
    float* dz = nullptr;                  // [n_h, d]
    bool accumulate_dz = false;           // add into dz instead of overwriting it (stream chunks)
};

relnn_status backward_fp32(Plan& p, const CallIO& io, const GradIO& g, cudaStream_t st);
relnn_status backward_tc(Plan& p, const CallIO& io, const GradIO& g, cudaStream_t st);

}  // namespace relnn
