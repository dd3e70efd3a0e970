// Forward of a planned rule: gather -> Concat -> Linear (+ReLU) -> segmented SUM by output key.
//
// Both forms cut the dst-sorted matched tuples into fixed tiles. Inside a tile every output row
// whose tuples all lie in the tile is written once with a plain store; a segment cut by a tile
// boundary leaves one partial per tile in `carry` (slot 0: the piece holding the tile's first row,
// slot 1: the piece holding its last row) and fixup_kernel adds the pieces in tile order
// (compensated with RELNN_FLAG_KAHAN) and writes the row. Results are deterministic.
#pragma once

#include "plan.cuh"

namespace relnn {

// Per-branch inputs of a forward/backward call, resolved from relnn_rule_params.
struct BranchIO {
    const void* r = nullptr;   // [n_tuples, d_r]
    const void* W = nullptr;   // [d_out, d_in]
    const float* b = nullptr;  // [d_out]
};

struct CallIO {
    const void* z = nullptr;
    int z_bf16 = 0, r_bf16 = 0, w_bf16 = 0;
    std::vector<BranchIO> br;
};

// The f32 H embedding rounded to bf16 (nearest even, as the tensor-core kernels round operands)
// in the plan's workspace, so that the tensor-core kernels gather it with cp.async; io.z unchanged
// when it is bf16 already. Returns the CallIO to use.
relnn_status with_bf16_z(Plan& p, const CallIO& io, CallIO& out, cudaStream_t st);

// dst[i] = bf16(src[i]) (nearest even) for n elements; n % 4 == 0, both pointers 16- and 8-byte aligned.
void f32_to_bf16(const float* src, int64_t n, uint16_t* dst, cudaStream_t st);

relnn_status forward_fp32(Plan& p, const CallIO& io, float* out, cudaStream_t st);
relnn_status forward_tc(Plan& p, const CallIO& io, float* out, cudaStream_t st);
// RELNN_FLAG_PUSHDOWN: the Linear once per H row, then per-tuple gathers and the SUM walk.
relnn_status forward_pushdown(Plan& p, const CallIO& io, float* out, cudaStream_t st);

// Attention over the plan's tuples (relnn_attention_forward / _backward; attention.cu).
relnn_status attention_forward(Plan& p, const relnn_attn_params* prm, float* out, float* lse, cudaStream_t st);
relnn_status attention_backward(Plan& p, const relnn_attn_params* prm, const float* fout, const float* flse,
                                const float* dout, float* dq, float* dk, float* dv, cudaStream_t st);

// Adds the carried partials of tile-split segments into `out` (see file comment).
relnn_status launch_fixup(const int32_t* seg, int64_t m, int tile, int64_t n_tiles, const float* carry,
                          float* out, int d_out, bool accumulate, bool kahan, DevBuf& jobs_buf, cudaStream_t st);

}  // namespace relnn
