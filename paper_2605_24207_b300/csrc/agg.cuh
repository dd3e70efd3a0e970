// Aggregate-first evaluation of linear SUM rules on tcgen05 tensor cores (agg.cu).
#pragma once

#include <cuda.h>

#include "bwd.cuh"

namespace relnn {

// Whether the forward of the plan runs aggregate-first with these inputs: BF16 form, no activation,
// SUM or MEAN, no per-tuple embedding, d a power of two in [8, 256], d_out <= 256 and a multiple
// of 4, not a streamed chunk, RELNN_FLAG_PER_TUPLE not set, z and out 16-byte aligned.
bool agg_forward_ok(const Plan& p, const CallIO& io, const float* out);
// The same for the backward (also: no MAX, d_out a power of two in [8, 256], d a multiple of 32,
// dOut and dz 16-byte aligned).
bool agg_backward_ok(const Plan& p, const CallIO& io, const GradIO& g);

relnn_status forward_agg(Plan& p, const CallIO& io, float* out, cudaStream_t st);
// FP32 form (f32 on CUDA cores), aggregate-first: no activation, SUM or MEAN, no per-tuple
// embedding, unique H keys (or no dst part), d in {4, 8, 16, 32}, d_out a multiple of 4 (<= 256),
// f32 z and W, z / W / out 16-byte aligned, RELNN_FLAG_PER_TUPLE not set, not a streamed chunk.
bool agg_forward_fp32_ok(const Plan& p, const CallIO& io, const float* out);
relnn_status forward_agg_fp32(Plan& p, const CallIO& io, float* out, cudaStream_t st);
// FP32 form, identity rules (no Linear, no activation, Concat = z_src only, no per-tuple embedding):
// the aggregate-first gather-sum for d in {4, 8, 16, 32, 64, 128}, f32 z, z / out 16-byte aligned,
// RELNN_FLAG_PER_TUPLE not set, not a streamed chunk.
bool agg_forward_identity_ok(const Plan& p, const CallIO& io, const float* out);
relnn_status forward_agg_identity(Plan& p, const CallIO& io, float* out, cudaStream_t st);
relnn_status backward_agg(Plan& p, const CallIO& io, const GradIO& g, cudaStream_t st);

// 2-D bf16 tensor map over a row-major [rows][cols] matrix, box 64 columns x box_rows rows, 128-byte
// swizzle (the K-major layout the tensor-core kernels stage their operands in); rows past the end
// load as zeros.
relnn_status encode_bf16_tile_map(CUtensorMap* m, void* base, uint64_t cols, uint64_t rows, uint32_t box_rows = 128);

}  // namespace relnn
