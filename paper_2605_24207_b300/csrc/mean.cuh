// MEAN aggregator helpers (see mean.cu).
#pragma once

#include "plan.cuh"

namespace relnn {

// 1 / (matched tuples of each output row) of a single-branch plan, built once into p.inv_cnt.
relnn_status ensure_inv_count(Plan& p, cudaStream_t st);
// cnt[seg[i]] += 1 for i < m (matched tuples per output row, added to existing counts).
relnn_status count_rows_into(const int32_t* seg, int64_t m, int32_t* cnt, cudaStream_t st);
// dst[k][:] = src[k][:] * inv[k] for n rows of width d (dst may equal src).
relnn_status scale_rows(const float* src, const float* inv, int64_t n, int d, float* dst, cudaStream_t st);

}  // namespace relnn
