// MAX aggregator helpers (see maxagg.cu).
#pragma once

#include "plan.cuh"

namespace relnn {

// Combines the (value, position) partials of tile-split segments in tile order into out / arg
// (arg = -1 where relu and the maximum is not positive).
relnn_status launch_fixup_max(const int32_t* seg, int64_t m, int tile, int64_t n_tiles, const float* carry,
                              const int32_t* carry_pos, float* out, int32_t* arg, int d_out, bool relu,
                              DevBuf& jobs_buf, cudaStream_t st);

// Words per tuple of the winner mask (the ReLU-mask layout: 4 words per 128 features).
int max_mask_words(int d_out);

// p.win_mask from p.max_arg of the plan's last forward (ENOTSUP if none ran).
relnn_status build_win_mask(Plan& p, cudaStream_t st);

}  // namespace relnn
