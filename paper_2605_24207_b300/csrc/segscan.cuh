// Register-level helpers shared by the tensor-core epilogues: a segmented running sum over the 32
// tuples (TMEM columns) one thread holds after a 32x32b.x32 load, and a select of v[j] for a
// warp-uniform run-time j. Both are branch-free so the unrolled bodies stay small in the I-cache.
#pragma once

#include "common.cuh"

namespace relnn {

// Segmented running sum over the 32 tuples of a chunk held by one epilogue thread (one feature):
// y = acc + bias (ReLU'd), sum restarts at every row whose bit is set in `startmask`, and v[j] is
// replaced by the sum of its piece up to row j. Branch-free, so the unrolled body stays small.
template <bool RELU, bool KAHAN, bool MASK>
__device__ __forceinline__ void seg_scan(uint32_t (&v)[32], float bo, unsigned startmask, float& sum, float& comp,
                                         uint32_t& mword, int lane) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        float y = __uint_as_float(v[j]) + bo;
        if (RELU) {
            if (MASK) {
                const unsigned w = __ballot_sync(0xffffffffu, y > 0.f);
                mword = (lane == j) ? w : mword;
            }
            y = fmaxf(y, 0.f);
        }
        const bool st = (startmask >> j) & 1u;
        if (KAHAN) {
            sum = st ? 0.f : sum;
            comp = st ? 0.f : comp;
            kahan_add(sum, comp, y);
        } else {
            sum = st ? y : sum + y;
        }
        v[j] = __float_as_uint(sum);
    }
}

// Segmented running maximum over the same 32 tuples: v[j] <- the maximum of its piece up to row j;
// bit j of `takemask` is set where row j becomes the piece's maximum (a piece start, or a value
// strictly above the running maximum), so the first position attaining the maximum of the piece
// up to row j is the highest set bit at or below j (or, with none, the carried position).
template <bool RELU>
__device__ __forceinline__ void seg_scan_max(uint32_t (&v)[32], float bo, unsigned startmask, float& run,
                                             unsigned& takemask) {
    unsigned tm = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        float y = __uint_as_float(v[j]) + bo;
        if (RELU) y = fmaxf(y, 0.f);
        const bool take = ((startmask >> j) & 1u) || y > run;
        run = take ? y : run;
        tm |= take ? (1u << j) : 0u;
        v[j] = __float_as_uint(run);
    }
    takemask = tm;
}

// v[j] for a warp-uniform run-time j without local-memory indexing (a 5-level select tree).
__device__ __forceinline__ uint32_t select32(const uint32_t (&v)[32], int j) {
    uint32_t t16[16], t8[8], t4[4];
#pragma unroll
    for (int i = 0; i < 16; ++i) t16[i] = (j & 1) ? v[2 * i + 1] : v[2 * i];
#pragma unroll
    for (int i = 0; i < 8; ++i) t8[i] = (j & 2) ? t16[2 * i + 1] : t16[2 * i];
#pragma unroll
    for (int i = 0; i < 4; ++i) t4[i] = (j & 4) ? t8[2 * i + 1] : t8[2 * i];
    const uint32_t a0 = (j & 8) ? t4[1] : t4[0];
    const uint32_t a1 = (j & 8) ? t4[3] : t4[2];
    return (j & 16) ? a1 : a0;
}

}  // namespace relnn
