// Boundary partials of segments cut by fixed tiles (shared by the fix-ups of the MAX aggregator
// and of attention): which boundary first cuts a segment, and where its pieces' partials live.
// A forward that cuts the dst-sorted tuples into tiles leaves, per tile, slot 0 = the piece holding
// the tile's first row and slot 1 = the piece holding its last row when those rows' segments cross
// the tile's edges.
#pragma once

#include "common.cuh"

namespace relnn {

// Boundary b (1 <= b < n_tiles, tiles of `tile` rows) is the first boundary that cuts segment s:
// returns true with s, the carry slot of s's piece in tile b - 1 and the last tile e whose first
// row lies in s. Warp-collective (all lanes return the same).
__device__ __forceinline__ bool first_cut(const int32_t* __restrict__ seg, int64_t m, int tile, int64_t b, int lane,
                                          int& s, int& first_slot, int64_t& e) {
    const int64_t row = b * tile;  // < m
    int v = -1;
    if (lane == 0) v = seg[row];
    else if (lane == 1) v = seg[row - 1];
    else if (lane == 2) v = seg[(b - 1) * tile];
    else if (lane == 3 && b >= 2) v = seg[(b - 1) * tile - 1];
    else if (lane == 4 && row + tile < m) v = seg[row + tile];
    s = __shfl_sync(0xffffffffu, v, 0);
    if (__shfl_sync(0xffffffffu, v, 1) != s) return false;          // b cuts no segment
    if (b >= 2 && __shfl_sync(0xffffffffu, v, 3) == s) return false;  // s was cut before b
    first_slot = __shfl_sync(0xffffffffu, v, 2) == s ? 0 : 1;
    e = b;
    if (__shfl_sync(0xffffffffu, v, 4) == s) {  // s reaches past tile b: find its last row
        int64_t last = 0;
        if (lane == 0) {
            int64_t lo = row + tile, hi = m;
            while (lo + 1 < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (seg[mid] == s) lo = mid;
                else hi = mid;
            }
            last = lo;
        }
        e = __shfl_sync(0xffffffffu, last, 0) / tile;
    }
    return true;
}

// piece i of the segment first cut at b: 0 = its piece in tile b - 1, i >= 1 = slot 0 of tile b + i - 1
__device__ __forceinline__ int64_t piece_slot(int64_t b, int first_slot, int64_t i) {
    return i == 0 ? (b - 1) * 2 + first_slot : (b + i - 1) * 2;
}

}  // namespace relnn
