// Device-wide primitives used by the content track (join build/probe and grouping): exclusive
// scan and a stable LSD radix sort of (key, value) pairs. All are hand-written kernels.
#pragma once

#include "common.cuh"

namespace relnn {

// Exclusive prefix sum of in[0..n) into out[0..n) (in == out allowed; inputs non-negative). If
// total != nullptr the sum of all n inputs is written there (device). Temporary
// storage is stream-ordered (cudaMallocAsync) and released before return; the call is asynchronous.
// 32-bit inputs above one tile (4096 items) take a single pass whose blocks wait (bounded) on earlier
// tiles; a wait that runs out raises RELNN_DEV_TIMEOUT in `status` (device status word, may be null).
template <class T>
relnn_status exclusive_scan(const T* in, T* out, int64_t n, T* total, cudaStream_t st, int* status = nullptr);

// Stable LSD radix sort of n (key, value) pairs by the low `nbits` bits of the key (K = uint32_t or
// uint64_t, V = int32_t or int64_t). keys_tmp/vals_tmp are scratch of n entries each. With
// result_in_tmp == nullptr the result is left in keys/vals; otherwise *result_in_tmp tells which
// pair of buffers holds it (an odd number of passes ends in the scratch pair).
template <class K, class V>
relnn_status radix_sort_pairs(K* keys, V* vals, K* keys_tmp, V* vals_tmp, int64_t n, int nbits, cudaStream_t st,
                              bool* result_in_tmp = nullptr);

// Number of significant bits of v (0 for v == 0).
inline int bit_length(uint64_t v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

}  // namespace relnn
