// Device-wide primitives used by the content track (join build/probe and grouping): exclusive
// scan and a stable LSD radix sort of (key, int32 value) pairs. All are hand-written kernels.
#pragma once

#include "common.cuh"

namespace relnn {

// Exclusive prefix sum of in[0..n) into out[0..n) (in == out allowed). If total != nullptr the
// sum of all n inputs is written there (device). Temporary storage is stream-ordered
// (cudaMallocAsync) and released before return; the call is asynchronous.
template <class T>
relnn_status exclusive_scan(const T* in, T* out, int64_t n, T* total, cudaStream_t st);

// Stable LSD radix sort of n (key, value) pairs by the low `nbits` bits of the key.
// keys/vals are sorted in place; keys_tmp/vals_tmp are scratch of n entries each.
template <class K>
relnn_status radix_sort_pairs(K* keys, int32_t* vals, K* keys_tmp, int32_t* vals_tmp, int64_t n,
                              int nbits, cudaStream_t st);

// out[i] = i for i < n.
relnn_status iota_i32(int32_t* out, int64_t n, cudaStream_t st);

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
