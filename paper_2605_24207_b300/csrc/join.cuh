// Join build side (paper Sec. 2.2 "Join"; Sec. 4.2: the join produces row-index tensors).
//
// Layout in HBM for a build column of n keys with U distinct values:
//   rows_sorted[n]   int32  H rows in ascending key order (stable: ascending row within a key)
//   run_start[U+1]   int32  first position in rows_sorted of each distinct key
//   uid_of_pos[n]    int32  distinct-key index of each sorted position
//   ukeys[U]         int64  distinct keys, ascending
//   lookup           direct-address table int32[max-min+1] when the key range is small, else an
//                    open-addressing hash table (linear probing, load <= 1/2) of int64 keys and int32
//                    distinct-key indices.
//   slot_rows        with the direct table and unique keys (dense build): the H row of each slot
//                    (-1: no key), so a probe that needs the row takes one lookup instead of two.
#pragma once

#include "common.cuh"

namespace relnn {

constexpr int64_t kEmptyKey = 0x7fffffffffffffffll;  // reserved key value (INT64_MAX)

struct JoinView {
    int mode;                  // 0 = hash, 1 = direct
    int64_t key_min;           // direct mode: key of slot 0
    int64_t direct_size;       // direct mode: table entries
    uint64_t mask;             // hash mode: capacity - 1
    const int64_t* slot_keys;  // hash mode
    const int32_t* slot_vals;  // distinct-key index per slot (-1 = empty)
    const int32_t* slot_rows;  // direct mode, unique keys: H row per slot, -1 if none (else null)
    const int32_t* rows_sorted;
    const int32_t* run_start;
    const int32_t* uid_of_pos;

    // Distinct-key index of `key`, or -1 if the key is not on the build side.
    __device__ __forceinline__ int32_t lookup(int64_t key) const {
        if (mode == 1) {
            uint64_t off = (uint64_t)key - (uint64_t)key_min;
            return off < (uint64_t)direct_size ? slot_vals[off] : -1;
        }
        uint64_t h = mix64((uint64_t)key) & mask;
        for (uint64_t it = 0; it <= mask; ++it) {
            int64_t k = slot_keys[h];
            if (k == key) return slot_vals[h];
            if (k == kEmptyKey) return -1;
            h = (h + 1) & mask;
        }
        return -1;
    }
};

struct JoinTable {
    int kt = RELNN_I32;
    int64_t n = 0;
    int64_t n_unique = 0;
    int mode = 0;
    int64_t key_min = 0, key_max = 0, direct_size = 0;
    uint64_t cap = 0;
    DevBuf rows_sorted, run_start, uid_of_pos, ukeys, slot_keys, slot_vals, slot_rows, status;

    JoinView view() const {
        JoinView v;
        v.mode = mode;
        v.key_min = key_min;
        v.direct_size = direct_size;
        v.mask = cap ? cap - 1 : 0;
        v.slot_keys = slot_keys.as<int64_t>();
        v.slot_vals = slot_vals.as<int32_t>();
        v.slot_rows = slot_rows.as<int32_t>();
        v.rows_sorted = rows_sorted.as<int32_t>();
        v.run_start = run_start.as<int32_t>();
        v.uid_of_pos = uid_of_pos.as<int32_t>();
        return v;
    }
};

// Builds `jt` over keys[0..n) (device, key type kt). Synchronises `st` (reading sizes back); with
// sync_end = false the last kernels of the dense build are left in flight on `st` (the caller's
// later work on `st` is ordered after them).
relnn_status join_table_build(JoinTable& jt, const void* keys, int64_t n, int kt, cudaStream_t st,
                              bool sync_end = true);

// Min and max of a key column (device -> host, synchronises `st`). Returns false if n == 0.
relnn_status key_range(const void* keys, int64_t n, int kt, int64_t* kmin, int64_t* kmax,
                       cudaStream_t st);

}  // namespace relnn

struct relnn_join_s {
    relnn::JoinTable t;
};
