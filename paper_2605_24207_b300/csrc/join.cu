// Join build (sort + distinct runs + lookup table) and the standalone probe entry point.
#include "join.cuh"
#include "primitives.cuh"

#include <algorithm>
#include <vector>

namespace relnn {

namespace {

__global__ void key_minmax_kernel(const void* keys, int64_t n, int kt, unsigned long long* mm) {
    __shared__ unsigned long long wl[8], wh[8];
    unsigned long long lo = ~0ull, hi = 0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long o = ordered64(load_key(keys, kt, i));
        lo = o < lo ? o : lo;
        hi = o > hi ? o : hi;
    }
#pragma unroll
    for (int s = 16; s; s >>= 1) {
        unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, s);
        unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, s);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    // one pair of atomics per block (per-warp atomics on two words serialise)
    if ((threadIdx.x & 31) == 0) {
        wl[threadIdx.x >> 5] = lo;
        wh[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = wl[w] < lo ? wl[w] : lo;
            hi = wh[w] > hi ? wh[w] : hi;
        }
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
}

// Sort keys: ordered(key) - ordered(min), as 32- or 64-bit unsigned; values = row numbers.
template <class K>
__global__ void make_sort_keys_kernel(const void* keys, int64_t n, int kt, uint64_t omin, K* sk,
                                      int32_t* rows) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        sk[i] = (K)(ordered64(load_key(keys, kt, i)) - omin);
        rows[i] = (int32_t)i;
    }
}

template <class K>
__global__ void run_flags_kernel(const K* sk, int64_t n, int32_t* flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || sk[i] != sk[i - 1]) ? 1 : 0;
}

// flags_excl = exclusive scan of run flags. Writes run_start, uid_of_pos and the distinct keys.
template <class K>
__global__ void runs_kernel(const K* sk, const int32_t* flags_excl, int64_t n, uint64_t omin,
                            int32_t* run_start, int32_t* uid_of_pos, int64_t* ukeys, int64_t U) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool head = (i == 0 || sk[i] != sk[i - 1]);
        int32_t u = flags_excl[i] + (head ? 0 : -1);
        uid_of_pos[i] = u;
        if (head) {
            run_start[u] = (int32_t)i;
            ukeys[u] = (int64_t)(((uint64_t)sk[i] + omin) ^ 0x8000000000000000ull);
        }
        if (i == 0) run_start[U] = (int32_t)n;
    }
}

__global__ void fill_i32_kernel(int32_t* p, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void fill_i64_kernel(int64_t* p, int64_t n, int64_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void direct_insert_kernel(const int64_t* ukeys, int64_t U, int64_t kmin, int32_t* table) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x)
        table[(uint64_t)ukeys[u] - (uint64_t)kmin] = (int32_t)u;
}

__global__ void hash_insert_kernel(const int64_t* ukeys, int64_t U, uint64_t mask,
                                   unsigned long long* slot_keys, int32_t* slot_vals, int* status) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long key = (unsigned long long)ukeys[u];
        uint64_t h = mix64(key) & mask;
        bool done = false;
        for (uint64_t it = 0; it <= mask; ++it) {
            unsigned long long prev = atomicCAS(&slot_keys[h], (unsigned long long)kEmptyKey, key);
            if (prev == (unsigned long long)kEmptyKey) {
                slot_vals[h] = (int32_t)u;
                done = true;
                break;
            }
            h = (h + 1) & mask;
        }
        if (!done) raise_status(status, RELNN_DEV_HASH_FULL);
    }
}

// ---- dense build: when the key span is small (at most 4n, or 2^20), a key's slot is key - key_min
// and the sort becomes a counting pass, one scan and a placement pass.
constexpr int kDenseRun = 64;  // longest run of equal keys the dense build orders itself

__global__ void dense_count_kernel(const void* keys, int64_t n, int kt, int64_t kmin, int32_t* cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[(uint64_t)load_key(keys, kt, i) - (uint64_t)kmin], 1);
}

// packed[s] = count | (count > 0) << 32, so that one exclusive scan gives each slot's first sorted
// position (low half) and distinct-key index (high half); *maxc = the largest count.
__global__ void dense_pack_kernel(const int32_t* cnt, int64_t S, int64_t* packed, int* maxc) {
    int m = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cnt[s];
        packed[s] = (int64_t)c | ((int64_t)(c > 0) << 32);
        m = c > m ? c : m;
    }
    m = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(maxc, m);
}

__global__ void dense_slots_kernel(const int32_t* cnt, const int64_t* excl, int64_t S, int64_t kmin, int64_t n,
                                   int64_t U, int32_t* slot_vals, int32_t* run_start, int64_t* ukeys,
                                   int32_t* slot_rows) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = excl[s];
        const int32_t u = (int32_t)(e >> 32);
        if (cnt[s] > 0) {
            slot_vals[s] = u;
            run_start[u] = (int32_t)(uint32_t)e;
            ukeys[u] = (int64_t)((uint64_t)kmin + (uint64_t)s);
        } else {
            slot_vals[s] = -1;
            if (slot_rows) slot_rows[s] = -1;  // (present slots get their row from the placement)
        }
        if (s == 0) run_start[U] = (int32_t)n;
    }
}

// Row i goes to its key's run (unique keys: the run's only position; else the next free one, in
// no particular order until dense_fix_kernel sorts the run).
__global__ void dense_place_kernel(const void* keys, int64_t n, int kt, int64_t kmin, const int64_t* excl,
                                   int32_t* cursor, int32_t* rows_sorted, int32_t* uid_of_pos, int32_t* slot_rows) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t s = (uint64_t)load_key(keys, kt, i) - (uint64_t)kmin;
        const int64_t e = excl[s];
        const int32_t pos = (int32_t)(uint32_t)e + (cursor ? atomicAdd(&cursor[s], 1) : 0);
        rows_sorted[pos] = (int32_t)i;
        uid_of_pos[pos] = (int32_t)(e >> 32);
        if (slot_rows) slot_rows[s] = (int32_t)i;  // unique keys only (one row per slot)
    }
}

// Runs of equal keys in ascending row order (insertion sort; runs are at most kDenseRun long).
__global__ void dense_fix_kernel(const int32_t* run_start, int64_t U, int32_t* rows_sorted) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = run_start[u], e = run_start[u + 1];
        for (int32_t i = b + 1; i < e; ++i) {
            const int32_t v = rows_sorted[i];
            int32_t j = i - 1;
            while (j >= b && rows_sorted[j] > v) {
                rows_sorted[j + 1] = rows_sorted[j];
                --j;
            }
            rows_sorted[j + 1] = v;
        }
    }
}

// Standalone probe, pass 1: distinct-key index and match count per probe row; per-warp totals.
__global__ void probe_count_kernel(JoinView j, const void* keys, int64_t m, int kt, int32_t* uarr,
                                   int64_t* warp_tot) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t cnt = 0;
    if (i < m) {
        int32_t u = j.lookup(load_key(keys, kt, i));
        uarr[i] = u;
        if (u >= 0) cnt = j.run_start[u + 1] - j.run_start[u];
    }
#pragma unroll
    for (int s = 16; s; s >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, s);
    if ((threadIdx.x & 31) == 0 && (i >> 5) * 32 < m) warp_tot[i >> 5] = cnt;
}

// Pass 2: each warp writes its pairs at its scanned offset; lanes find their slot with a ballot
// (all counts <= 1, the unique-key case) or a shuffle scan (multi-match).
__global__ void probe_emit_kernel(JoinView j, const int32_t* uarr, int64_t m, const int64_t* warp_off,
                                  int32_t* probe_idx, int32_t* build_idx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int32_t u = -1;
    int64_t cnt = 0;
    if (i < m) {
        u = uarr[i];
        if (u >= 0) cnt = j.run_start[u + 1] - j.run_start[u];
    }
    int64_t pre;
    if (__all_sync(0xffffffffu, cnt <= 1)) {
        pre = __popc(__ballot_sync(0xffffffffu, cnt != 0) & lanemask_lt());
    } else {
        int64_t v = cnt;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, v, s);
            if (lane >= s) v += t;
        }
        pre = v - cnt;
    }
    if (cnt == 0) return;
    const int64_t base = warp_off[i >> 5] + pre;
    const int32_t rs = j.run_start[u];
    for (int64_t k = 0; k < cnt; ++k) {
        probe_idx[base + k] = (int32_t)i;
        build_idx[base + k] = j.rows_sorted[rs + k];
    }
}

inline int grid_for(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 16));
}

}  // namespace

relnn_status key_range(const void* keys, int64_t n, int kt, int64_t* kmin, int64_t* kmax,
                       cudaStream_t st) {
    *kmin = *kmax = 0;
    if (n <= 0) return RELNN_OK;
    unsigned long long* mm = nullptr;
    RELNN_CUDA(cudaMallocAsync(&mm, 16, st));
    unsigned long long init[2] = {~0ull, 0ull};
    cudaMemcpyAsync(mm, init, 16, cudaMemcpyHostToDevice, st);
    { key_minmax_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256 * 8), num_sms() * 4)), 256, 0, st>>>(keys, n, kt, mm); note_launch(); }
    unsigned long long h[2];
    cudaMemcpyAsync(h, mm, 16, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(mm, st);
    RELNN_CUDA(cudaStreamSynchronize(st));
    *kmin = (int64_t)(h[0] ^ 0x8000000000000000ull);
    *kmax = (int64_t)(h[1] ^ 0x8000000000000000ull);
    return RELNN_OK;
}

namespace {

// The dense build over S = span + 1 slots; *done = false (nothing changed) when a key repeats more
// than kDenseRun times, which the sort path handles.
relnn_status dense_build(JoinTable& jt, const void* keys, int64_t n, int kt, int64_t kmin, int64_t S, bool* done,
                         bool sync_end, cudaStream_t st) {
    *done = false;
    DevBuf cnt, packed;
    RELNN_TRY(cnt.alloc_tmp(sizeof(int32_t) * (S + 1), st));
    RELNN_TRY(packed.alloc_tmp(sizeof(int64_t) * (S + 1), st));
    int32_t* maxc = cnt.as<int32_t>() + S;
    RELNN_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (S + 1), st));
    const int gn = grid_for(n), gs = grid_for(S);
    { dense_count_kernel<<<gn, 256, 0, st>>>(keys, n, kt, kmin, cnt.as<int32_t>()); note_launch(); }
    { dense_pack_kernel<<<gs, 256, 0, st>>>(cnt.as<int32_t>(), S, packed.as<int64_t>(), maxc); note_launch(); }
    RELNN_TRY(exclusive_scan<int64_t>(packed.as<int64_t>(), packed.as<int64_t>(), S, packed.as<int64_t>() + S, st));
    int64_t total = 0;
    int32_t mc = 0;
    RELNN_CUDA(cudaMemcpyAsync(&total, packed.as<int64_t>() + S, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaMemcpyAsync(&mc, maxc, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaStreamSynchronize(st));
    if (mc > kDenseRun) return RELNN_OK;
    const int64_t U = total >> 32;
    jt.n_unique = U;
    jt.mode = 1;
    jt.direct_size = S;
    jt.cap = 0;
    RELNN_TRY(jt.run_start.alloc_nosync(sizeof(int32_t) * (U + 1), st));
    RELNN_TRY(jt.ukeys.alloc_nosync(sizeof(int64_t) * std::max<int64_t>(U, 1), st));
    RELNN_TRY(jt.slot_vals.alloc_nosync(sizeof(int32_t) * S, st));
    const bool dup = U < n;
    if (!dup) RELNN_TRY(jt.slot_rows.alloc_nosync(sizeof(int32_t) * S, st));  // -1 for an empty slot
    { dense_slots_kernel<<<gs, 256, 0, st>>>(cnt.as<int32_t>(), packed.as<int64_t>(), S, kmin, n, U,
                                             jt.slot_vals.as<int32_t>(), jt.run_start.as<int32_t>(),
                                             jt.ukeys.as<int64_t>(), dup ? nullptr : jt.slot_rows.as<int32_t>()); note_launch(); }
    if (dup) RELNN_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * S, st));
    { dense_place_kernel<<<gn, 256, 0, st>>>(keys, n, kt, kmin, packed.as<int64_t>(), dup ? cnt.as<int32_t>() : nullptr,
                                             jt.rows_sorted.as<int32_t>(), jt.uid_of_pos.as<int32_t>(),
                                             dup ? nullptr : jt.slot_rows.as<int32_t>()); note_launch(); }
    if (dup) { dense_fix_kernel<<<grid_for(U), 256, 0, st>>>(jt.run_start.as<int32_t>(), U, jt.rows_sorted.as<int32_t>()); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    if (sync_end) RELNN_CUDA(cudaStreamSynchronize(st));
    *done = true;
    return RELNN_OK;
}

}  // namespace

relnn_status join_table_build(JoinTable& jt, const void* keys, int64_t n, int kt, cudaStream_t st, bool sync_end) {
    RELNN_CHECK_ARG(n >= 0 && n < (1ll << 31) - 1, "join build: n out of range");
    RELNN_CHECK_ARG(n == 0 || keys, "join build: null keys");
    jt.kt = kt;
    jt.n = n;
    jt.slot_rows.release();  // only a dense build over unique keys sets it
    RELNN_TRY(jt.status.alloc_nosync(sizeof(int) * kStatusInts, st));
    RELNN_CUDA(cudaMemsetAsync(jt.status.p, 0, sizeof(int) * kStatusInts, st));
    RELNN_TRY(jt.rows_sorted.alloc_nosync(sizeof(int32_t) * std::max<int64_t>(n, 1), st));
    RELNN_TRY(jt.uid_of_pos.alloc_nosync(sizeof(int32_t) * std::max<int64_t>(n, 1), st));
    if (n == 0) {
        jt.n_unique = 0;
        RELNN_TRY(jt.run_start.alloc_nosync(sizeof(int32_t), st));
        RELNN_CUDA(cudaMemsetAsync(jt.run_start.p, 0, sizeof(int32_t), st));
        RELNN_TRY(jt.ukeys.alloc_nosync(sizeof(int64_t), st));
        jt.mode = 1;
        jt.direct_size = 0;
        RELNN_TRY(jt.slot_vals.alloc_nosync(sizeof(int32_t), st));
        RELNN_CUDA(cudaStreamSynchronize(st));
        return RELNN_OK;
    }
    int64_t kmin, kmax;
    RELNN_TRY(key_range(keys, n, kt, &kmin, &kmax, st));
    RELNN_CHECK_ARG(kmax != kEmptyKey, "join build: key INT64_MAX is reserved");
    jt.key_min = kmin;
    jt.key_max = kmax;
    const uint64_t omin = (uint64_t)kmin ^ 0x8000000000000000ull;
    const uint64_t span = ((uint64_t)kmax ^ 0x8000000000000000ull) - omin;
    if (span < (uint64_t)std::max<int64_t>(4 * n, 1 << 20)) {
        bool done = false;
        RELNN_TRY(dense_build(jt, keys, n, kt, kmin, (int64_t)span + 1, &done, sync_end, st));
        if (done) return RELNN_OK;
    }
    const int nbits = bit_length(span);
    const bool narrow = nbits <= 32;
    const size_t kb = narrow ? 4 : 8;
    DevBuf sk, sk_tmp, rows_tmp, flags;
    RELNN_TRY(sk.alloc_tmp(kb * n, st));
    RELNN_TRY(sk_tmp.alloc_tmp(kb * n, st));
    RELNN_TRY(rows_tmp.alloc_tmp(sizeof(int32_t) * n, st));
    RELNN_TRY(flags.alloc_tmp(sizeof(int32_t) * (n + 1), st));
    int32_t* rows = jt.rows_sorted.as<int32_t>();
    const int g = grid_for(n);
    if (narrow) {
        { make_sort_keys_kernel<uint32_t><<<g, 256, 0, st>>>(keys, n, kt, omin, sk.as<uint32_t>(), rows); note_launch(); }
        RELNN_TRY((radix_sort_pairs<uint32_t, int32_t>(sk.as<uint32_t>(), rows, sk_tmp.as<uint32_t>(),
                                                       rows_tmp.as<int32_t>(), n, nbits, st)));
        { run_flags_kernel<uint32_t><<<g, 256, 0, st>>>(sk.as<uint32_t>(), n, flags.as<int32_t>()); note_launch(); }
    } else {
        { make_sort_keys_kernel<uint64_t><<<g, 256, 0, st>>>(keys, n, kt, omin, sk.as<uint64_t>(), rows); note_launch(); }
        RELNN_TRY((radix_sort_pairs<uint64_t, int32_t>(sk.as<uint64_t>(), rows, sk_tmp.as<uint64_t>(),
                                                       rows_tmp.as<int32_t>(), n, nbits, st)));
        { run_flags_kernel<uint64_t><<<g, 256, 0, st>>>(sk.as<uint64_t>(), n, flags.as<int32_t>()); note_launch(); }
    }
    RELNN_TRY(exclusive_scan<int32_t>(flags.as<int32_t>(), flags.as<int32_t>(), n,
                                      flags.as<int32_t>() + n, st));
    int32_t U32 = 0;
    RELNN_CUDA(cudaMemcpyAsync(&U32, flags.as<int32_t>() + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaStreamSynchronize(st));
    const int64_t U = U32;
    jt.n_unique = U;
    RELNN_TRY(jt.run_start.alloc_nosync(sizeof(int32_t) * (U + 1), st));
    RELNN_TRY(jt.ukeys.alloc_nosync(sizeof(int64_t) * std::max<int64_t>(U, 1), st));
    if (narrow)
        { runs_kernel<uint32_t><<<g, 256, 0, st>>>(sk.as<uint32_t>(), flags.as<int32_t>(), n, omin,
                                                 jt.run_start.as<int32_t>(), jt.uid_of_pos.as<int32_t>(),
                                                 jt.ukeys.as<int64_t>(), U); note_launch(); }
    else
        { runs_kernel<uint64_t><<<g, 256, 0, st>>>(sk.as<uint64_t>(), flags.as<int32_t>(), n, omin,
                                                 jt.run_start.as<int32_t>(), jt.uid_of_pos.as<int32_t>(),
                                                 jt.ukeys.as<int64_t>(), U); note_launch(); }
    // Lookup: direct addressing when the key span is at most 4x the distinct keys (+1M slack).
    const uint64_t direct_limit = (uint64_t)std::max<int64_t>(4 * U, 1 << 20);
    if (span < direct_limit) {
        jt.mode = 1;
        jt.direct_size = (int64_t)span + 1;
        jt.cap = 0;
        RELNN_TRY(jt.slot_vals.alloc_nosync(sizeof(int32_t) * jt.direct_size, st));
        { fill_i32_kernel<<<grid_for(jt.direct_size), 256, 0, st>>>(jt.slot_vals.as<int32_t>(), jt.direct_size, -1); note_launch(); }
        { direct_insert_kernel<<<grid_for(U), 256, 0, st>>>(jt.ukeys.as<int64_t>(), U, kmin,
                                                          jt.slot_vals.as<int32_t>()); note_launch(); }
    } else {
        jt.mode = 0;
        uint64_t cap = 1024;
        while (cap < (uint64_t)(2 * U)) cap <<= 1;
        jt.cap = cap;
        RELNN_TRY(jt.slot_keys.alloc_nosync(sizeof(int64_t) * cap, st));
        RELNN_TRY(jt.slot_vals.alloc_nosync(sizeof(int32_t) * cap, st));
        { fill_i64_kernel<<<grid_for(cap), 256, 0, st>>>(jt.slot_keys.as<int64_t>(), cap, kEmptyKey); note_launch(); }
        { fill_i32_kernel<<<grid_for(cap), 256, 0, st>>>(jt.slot_vals.as<int32_t>(), cap, -1); note_launch(); }
        { hash_insert_kernel<<<grid_for(U), 256, 0, st>>>(jt.ukeys.as<int64_t>(), U, cap - 1,
                                                        jt.slot_keys.as<unsigned long long>(),
                                                        jt.slot_vals.as<int32_t>(), jt.status.as<int>()); note_launch(); }
    }
    RELNN_CUDA(cudaGetLastError());
    int dev_status = 0;
    RELNN_CUDA(cudaMemcpyAsync(&dev_status, jt.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaStreamSynchronize(st));
    if (dev_status) {
        set_device_error(dev_status);
        set_error("join build: device check failed");
        return RELNN_EDEVICE;
    }
    return RELNN_OK;
}

relnn_status join_probe_pairs(const JoinTable& jt, const void* probe, int64_t m, int32_t* probe_idx,
                              int32_t* build_idx, int64_t capacity, int64_t* d_count, cudaStream_t st) {
    if (m == 0) {
        if (d_count) RELNN_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int64_t), st));
        RELNN_CUDA(cudaStreamSynchronize(st));
        return RELNN_OK;
    }
    const int64_t nwarps = ceil_div(m, 32);
    DevBuf uarr, wt;
    RELNN_TRY(uarr.alloc_tmp(sizeof(int32_t) * m, st));
    RELNN_TRY(wt.alloc_tmp(sizeof(int64_t) * (nwarps + 1), st));
    const JoinView v = jt.view();
    const int blocks = (int)ceil_div(m, 256);
    { probe_count_kernel<<<blocks, 256, 0, st>>>(v, probe, m, jt.kt, uarr.as<int32_t>(), wt.as<int64_t>()); note_launch(); }
    RELNN_TRY(exclusive_scan<int64_t>(wt.as<int64_t>(), wt.as<int64_t>(), nwarps, wt.as<int64_t>() + nwarps, st));
    int64_t total = 0;
    RELNN_CUDA(cudaMemcpyAsync(&total, wt.as<int64_t>() + nwarps, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaStreamSynchronize(st));
    if (d_count) RELNN_CUDA(cudaMemcpyAsync(d_count, &total, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (total > capacity) {
        RELNN_CUDA(cudaStreamSynchronize(st));
        set_error("join probe: " + std::to_string(total) + " pairs exceed capacity " + std::to_string(capacity));
        return RELNN_ENOSPC;
    }
    { probe_emit_kernel<<<blocks, 256, 0, st>>>(v, uarr.as<int32_t>(), m, wt.as<int64_t>(), probe_idx, build_idx); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    RELNN_CUDA(cudaStreamSynchronize(st));
    return RELNN_OK;
}

}  // namespace relnn
