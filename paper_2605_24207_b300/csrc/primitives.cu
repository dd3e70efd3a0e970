// Exclusive scan and stable LSD radix sort (hand-written; no CUB).
//
// Scan: reduce-then-scan. A block owns 4096 consecutive items (512 threads x 8 items in blocked
// order); the block sums are scanned recursively and added back.
//
// Radix sort: the key bits are split into passes of equal width of at most RELNN_TUNE_SORT_BITS
// bits (default 8: a 20-bit key takes three passes of 7, so each digit of a 4096-key tile leaves as
// a run of about 32 keys). Each block owns a tile of 4096 keys split into 8 warp sub-tiles of 512
// keys that a warp visits in 16 steps of 32. Pass = (1) per-block digit histogram with
// shared-memory atomics, (2) exclusive scan of the digit-major histogram, (3) stable scatter: a
// key's destination is digit base + (keys of its digit in earlier blocks) + (in earlier warps of
// its block) + (in earlier steps of its warp) + (in lower lanes of its step), the lanes of equal
// digit found with one ballot per digit bit; the block reorders its tile by digit in shared memory
// first, so each digit's keys are stored as one contiguous run.
#include "primitives.cuh"

#include <algorithm>

namespace relnn {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

template <class T>
__global__ void scan_reduce_kernel(const T* __restrict__ in, int64_t n, T* __restrict__ sums) {
    __shared__ T ws[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T s = 0;
    for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
        int64_t i = base + j;
        if (i < n) s += in[i];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        T v = threadIdx.x < kScanThreads / 32 ? ws[threadIdx.x] : T(0);
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

// Block-local exclusive scan of a 4096-item tile plus an optional per-block offset.
template <class T>
__global__ void scan_apply_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t n,
                                  const T* __restrict__ block_off, T* __restrict__ total) {
    __shared__ T ws[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : T(0);
        T t = v[k];
        v[k] = run;
        run += t;
    }
    T incl = warp_incl_scan(run);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kScanThreads / 32 ? ws[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) ws[lane] = wi - w;
    }
    __syncthreads();
    T off = ws[warp] + incl - run + (block_off ? block_off[blockIdx.x] : T(0));
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = v[k] + off;
    }
    if (total && threadIdx.x == kScanThreads - 1 && blockIdx.x == gridDim.x - 1) {
        *total = off + run;  // the last thread's exclusive offset plus its own items
    }
}

// Single-pass form (inputs above one tile): each block takes the next tile from a counter (so every
// earlier tile has started), scans it, publishes its sum, looks back over the published states of
// the earlier tiles 32 at a time (a tile that has its inclusive prefix ends the walk) and publishes
// its own inclusive prefix. State word of a tile: flag in the top two bits (1: sum only, 2:
// inclusive prefix), value in the low 62 (32-bit non-negative counts). Waits are bounded: after
// the wait budget the block gives up, raises RELNN_DEV_TIMEOUT in `status` (if given) and uses what
// it has. One launch instead of reduce, scan of the block sums and apply.
constexpr unsigned long long kScanAgg = 1ull << 62, kScanInc = 2ull << 62, kScanVal = (1ull << 62) - 1;

template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_lb_kernel(const T* in, T* out, int64_t n, T* total,
                                                           unsigned long long* words, int* status) {
    __shared__ T ws[kScanThreads / 32];
    __shared__ int tile_s;
    __shared__ T excl_s;
    if (threadIdx.x == 0) tile_s = (int)atomicAdd(reinterpret_cast<unsigned*>(words), 1u);
    __syncthreads();
    const int tile = tile_s;
    unsigned long long* state = words + 1;
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        const T t = i < n ? in[i] : T(0);
        v[k] = run;
        run += t;
    }
    const T incl = warp_incl_scan(run);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    T woff = 0, btot = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        woff += w < warp ? ws[w] : T(0);
        btot += ws[w];
    }
    if (warp == 0) {
        if (lane == 0)
            atomicExch(&state[tile], (tile == 0 ? kScanInc : kScanAgg) | ((unsigned long long)btot & kScanVal));
        long long excl = 0;
        int window = tile - 1;
        const unsigned long long t_start = globaltimer_ns();
        const unsigned long long budget = wait_budget_ns(status);
        unsigned spins = 0;
        while (window >= 0) {
            const int idx = window - lane;
            unsigned long long w = kScanInc;  // before tile 0: an inclusive zero
            if (idx >= 0) w = *reinterpret_cast<volatile unsigned long long*>(&state[idx]);
            const unsigned flag = (unsigned)(w >> 62);
            if (__any_sync(0xffffffffu, flag == 0)) {  // an earlier tile has not published yet
                if ((++spins & 63u) == 0 && globaltimer_ns() - t_start > budget) {
                    if (lane == 0) raise_status(status, RELNN_DEV_TIMEOUT);
                    break;
                }
                continue;
            }
            const unsigned inc_mask = __ballot_sync(0xffffffffu, flag == 2);
            const int stop = inc_mask ? __ffs(inc_mask) - 1 : 31;  // lanes 0..stop contribute
            long long x = lane <= stop ? (long long)(w & kScanVal) : 0;
#pragma unroll
            for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            excl += x;
            if (inc_mask) break;
            window -= 32;
        }
        if (lane == 0) {
            if (tile > 0) atomicExch(&state[tile], kScanInc | ((unsigned long long)(excl + (long long)btot) & kScanVal));
            excl_s = (T)excl;
        }
    }
    __syncthreads();
    const T off = excl_s + woff + incl - run;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = v[k] + off;
    }
    // the last tile's last thread: its exclusive offset plus its own items is the sum of all n
    if (total && tile == (int)gridDim.x - 1 && threadIdx.x == kScanThreads - 1) *total = off + run;
}

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortSteps = 16;
constexpr int kSortTile = kSortThreads * kSortSteps;  // 4096
constexpr int kMaxDigitBits = 11;

// Per-block digit counts of one pass (digit = (key >> shift) & mask, bins = mask + 1), stored
// digit-major: hist[d * nblocks + block]. Shared-memory atomics per key (with 2^11 bins the lanes of
// a warp rarely share a digit).
template <class K>
__global__ void rs_hist_kernel(const K* __restrict__ keys, int64_t n, int shift, unsigned mask,
                               int32_t* __restrict__ hist, int nblocks) {
    extern __shared__ int32_t h[];
    const int bins = (int)mask + 1;
    for (int i = threadIdx.x; i < bins; i += kSortThreads) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (32 * kSortSteps);
    // all of the thread's keys are loaded before the first atomic (one memory round trip, not 16)
    K k[kSortSteps];
#pragma unroll
    for (int s = 0; s < kSortSteps; ++s) {
        const int64_t i = base + s * 32 + lane;
        k[s] = i < n ? __ldg(keys + i) : K(0);
    }
#pragma unroll
    for (int s = 0; s < kSortSteps; ++s)
        if (base + s * 32 + lane < n) atomicAdd(&h[(unsigned)((k[s] >> shift) & mask)], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < bins; i += kSortThreads) hist[(int64_t)i * nblocks + blockIdx.x] = h[i];
}

// Exclusive scan of v[0..count) in place by one block of kSortThreads threads (count <= 8 x 256).
__device__ void block_excl_scan_small(int32_t* v, int count, int32_t* warp_tot) {
    const int per = (count + kSortThreads - 1) / kSortThreads;
    const int b0 = threadIdx.x * per;
    int32_t run = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < count) run += v[b0 + i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int32_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += warp_tot[w];
    int32_t off = woff + incl - run;
    for (int i = 0; i < per; ++i)
        if (b0 + i < count) {
            const int32_t t = v[b0 + i];
            v[b0 + i] = off;
            off += t;
        }
    __syncthreads();
}

// Stable scatter of one pass: a key's destination is its digit's base for this block (scanned
// histogram) + the keys of that digit in earlier warps of the block + in earlier steps of its warp
// + in lower lanes of its step (__match_any_sync / popc). The block first reorders its tile by
// digit in shared memory, so that each digit's keys leave as one contiguous run (coalesced stores).
template <class K, class V>
__global__ void __launch_bounds__(kSortThreads, 4) rs_scatter_kernel(const K* __restrict__ keys, const V* __restrict__ vals,
                                  K* __restrict__ okeys, V* __restrict__ ovals, int64_t n,
                                  int shift, unsigned mask, const int32_t* __restrict__ offs, int nblocks) {
    extern __shared__ __align__(16) int32_t sm[];
    const int bins = (int)mask + 1;
    int32_t* gbase = sm;                               // [bins]
    int32_t* wcnt = sm + bins;                         // [kSortWarps][bins]
    int32_t* dstart = wcnt + kSortWarps * bins;        // [bins] block-local start of each digit
    int32_t* wtot = dstart + bins;                     // [kSortWarps]
    K* tk = reinterpret_cast<K*>(sm + ((bins * (kSortWarps + 2) + kSortWarps + 3) & ~3));  // [kSortTile]
    V* tv = reinterpret_cast<V*>(tk + kSortTile);                                        // [kSortTile]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < bins; i += kSortThreads) {
        gbase[i] = offs[(int64_t)i * nblocks + blockIdx.x];
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) wcnt[w * bins + i] = 0;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (32 * kSortSteps);
    K k[kSortSteps];
    V v[kSortSteps];
    int32_t rank[kSortSteps];
#pragma unroll
    for (int s = 0; s < kSortSteps; ++s) {
        int64_t i = base + s * 32 + lane;
        bool valid = i < n;
        k[s] = valid ? keys[i] : K(0);
        v[s] = valid ? vals[i] : V(0);
    }
#pragma unroll
    for (int s = 0; s < kSortSteps; ++s) {
        int64_t i = base + s * 32 + lane;
        bool valid = i < n;
        unsigned d = valid ? (unsigned)((k[s] >> shift) & mask) : 0u;
        // lanes with this lane's digit: one ballot per digit bit (a loop kept rolled: the unrolled
        // 16 x 11 ballots stalled the kernel on instruction fetch; rolled, the plan's three scatter
        // passes over 16M pairs are 30 us faster)
        unsigned peers = __ballot_sync(0xffffffffu, valid);
        const int nbits_d = __popc(mask);
#pragma unroll 1
        for (int b = 0; b < nbits_d; ++b) {
            const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bb : ~bb;
        }
        const int old = valid ? wcnt[warp * bins + d] : 0;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp * bins + d] = old + __popc(peers);
        rank[s] = old + __popc(peers & lanemask_lt());
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < bins; i += kSortThreads) {
        int32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            int32_t t = wcnt[w * bins + i];
            wcnt[w * bins + i] = run;
            run += t;
        }
        dstart[i] = run;  // the block's count of digit i, scanned next
    }
    __syncthreads();
    block_excl_scan_small(dstart, bins, wtot);
#pragma unroll
    for (int s = 0; s < kSortSteps; ++s) {
        int64_t i = base + s * 32 + lane;
        if (i < n) {
            unsigned d = (unsigned)((k[s] >> shift) & mask);
            const int lp = dstart[d] + wcnt[warp * bins + d] + rank[s];
            tk[lp] = k[s];
            tv[lp] = v[s];
        }
    }
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
    const int cnt = (int)(n - t0 < kSortTile ? n - t0 : kSortTile);
    for (int i = threadIdx.x; i < cnt; i += kSortThreads) {
        const K key = tk[i];
        const unsigned d = (unsigned)((key >> shift) & mask);
        const int64_t pos = (int64_t)gbase[d] + (i - dstart[d]);
        okeys[pos] = key;
        ovals[pos] = tv[i];
    }
}

}  // namespace

template <class T>
relnn_status exclusive_scan(const T* in, T* out, int64_t n, T* total, cudaStream_t st, int* status) {
    if (n <= 0) {
        if (total) RELNN_CUDA(cudaMemsetAsync(total, 0, sizeof(T), st));
        return RELNN_OK;
    }
    const int64_t nb = ceil_div(n, kScanTile);
    if (nb == 1) {
        { scan_apply_kernel<T><<<1, kScanThreads, 0, st>>>(in, out, n, nullptr, total); note_launch(); }
        RELNN_CUDA(cudaGetLastError());
        return RELNN_OK;
    }
    if (sizeof(T) == 8) {
        // 64-bit inputs (packed (count, present) pairs can pass 2^62): reduce, scan the block sums, apply
        T* sums = nullptr;
        RELNN_CUDA(cudaMallocAsync(&sums, sizeof(T) * nb, st));
        { scan_reduce_kernel<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums); note_launch(); }
        relnn_status s = exclusive_scan<T>(sums, sums, nb, nullptr, st, status);
        if (s == RELNN_OK) {
            { scan_apply_kernel<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums, total); note_launch(); }
            if (cudaGetLastError() != cudaSuccess) s = RELNN_ECUDA;
        }
        cudaFreeAsync(sums, st);
        return s;
    }
    // single pass with a decoupled look-back: the tile counter and one state word per tile (32-bit
    // inputs: n < 2^31 counts below 2^31 sum below 2^62)
    unsigned long long* words = nullptr;
    RELNN_CUDA(cudaMallocAsync(&words, sizeof(unsigned long long) * (nb + 1), st));
    relnn_status s = RELNN_OK;
    if (cudaMemsetAsync(words, 0, sizeof(unsigned long long) * (nb + 1), st) != cudaSuccess) s = RELNN_ECUDA;
    if (s == RELNN_OK) {
        { scan_lb_kernel<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, total, words, status); note_launch(); }
        if (cudaGetLastError() != cudaSuccess) s = RELNN_ECUDA;
    }
    cudaFreeAsync(words, st);
    return s;
}

template relnn_status exclusive_scan<int32_t>(const int32_t*, int32_t*, int64_t, int32_t*, cudaStream_t, int*);
template relnn_status exclusive_scan<int64_t>(const int64_t*, int64_t*, int64_t, int64_t*, cudaStream_t, int*);

template <class K, class V>
relnn_status radix_sort_pairs(K* keys, V* vals, K* keys_tmp, V* vals_tmp, int64_t n, int nbits, cudaStream_t st,
                              bool* result_in_tmp) {
    if (result_in_tmp) *result_in_tmp = false;
    if (n <= 1 || nbits <= 0) return RELNN_OK;
    const int64_t nb64 = ceil_div(n, kSortTile);
    // passes of equal width, at most RELNN_TUNE_SORT_BITS (<= kMaxDigitBits) bits each
    const int max_bits = (int)std::min<int64_t>(kMaxDigitBits, std::max<int64_t>(4, tune_get(RELNN_TUNE_SORT_BITS)));
    const int passes = (nbits + max_bits - 1) / max_bits;
    const int bits = (nbits + passes - 1) / passes;
    const unsigned mask = (1u << bits) - 1u;
    const int bins = (int)mask + 1;
    RELNN_CHECK_ARG(nb64 * bins < (1ll << 31), "radix sort: too many keys");
    const int nb = (int)nb64;
    auto smem_of = [](int nbins) {
        return sizeof(int32_t) * (size_t)((nbins * (kSortWarps + 2) + kSortWarps + 3) & ~3) +
               (sizeof(K) + sizeof(V)) * (size_t)kSortTile;
    };
    const size_t scatter_smem = smem_of(bins);
    static bool attr_set = false;
    if (!attr_set) {
        RELNN_CUDA(cudaFuncSetAttribute(rs_scatter_kernel<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_of(1 << kMaxDigitBits)));
        attr_set = true;
    }
    int32_t* hist = nullptr;
    RELNN_CUDA(cudaMallocAsync(&hist, sizeof(int32_t) * (size_t)bins * nb, st));
    K *src_k = keys, *dst_k = keys_tmp;
    V *src_v = vals, *dst_v = vals_tmp;
    relnn_status s = RELNN_OK;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * bits;
        { rs_hist_kernel<K><<<nb, kSortThreads, sizeof(int32_t) * bins, st>>>(src_k, n, shift, mask, hist, nb); note_launch(); }
        s = exclusive_scan<int32_t>(hist, hist, (int64_t)bins * nb, nullptr, st);
        if (s != RELNN_OK) break;
        { rs_scatter_kernel<K, V><<<nb, kSortThreads, scatter_smem, st>>>(src_k, src_v, dst_k, dst_v, n, shift, mask, hist, nb); note_launch(); }
        if (cudaGetLastError() != cudaSuccess) {
            s = RELNN_ECUDA;
            break;
        }
        K* tk = src_k; src_k = dst_k; dst_k = tk;
        V* tv = src_v; src_v = dst_v; dst_v = tv;
    }
    if (s == RELNN_OK && (passes & 1)) {
        if (result_in_tmp) {
            *result_in_tmp = true;
        } else {
            cudaMemcpyAsync(keys, keys_tmp, sizeof(K) * n, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(vals, vals_tmp, sizeof(V) * n, cudaMemcpyDeviceToDevice, st);
        }
    }
    cudaFreeAsync(hist, st);
    if (s != RELNN_OK) set_error("radix sort failed");
    return s;
}

template relnn_status radix_sort_pairs<uint32_t, int32_t>(uint32_t*, int32_t*, uint32_t*, int32_t*, int64_t, int,
                                                          cudaStream_t, bool*);
template relnn_status radix_sort_pairs<uint64_t, int32_t>(uint64_t*, int32_t*, uint64_t*, int32_t*, int64_t, int,
                                                          cudaStream_t, bool*);
template relnn_status radix_sort_pairs<uint32_t, int64_t>(uint32_t*, int64_t*, uint32_t*, int64_t*, int64_t, int,
                                                          cudaStream_t, bool*);
template relnn_status radix_sort_pairs<uint64_t, int64_t>(uint64_t*, int64_t*, uint64_t*, int64_t*, int64_t, int,
                                                          cudaStream_t, bool*);

}  // namespace relnn
