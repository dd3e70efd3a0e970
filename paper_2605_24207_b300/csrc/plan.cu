// Content track of a rule (join build, probe of src and dst, grouping by output key).
// Follows the join rule of Sec. 3.1: E |><| H(src) |><| H(dst) under bag semantics, then the
// projected union over dst (Sec. 2.2) whose group index is built here once and cached.
#include "plan.cuh"
#include "primitives.cuh"

#include <algorithm>

namespace relnn {

namespace {

// One thread per kIlp items, no grid-stride loop.
constexpr int kIlp = 4;
// Counting group-by: the largest group it orders itself (a larger one sends the plan to the radix
// sort) and the largest group one lane orders (larger ones: a block each).
constexpr int kGroupBig = 4096;
constexpr int kGroupLane = 32;
inline unsigned ilp_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, ceil_div(n, 256 * kIlp)); }

inline int grid_for(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 16));
}

// Conjunctive selection over a tuple's src and dst keys (relnn_filter), passed by value.
struct FilterSet {
    int n = 0;
    bool uses_dst = false;
    relnn_filter f[RELNN_MAX_FILTERS];
    __device__ __forceinline__ bool pass(int64_t s, int64_t d) const {
        bool ok = true;
#pragma unroll
        for (int i = 0; i < RELNN_MAX_FILTERS; ++i) {
            if (i >= n) break;
            const int64_t a = f[i].lhs == RELNN_TERM_SRC ? s : (f[i].lhs == RELNN_TERM_DST ? d : f[i].lhs_const);
            const int64_t b = f[i].rhs == RELNN_TERM_SRC ? s : (f[i].rhs == RELNN_TERM_DST ? d : f[i].rhs_const);
            switch (f[i].op) {
                case RELNN_CMP_EQ: ok = ok && a == b; break;
                case RELNN_CMP_NE: ok = ok && a != b; break;
                case RELNN_CMP_LT: ok = ok && a < b; break;
                case RELNN_CMP_LE: ok = ok && a <= b; break;
                case RELNN_CMP_GT: ok = ok && a > b; break;
                default: ok = ok && a >= b; break;
            }
        }
        return ok;
    }
};

// Pass 1 over E: distinct-key indices of src and dst, matches per tuple, per-warp totals. A tuple
// that fails the selection counts as unmatched.
__global__ void tri_count_kernel(JoinView j, const void* src, const void* dst, int64_t T, int kt,
                                 bool join_dst, FilterSet flt, int32_t* us, int32_t* ud, int64_t* warp_tot) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t m = 0;
    if (e < T) {
        const int64_t ks = load_key(src, kt, e);
        const int64_t kd = (join_dst || flt.uses_dst) ? load_key(dst, kt, e) : 0;
        int32_t a = flt.pass(ks, kd) ? j.lookup(ks) : -1;
        int32_t b = join_dst ? j.lookup(kd) : 0;
        us[e] = a;
        ud[e] = b;
        if (a >= 0 && b >= 0) {
            int64_t cs = j.run_start[a + 1] - j.run_start[a];
            int64_t cd = join_dst ? (int64_t)(j.run_start[b + 1] - j.run_start[b]) : 1;
            m = cs * cd;
        }
    }
#pragma unroll
    for (int s = 16; s; s >>= 1) m += __shfl_xor_sync(0xffffffffu, m, s);
    if ((threadIdx.x & 31) == 0 && e < T) warp_tot[e >> 5] = m;
}

// Pass 2 over E: emit the join-output tuples in (e, hs, hd) order as (group key, payload) pairs.
// The group key is the sorted position of the dst H row (rows of one key are contiguous there, so
// sorting by it groups by key, then by H row) or, without a dst join, the raw dst key. The payload
// is the src H row, or (src H row << 32 | E row) when the E row is needed later (r attributes).
// Lane offsets inside a warp come from a ballot when every tuple matches at most once (unique
// keys) and from a shuffle scan otherwise.
template <class K, class V>
__global__ void tri_emit_kernel(JoinView j, const void* dst, int64_t T, int kt, bool join_dst,
                                uint64_t omin, const int32_t* us, const int32_t* ud,
                                const int64_t* warp_off, K* t_key, V* t_val) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int32_t a = -1, b = -1;
    int64_t cs = 0, cd = 0;
    if (e < T) {
        a = us[e];
        b = ud[e];
        if (a >= 0 && b >= 0) {
            cs = j.run_start[a + 1] - j.run_start[a];
            cd = join_dst ? (int64_t)(j.run_start[b + 1] - j.run_start[b]) : 1;
        }
    }
    const int64_t cnt = cs * cd;
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
    int64_t pos = warp_off[e >> 5] + pre;
    const int32_t rs = j.run_start[a];
    const int32_t rd = join_dst ? j.run_start[b] : 0;
    K rawkey = 0;
    if (!join_dst) rawkey = (K)(ordered64(load_key(dst, kt, e)) - omin);
    for (int64_t x = 0; x < cs; ++x) {
        const int32_t hs = j.rows_sorted[rs + x];
        V val;
        if (sizeof(V) == 8) val = (V)(((uint64_t)(uint32_t)hs << 32) | (uint32_t)e);
        else val = (V)hs;
        for (int64_t y = 0; y < cd; ++y, ++pos) {
            t_key[pos] = join_dst ? (K)(rd + y) : rawkey;
            t_val[pos] = val;
        }
    }
}

// Unique H keys (every tuple matches at most once): pass 1 and 2 in one. A block takes the next tile
// of kEmitTile consecutive E rows (tile numbers are handed out in launch order), counts its matches,
// publishes the count, adds the counts of the tiles before it (a decoupled look-back that waits,
// bounded, for tiles still counting) and writes its pairs in E order: the same output as the
// two passes, without storing the per-tuple lookups.
constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 8;  // consecutive E rows per thread
constexpr int kEmitTile = kEmitThreads * kEmitItems;
constexpr unsigned long long kTileAgg = 1ull << 62, kTileInc = 2ull << 62, kTileVal = (1ull << 62) - 1;

template <class K, class V>
__global__ void __launch_bounds__(kEmitThreads) emit_unique_kernel(
    JoinView j, const void* src, const void* dst, int64_t T, int kt, bool join_dst, FilterSet flt, uint64_t omin,
    unsigned* tile_ctr, unsigned long long* tile_state, unsigned long long* total, int* status, K* t_key, V* t_val) {
    __shared__ int tile_s;
    __shared__ int warp_tot[kEmitThreads / 32];
    __shared__ long long base_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) tile_s = (int)atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int tile = tile_s;
    const int64_t e0 = (int64_t)tile * kEmitTile + (int64_t)threadIdx.x * kEmitItems;
    int64_t ks[kEmitItems], kd[kEmitItems];
#pragma unroll
    for (int i = 0; i < kEmitItems; ++i) {
        const int64_t e = e0 + i;
        ks[i] = e < T ? load_key(src, kt, e) : 0;
        kd[i] = (e < T && (join_dst || flt.uses_dst)) ? load_key(dst, kt, e) : 0;
    }
    int32_t a[kEmitItems], bb[kEmitItems];
    int cnt = 0;
    if (j.mode == 1) {  // direct addressing: independent table reads
#pragma unroll
        for (int i = 0; i < kEmitItems; ++i) {
            const uint64_t os = (uint64_t)ks[i] - (uint64_t)j.key_min, od = (uint64_t)kd[i] - (uint64_t)j.key_min;
            a[i] = os < (uint64_t)j.direct_size ? __ldg(j.slot_vals + os) : -1;
            bb[i] = !join_dst ? 0 : (od < (uint64_t)j.direct_size ? __ldg(j.slot_vals + od) : -1);
        }
    } else {
#pragma unroll
        for (int i = 0; i < kEmitItems; ++i) {
            a[i] = j.lookup(ks[i]);
            bb[i] = join_dst ? j.lookup(kd[i]) : 0;
        }
    }
#pragma unroll
    for (int i = 0; i < kEmitItems; ++i) {
        if (e0 + i >= T || (flt.n && !flt.pass(ks[i], kd[i]))) a[i] = -1;
        cnt += (a[i] >= 0 && bb[i] >= 0) ? 1 : 0;
    }
    // block-wide exclusive scan of the per-thread counts
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int woff = 0, btot = 0;
#pragma unroll
    for (int w = 0; w < kEmitThreads / 32; ++w) {
        woff += w < warp ? warp_tot[w] : 0;
        btot += warp_tot[w];
    }
    if (warp == 0) {
        // warp-wide look-back: 32 predecessors per step, nearest first (lane 0 = tile - 1)
        long long excl = 0;
        if (lane == 0) atomicExch(&tile_state[tile], (tile == 0 ? kTileInc : kTileAgg) | (unsigned long long)btot);
        int window = tile - 1;
        const unsigned long long t_start = globaltimer_ns();
        const unsigned long long budget = wait_budget_ns(status);
        unsigned spins = 0;
        while (window >= 0) {
            const int idx = window - lane;
            unsigned long long w = kTileInc | 0ull;  // before tile 0: an inclusive zero
            if (idx >= 0) w = *reinterpret_cast<volatile unsigned long long*>(&tile_state[idx]);
            const unsigned flag = (unsigned)(w >> 62);
            if (__any_sync(0xffffffffu, flag == 0)) {  // a predecessor is still counting
                if ((++spins & 63u) == 0 && globaltimer_ns() - t_start > budget) {
                    if (lane == 0) raise_status(status, RELNN_DEV_TIMEOUT);
                    break;
                }
                continue;
            }
            const unsigned inc_mask = __ballot_sync(0xffffffffu, flag == 2);
            const int stop = inc_mask ? __ffs(inc_mask) - 1 : 31;  // lanes 0..stop contribute
            long long v = lane <= stop ? (long long)(w & kTileVal) : 0;
#pragma unroll
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            excl += v;
            if (inc_mask) break;
            window -= 32;
        }
        if (lane == 0) {
            if (tile > 0) atomicExch(&tile_state[tile], kTileInc | (unsigned long long)(excl + btot));
            atomicAdd(total, (unsigned long long)btot);
            base_s = excl;
        }
    }
    // unique keys: a key's distinct index is its sorted position, so rd = run_start[b] = b and the
    // src H row is rows_sorted[a]. The tile's pairs are staged in shared memory in output order and
    // then stored by consecutive threads (the block's output range is contiguous).
    __shared__ K sk[kEmitTile];
    __shared__ V sv[kEmitTile];
    int32_t hsv[kEmitItems];
#pragma unroll
    for (int i = 0; i < kEmitItems; ++i) hsv[i] = (a[i] >= 0 && bb[i] >= 0) ? __ldg(j.rows_sorted + a[i]) : 0;
    int lp = woff + (incl - cnt);
#pragma unroll
    for (int i = 0; i < kEmitItems; ++i) {
        if (a[i] < 0 || bb[i] < 0) continue;
        const int64_t e = e0 + i;
        const int32_t hs = hsv[i];
        V val;
        if (sizeof(V) == 8) val = (V)(((uint64_t)(uint32_t)hs << 32) | (uint32_t)e);
        else val = (V)hs;
        sk[lp] = join_dst ? (K)bb[i] : (K)(ordered64(load_key(dst, kt, e)) - omin);
        sv[lp] = val;
        ++lp;
    }
    __syncthreads();
    const int64_t base = base_s;
    for (int i = threadIdx.x; i < btot; i += kEmitThreads) {
        t_key[base + i] = sk[i];
        t_val[base + i] = sv[i];
    }
}

// Unique H keys, no selection: if every tuple matches, tuple e's pair goes to position e. This pass
// assumes so (plain streaming, no look-back) and counts the tuples that do not match; when the count
// is not zero, the caller runs emit_unique_kernel over the same outputs.
// A tuple that matches nothing gets the group key `sentinel` (above every real key: it sorts to the
// end, behind the matched tuples, which keep their E order).
template <class K, class V>
__global__ void emit_all_kernel(JoinView j, const void* src, const void* dst, int64_t T, int kt, bool join_dst,
                                uint64_t omin, unsigned long long* misses, K* t_key, V* t_val, int32_t* cnt,
                                unsigned* big, K sentinel) {
    const int64_t e0 = (blockIdx.x * (int64_t)blockDim.x) * kIlp + threadIdx.x;
    int64_t ks[kIlp], kd[kIlp];
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
        const int64_t e = e0 + (int64_t)k * blockDim.x;
        ks[k] = e < T ? load_key(src, kt, e) : 0;
        kd[k] = e < T ? load_key(dst, kt, e) : 0;
    }
    int32_t a[kIlp], b[kIlp], hs[kIlp];
    if (j.slot_rows) {
        // direct table with unique keys: the src H row in one lookup (-1: no such key)
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const uint64_t os = (uint64_t)ks[k] - (uint64_t)j.key_min, od = (uint64_t)kd[k] - (uint64_t)j.key_min;
            hs[k] = os < (uint64_t)j.direct_size ? __ldg(j.slot_rows + os) : -1;
            a[k] = hs[k];
            b[k] = !join_dst ? 0 : (od < (uint64_t)j.direct_size ? __ldg(j.slot_vals + od) : -1);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            a[k] = j.lookup(ks[k]);
            b[k] = join_dst ? j.lookup(kd[k]) : 0;
        }
    }
    unsigned miss = 0;
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
        const bool in = e0 + (int64_t)k * blockDim.x < T;
        const bool ok = a[k] >= 0 && b[k] >= 0;
        miss += (in && !ok) ? 1u : 0u;
        if (!j.slot_rows) hs[k] = in && ok ? __ldg(j.rows_sorted + a[k]) : 0;
    }
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
        const int64_t e = e0 + (int64_t)k * blockDim.x;
        if (e < T) {
            const bool ok = a[k] >= 0 && b[k] >= 0;
            t_key[e] = !ok ? sentinel : join_dst ? (K)b[k] : (K)(ordered64(kd[k]) - omin);
            if (sizeof(V) == 8) t_val[e] = (V)(((uint64_t)(uint32_t)hs[k] << 32) | (uint32_t)e);
            else t_val[e] = (V)hs[k];
        }
    }
    miss = __reduce_add_sync(0xffffffffu, miss);
    if ((threadIdx.x & 31) == 0 && miss) atomicAdd(misses, (unsigned long long)miss);
    if (cnt) {
        // tuples per group key (the counting group-by); lanes holding the same key add once, and
        // a count passing kGroupBig is flagged (that group-by then takes the radix sort)
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const bool in = e0 + (int64_t)k * blockDim.x < T && a[k] >= 0 && b[k] >= 0;
            const int key = in ? (int)b[k] : -1;
            const unsigned mm = __match_any_sync(0xffffffffu, key);
            if (in && lane == __ffs(mm) - 1) {
                const int c = __popc(mm);
                if (atomicAdd(&cnt[key], c) + c > kGroupBig) atomicOr(big, 1u);
            }
        }
    }
}

// ---- counting group-by (one branch, unique H keys, E rows not carried): the emission counted the
// tuples per group key b; one exclusive scan of packed (count, present) pairs gives each group's first
// position and output row; an atomic scatter places every tuple's (hs, hd, seg) in its group; each
// group is then sorted by hs, which makes the order, and so every later sum, the same run to run
// (tuples with equal hs are equal rows, so their mutual order does not matter).
__global__ void group_pack_kernel(const int32_t* __restrict__ cnt, int64_t n, int64_t* __restrict__ packed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cnt[i];
        packed[i] = (int64_t)c | ((int64_t)(c > 0) << 32);
    }
}

// Per group key b: its scatter cursor (first position) and, if present, its output key.
__global__ void group_heads_kernel(const int32_t* __restrict__ cnt, const int64_t* __restrict__ excl, int64_t n,
                                   const int64_t* __restrict__ ukeys, int32_t* __restrict__ cur,
                                   int64_t* __restrict__ out_keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = excl[i];
        cur[i] = (int32_t)(uint32_t)e;
        if (cnt[i] > 0) out_keys[e >> 32] = ukeys[i];
    }
}

// Tuple i (E order) to the next free position of its group (lanes with the same key take one
// atomic and consecutive positions); writes its src H row there. (One scattered 4-byte store per
// tuple into one array that fits in L2; the group's dst H row and output row are written per group,
// contiguously, by the sort kernels.)
__global__ void group_scatter_kernel(const uint32_t* __restrict__ key, const int32_t* __restrict__ val, int64_t m,
                                     int32_t* __restrict__ cur, int32_t* __restrict__ hs) {
    const int lane = threadIdx.x & 31;
    const int64_t i0 = (blockIdx.x * (int64_t)blockDim.x) * kIlp + threadIdx.x;
    uint32_t k[kIlp];
    int32_t v[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        k[u] = i < m ? __ldg(key + i) : 0xffffffffu;
        v[u] = i < m ? __ldg(val + i) : 0;
    }
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
        const bool in = i0 + (int64_t)u * blockDim.x < m;
        const unsigned mm = __match_any_sync(0xffffffffu, k[u]);
        const int leader = __ffs(mm) - 1;
        int base = 0;
        if (in && lane == leader) base = atomicAdd(&cur[k[u]], __popc(mm));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (in) hs[base + __popc(mm & ((1u << lane) - 1u))] = v[u];
    }
}

// Groups of at most kGroupLane tuples: a warp takes 32 consecutive group keys, one per lane. When
// their tuples fit (at most 32 x 32), the warp's range of hs is loaded into shared memory with
// coalesced loads, each lane sorts its group's slice (insertion sort), and the range is stored back
// coalesced; otherwise each lane sorts its group in place. Each lane then writes its group's dst H
// row and output row over the group's positions. Larger groups are listed for
// group_sort_block_kernel (which writes their hd / seg as well).
__global__ void __launch_bounds__(256) group_sort_warp_kernel(const int32_t* __restrict__ cnt,
                                                              const int64_t* __restrict__ excl, int64_t n,
                                                              const int32_t* __restrict__ rows_sorted,
                                                              int32_t* __restrict__ hs, int32_t* __restrict__ hd,
                                                              int32_t* __restrict__ seg, int32_t* __restrict__ big_list,
                                                              int* __restrict__ n_big) {
    __shared__ int32_t sm[8][kGroupLane * 32];
    const int lane = threadIdx.x & 31;
    int32_t* buf = sm[threadIdx.x >> 5];
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w * 32 < n; w += nw) {
        const int64_t g = w * 32 + lane;
        const int c = g < n ? cnt[g] : 0;
        const int64_t e = g < n ? excl[g] : 0;
        const int64_t s = (int64_t)(uint32_t)e;
        const int32_t orow = (int32_t)(e >> 32);
        const bool big = c > kGroupLane;
        if (big) big_list[atomicAdd(n_big, 1)] = (int32_t)g;
        // the warp's range of positions: from the first present group's start to the last one's end
        const int64_t lo = __reduce_min_sync(0xffffffffu, c > 0 ? (unsigned)s : 0xffffffffu);
        const int64_t hi = __reduce_max_sync(0xffffffffu, c > 0 ? (unsigned)(s + c) : 0u);
        const bool staged = !__any_sync(0xffffffffu, big) && hi > lo && hi - lo <= kGroupLane * 32;
        if (staged) {
            const int len = (int)(hi - lo);
            for (int i = lane; i < len; i += 32) buf[i] = hs[lo + i];
            __syncwarp();
            int32_t* col = buf + (s - lo);
            for (int j = 1; j < c; ++j) {
                const int32_t x = col[j];
                int i = j - 1;
                while (i >= 0 && col[i] > x) {
                    col[i + 1] = col[i];
                    --i;
                }
                col[i + 1] = x;
            }
            __syncwarp();
            for (int i = lane; i < len; i += 32) hs[lo + i] = buf[i];
            __syncwarp();
        } else if (!big && c > 1) {
            int32_t* col = buf;  // lane-private column: element j at j * 32 + lane
            for (int j = 0; j < c; ++j) col[j * 32 + lane] = hs[s + j];
            for (int j = 1; j < c; ++j) {
                const int32_t x = col[j * 32 + lane];
                int i = j - 1;
                while (i >= 0 && col[i * 32 + lane] > x) {
                    col[(i + 1) * 32 + lane] = col[i * 32 + lane];
                    --i;
                }
                col[(i + 1) * 32 + lane] = x;
            }
            for (int j = 0; j < c; ++j) hs[s + j] = col[j * 32 + lane];
        }
        __syncwarp();
        if (!big && c > 0) {
            const int32_t r = rows_sorted[g];
            for (int j = 0; j < c; ++j) {
                hd[s + j] = r;
                seg[s + j] = orow;
            }
        }
    }
}

// Listed groups (kGroupLane < count <= kGroupBig), one block each at a time: bitonic sort in
// shared memory (padded with INT_MAX to a power of two).
__global__ void __launch_bounds__(256) group_sort_block_kernel(const int32_t* __restrict__ cnt,
                                                               const int64_t* __restrict__ excl,
                                                               const int32_t* __restrict__ big_list,
                                                               const int* __restrict__ n_big,
                                                               const int32_t* __restrict__ rows_sorted,
                                                               int32_t* __restrict__ hs, int32_t* __restrict__ hd,
                                                               int32_t* __restrict__ seg) {
    __shared__ int32_t sm[kGroupBig];
    const int nb = *n_big;
    for (int li = blockIdx.x; li < nb; li += gridDim.x) {
        const int32_t g = big_list[li];
        const int c = cnt[g];
        const int64_t s = (int64_t)(uint32_t)excl[g];
        int P = 1;
        while (P < c) P <<= 1;
        __syncthreads();
        for (int j = threadIdx.x; j < P; j += blockDim.x) sm[j] = j < c ? hs[s + j] : INT_MAX;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    const int l = i ^ jj;
                    if (l > i) {
                        const int32_t a = sm[i], b = sm[l];
                        const bool up = (i & k) == 0;
                        if ((a > b) == up) {
                            sm[i] = b;
                            sm[l] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        const int32_t r = rows_sorted[g], orow = (int32_t)(excl[g] >> 32);
        for (int j = threadIdx.x; j < c; j += blockDim.x) {
            hs[s + j] = sm[j];
            hd[s + j] = r;
            seg[s + j] = orow;
        }
    }
}

// Splits (src H row << 32 | E row) payloads into hs / er.
__global__ void split_pair_kernel(const int64_t* val, int64_t m, int32_t* hs, int32_t* er) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t v = (uint64_t)val[i];
        hs[i] = (int32_t)(v >> 32);
        er[i] = (int32_t)(uint32_t)v;
    }
}

// After grouping by dst position: the dst H row and the output row of every matched tuple. Each
// thread takes kIlp tuples with all of their loads issued before the first use (the lookups are
// dependent loads; one tuple at a time leaves the memory system idle).

__global__ void finalize_dst_kernel(const uint32_t* pos_d, int64_t m, const int32_t* rows_sorted,
                                    const int32_t* uid_of_pos, const int32_t* out_row, int32_t* hd, int32_t* seg,
                                    uint32_t limit) {
    const int64_t i0 = (blockIdx.x * (int64_t)blockDim.x) * kIlp + threadIdx.x;
    uint32_t p[kIlp];
    int32_t h[kIlp], u[kIlp];
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
        const int64_t i = i0 + (int64_t)k * blockDim.x;
        p[k] = i < m ? __ldg(pos_d + i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
        const bool ok = i0 + (int64_t)k * blockDim.x < m && p[k] < limit;
        h[k] = ok ? __ldg(rows_sorted + p[k]) : -1;
        u[k] = ok ? __ldg(uid_of_pos + p[k]) : -1;
    }
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
        const int64_t i = i0 + (int64_t)k * blockDim.x;
        if (i < m) {
            hd[i] = h[k];
            seg[i] = u[k] >= 0 ? __ldg(out_row + u[k]) : -1;  // -1: a tuple past the matched ones
        }
    }
}

__global__ void mark_present_kernel(const uint32_t* pos_d, int64_t m, const int32_t* uid_of_pos,
                                    int32_t* present, uint32_t limit) {
    const int64_t i0 = (blockIdx.x * (int64_t)blockDim.x) * kIlp + threadIdx.x;
    uint32_t p[kIlp];
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
        const int64_t i = i0 + (int64_t)k * blockDim.x;
        p[k] = i < m ? __ldg(pos_d + i) : 0u;
    }
    int32_t u[kIlp];
#pragma unroll
    for (int k = 0; k < kIlp; ++k)
        u[k] = i0 + (int64_t)k * blockDim.x < m && p[k] < limit ? __ldg(uid_of_pos + p[k]) : -1;
#pragma unroll
    for (int k = 0; k < kIlp; ++k)
        if (u[k] >= 0) present[u[k]] = 1;
}

// present / out_row: exclusive scan of the presence flags; writes the output keys.
__global__ void out_keys_kernel(const int32_t* present, const int32_t* out_row, const int64_t* ukeys,
                                int64_t U, int64_t* out_keys) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x)
        if (present[u]) out_keys[out_row[u]] = ukeys[u];
}

template <class K>
__global__ void key_flags_kernel(const K* key, int64_t m, int32_t* flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

template <class K>
__global__ void raw_seg_kernel(const K* key, const int32_t* flags_excl, int64_t m, uint64_t omin,
                               int32_t* seg, int64_t* out_keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool head = (i == 0 || key[i] != key[i - 1]);
        int32_t s = flags_excl[i] - (head ? 0 : 1);
        seg[i] = s;
        if (head) out_keys[s] = (int64_t)(((uint64_t)key[i] + omin) ^ 0x8000000000000000ull);
    }
}

// (src H row, position) pairs of the grouped tuples, to be sorted into src order.
__global__ void src_pairs_kernel(const int32_t* hs, int64_t m, uint32_t* key, int32_t* val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = (uint32_t)hs[i];
        val[i] = (int32_t)i;
    }
}

__global__ void gather_i32_kernel(const int32_t* src, const int32_t* idx, int64_t m, int32_t* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = src[idx[i]];
}

// Branch-local matched tuples while they are grouped: group keys (u32 dst position or u32/u64 raw
// key) and payloads (int32 src H row, or int64 src H row << 32 | E row).
struct Tmp {
    DevBuf key, key_tmp, val, val_tmp;
    bool wide = false;    // 64-bit raw keys
    bool pair = false;    // 64-bit payloads (the E row rides along)
    bool in_tmp = false;  // the sorted pairs are in key_tmp / val_tmp
    uint64_t omin = 0;
    // counting group-by: requested (eligible plan), taken (every tuple matched, no group above
    // kGroupBig); the counts per group key (+ the flag word) and the scanned (count, present) pairs,
    // whose total (matched tuples | output rows << 32) is read with the plan's final synchronisation
    bool want_count = false, counted = false;
    DevBuf cnt, gpacked;
    // unique H keys, no selection, a dst join: tuples that match nothing are emitted with the
    // sentinel key and sorted behind the matched ones; their count (in `miss`) is read with the plan's
    // final synchronisation, and the branch's m is an upper bound (every E row) until then
    bool defer = false;
    uint32_t sentinel = 0xffffffffu;
    DevBuf miss;
    template <class K>
    const K* keys() const { return in_tmp ? key_tmp.as<K>() : key.as<K>(); }
    DevBuf& sorted_val() { return in_tmp ? val_tmp : val; }
};

// The branch's selection predicates as a kernel argument.
FilterSet filters_of(const relnn_branch_desc& bd) {
    FilterSet fs;
    fs.n = bd.filters ? bd.n_filters : 0;
    for (int i = 0; i < fs.n; ++i) {
        fs.f[i] = bd.filters[i];
        fs.uses_dst = fs.uses_dst || fs.f[i].lhs == RELNN_TERM_DST || fs.f[i].rhs == RELNN_TERM_DST;
    }
    return fs;
}

// Emits the matched tuples as (group key, payload) pairs into t.key / t.val and returns their count
// in *M. Unique H keys: one pass (buffers sized for every E row); otherwise a counting pass first.
template <class K, class V>
relnn_status emit_pairs(Plan& p, const relnn_branch_desc& bd, Tmp& t, int64_t* M_out, cudaStream_t st) {
    const int64_t T = bd.n_tuples;
    const JoinView v = p.Ht().view();
    int64_t M = 0;
    if (p.Ht().n_unique == p.n_h) {
        const int64_t cap = std::max<int64_t>(T, 1);
        RELNN_TRY(t.key.alloc_tmp(sizeof(K) * cap, st));
        RELNN_TRY(t.key_tmp.alloc_tmp(sizeof(K) * cap, st));
        RELNN_TRY(t.val.alloc_tmp(sizeof(V) * cap, st));
        RELNN_TRY(t.val_tmp.alloc_tmp(sizeof(V) * cap, st));
        bool all_matched = false;
        if (T > 0 && t.defer) {
            RELNN_TRY(t.miss.alloc_tmp(sizeof(unsigned long long), st));
            RELNN_CUDA(cudaMemsetAsync(t.miss.p, 0, sizeof(unsigned long long), st));
            { emit_all_kernel<K, V><<<ilp_grid(T), 256, 0, st>>>(v, bd.d_src, bd.d_dst, T, p.kt, p.join_dst, t.omin,
                                                              t.miss.as<unsigned long long>(), t.key.as<K>(), t.val.as<V>(),
                                                              nullptr, nullptr, (K)t.sentinel); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
            *M_out = T;  // an upper bound; the misses are subtracted after the final synchronisation
            return RELNN_OK;
        }
        if (T > 0 && filters_of(bd).n == 0) {
            DevBuf miss;  // misses (u64) | the big-group flag (u32)
            RELNN_TRY(miss.alloc_tmp(2 * sizeof(unsigned long long), st));
            RELNN_CUDA(cudaMemsetAsync(miss.p, 0, 2 * sizeof(unsigned long long), st));
            unsigned* big = reinterpret_cast<unsigned*>(miss.as<unsigned long long>() + 1);
            if (t.want_count) {
                RELNN_TRY(t.cnt.alloc_tmp(sizeof(int32_t) * std::max<int64_t>(p.n_h, 1), st));
                RELNN_CUDA(cudaMemsetAsync(t.cnt.p, 0, sizeof(int32_t) * std::max<int64_t>(p.n_h, 1), st));
            }
            { emit_all_kernel<K, V><<<ilp_grid(T), 256, 0, st>>>(v, bd.d_src, bd.d_dst, T, p.kt, p.join_dst, t.omin,
                                                              miss.as<unsigned long long>(), t.key.as<K>(), t.val.as<V>(),
                                                              t.want_count ? t.cnt.as<int32_t>() : nullptr, big,
                                                              (K)t.sentinel); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
            unsigned long long mu[2] = {0, 0};
            RELNN_CUDA(cudaMemcpyAsync(mu, miss.p, sizeof(mu), cudaMemcpyDeviceToHost, st));
            RELNN_CUDA(cudaStreamSynchronize(st));
            all_matched = mu[0] == 0;
            if (all_matched) M = T;
            t.counted = t.want_count && all_matched && (unsigned)mu[1] == 0;
        }
        if (T > 0 && !all_matched) {
            const int64_t n_tiles = ceil_div(T, kEmitTile);
            DevBuf ctl;  // tile states, tile counter, total
            const size_t ctl_bytes = sizeof(unsigned long long) * (n_tiles + 2);
            RELNN_TRY(ctl.alloc_tmp(ctl_bytes, st));
            RELNN_CUDA(cudaMemsetAsync(ctl.p, 0, ctl_bytes, st));
            unsigned long long* st_words = ctl.as<unsigned long long>();
            { emit_unique_kernel<K, V><<<(unsigned)n_tiles, kEmitThreads, 0, st>>>(
                v, bd.d_src, bd.d_dst, T, p.kt, p.join_dst, filters_of(bd), t.omin, reinterpret_cast<unsigned*>(st_words + n_tiles),
                st_words, st_words + n_tiles + 1, p.status.as<int>(), t.key.as<K>(), t.val.as<V>()); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
            unsigned long long Mu = 0;
            RELNN_CUDA(cudaMemcpyAsync(&Mu, st_words + n_tiles + 1, sizeof(Mu), cudaMemcpyDeviceToHost, st));
            RELNN_CUDA(cudaStreamSynchronize(st));
            M = (int64_t)Mu;
        }
    } else {
        const int64_t nwarps = ceil_div(std::max<int64_t>(T, 1), 32);
        DevBuf us, ud, wt;
        RELNN_TRY(us.alloc_tmp(sizeof(int32_t) * std::max<int64_t>(T, 1), st));
        RELNN_TRY(ud.alloc_tmp(sizeof(int32_t) * std::max<int64_t>(T, 1), st));
        RELNN_TRY(wt.alloc_tmp(sizeof(int64_t) * (nwarps + 1), st));
        RELNN_CUDA(cudaMemsetAsync(wt.p, 0, sizeof(int64_t) * (nwarps + 1), st));
        const int blocks = (int)ceil_div(std::max<int64_t>(T, 1), 256);
        if (T > 0)
            { tri_count_kernel<<<blocks, 256, 0, st>>>(v, bd.d_src, bd.d_dst, T, p.kt, p.join_dst, filters_of(bd),
                                                     us.as<int32_t>(), ud.as<int32_t>(), wt.as<int64_t>()); note_launch(); }
        RELNN_TRY(exclusive_scan<int64_t>(wt.as<int64_t>(), wt.as<int64_t>(), nwarps, wt.as<int64_t>() + nwarps, st));
        RELNN_CUDA(cudaMemcpyAsync(&M, wt.as<int64_t>() + nwarps, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        RELNN_CUDA(cudaStreamSynchronize(st));
        if (M >= (1ll << 31) - 1) {
            *M_out = M;
            return RELNN_OK;  // rejected by the caller
        }
        const int64_t m1 = std::max<int64_t>(M, 1);
        RELNN_TRY(t.key.alloc_tmp(sizeof(K) * m1, st));
        RELNN_TRY(t.key_tmp.alloc_tmp(sizeof(K) * m1, st));
        RELNN_TRY(t.val.alloc_tmp(sizeof(V) * m1, st));
        RELNN_TRY(t.val_tmp.alloc_tmp(sizeof(V) * m1, st));
        if (T > 0) {
            { tri_emit_kernel<K, V><<<blocks, 256, 0, st>>>(v, bd.d_dst, T, p.kt, p.join_dst, t.omin, us.as<int32_t>(),
                                                          ud.as<int32_t>(), wt.as<int64_t>(), t.key.as<K>(),
                                                          t.val.as<V>()); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
        }
    }
    *M_out = M;
    return RELNN_OK;
}

template <class K, class V>
relnn_status emit_and_sort(Plan& p, const relnn_branch_desc& bd, Tmp& t, int64_t* M, int nbits, cudaStream_t st) {
    RELNN_TRY((emit_pairs<K, V>(p, bd, t, M, st)));
    if (*M >= (1ll << 31) - 1 || t.counted) return RELNN_OK;  // counted: grouped by group_by_counting
    return radix_sort_pairs<K, V>(t.key.as<K>(), t.val.as<V>(), t.key_tmp.as<K>(), t.val_tmp.as<V>(), *M, nbits, st,
                                  &t.in_tmp);
}

// The counting group-by of an emitted branch (t.counted): hs, hd and seg of every tuple in output
// order, the output keys, and in t.gpacked the scanned (count, present) pairs.
relnn_status group_by_counting(Plan& p, BranchPlan& b, Tmp& t, cudaStream_t st) {
    const JoinTable& HT = p.Ht();
    const int64_t n = p.n_h, M = b.m;
    RELNN_TRY(t.gpacked.alloc_tmp(sizeof(int64_t) * (n + 1), st));
    { group_pack_kernel<<<grid_for(n), 256, 0, st>>>(t.cnt.as<int32_t>(), n, t.gpacked.as<int64_t>()); note_launch(); }
    RELNN_TRY(exclusive_scan<int64_t>(t.gpacked.as<int64_t>(), t.gpacked.as<int64_t>(), n, t.gpacked.as<int64_t>() + n, st));
    RELNN_TRY(p.out_keys.alloc_nosync(sizeof(int64_t) * std::max<int64_t>(n, 1), st));
    DevBuf cur, lst;
    RELNN_TRY(cur.alloc_tmp(sizeof(int32_t) * std::max<int64_t>(n, 1), st));
    { group_heads_kernel<<<grid_for(n), 256, 0, st>>>(t.cnt.as<int32_t>(), t.gpacked.as<int64_t>(), n,
                                                    HT.ukeys.as<int64_t>(), cur.as<int32_t>(),
                                                    p.out_keys.as<int64_t>()); note_launch(); }
    if (M > 0)
        { group_scatter_kernel<<<ilp_grid(M), 256, 0, st>>>(t.key.as<uint32_t>(), t.val.as<int32_t>(), M,
                                                            cur.as<int32_t>(), b.hs.as<int32_t>()); note_launch(); }
    // groups above kGroupLane tuples: at most M / (kGroupLane + 1) of them, listed, then one block each
    const int64_t n_list = M / (kGroupLane + 1) + 1;
    RELNN_TRY(lst.alloc_tmp(sizeof(int32_t) * (n_list + 1), st));
    int* n_big = lst.as<int>() + n_list;
    RELNN_CUDA(cudaMemsetAsync(n_big, 0, sizeof(int), st));
    { group_sort_warp_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8)),
                                256, 0, st>>>(t.cnt.as<int32_t>(), t.gpacked.as<int64_t>(), n, HT.rows_sorted.as<int32_t>(),
                                              b.hs.as<int32_t>(), b.hd.as<int32_t>(), b.seg.as<int32_t>(),
                                              lst.as<int32_t>(), n_big); note_launch(); }
    { group_sort_block_kernel<<<(unsigned)std::min<int64_t>(n_list, (int64_t)num_sms() * 4), 256, 0, st>>>(
        t.cnt.as<int32_t>(), t.gpacked.as<int64_t>(), lst.as<int32_t>(), n_big, HT.rows_sorted.as<int32_t>(),
        b.hs.as<int32_t>(), b.hd.as<int32_t>(), b.seg.as<int32_t>()); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

relnn_status emit_branch(Plan& p, BranchPlan& b, const relnn_branch_desc& bd, Tmp& t, cudaStream_t st) {
    const int64_t T = bd.n_tuples;
    // group key width: dst sorted position (n_h < 2^31) or the raw dst key span
    int nbits = 0;
    if (p.join_dst) {
        nbits = bit_length((uint64_t)std::max<int64_t>(p.n_h - 1, 0));
        t.wide = false;
    } else {
        int64_t kmin = 0, kmax = 0;
        RELNN_TRY(key_range(bd.d_dst, T, p.kt, &kmin, &kmax, st));
        t.omin = (uint64_t)kmin ^ 0x8000000000000000ull;
        uint64_t span = ((uint64_t)kmax ^ 0x8000000000000000ull) - t.omin;
        nbits = bit_length(span);
        t.wide = nbits > 32;
    }
    t.pair = b.d_r > 0;
    // the counting group-by: one branch, a dst join over unique H keys, no E row carried, no
    // selection, no MAX (its tie order is the E order), not a stream chunk
    t.want_count = p.join_dst && !t.wide && !t.pair && p.br.size() == 1 && p.Ht().n_unique == p.n_h &&
                   !(p.flags & RELNN_FLAG_MAX) && !p.dense_out && filters_of(bd).n == 0 &&
                   tune_get(RELNN_TUNE_GROUP_SORT) == 1;
    t.defer = p.join_dst && !t.want_count && p.Ht().n_unique == p.n_h && filters_of(bd).n == 0 && T > 0;
    if (t.defer) {
        // the sentinel 2^nbits - 1 must lie above every dst position (< n_h)
        if (p.n_h > 0 && (uint64_t)p.n_h == (1ull << nbits)) ++nbits;
        t.sentinel = nbits >= 32 ? 0xffffffffu : (uint32_t)((1ull << nbits) - 1);
    }
    int64_t M = 0;
    if (t.wide) {
        if (t.pair) RELNN_TRY((emit_and_sort<uint64_t, int64_t>(p, bd, t, &M, nbits, st)));
        else RELNN_TRY((emit_and_sort<uint64_t, int32_t>(p, bd, t, &M, nbits, st)));
    } else {
        if (t.pair) RELNN_TRY((emit_and_sort<uint32_t, int64_t>(p, bd, t, &M, nbits, st)));
        else RELNN_TRY((emit_and_sort<uint32_t, int32_t>(p, bd, t, &M, nbits, st)));
    }
    if (M >= (1ll << 31) - 1) {
        set_error("rule plan: join output of " + std::to_string(M) + " tuples exceeds 2^31-1");
        return RELNN_ENOTSUP;
    }
    b.m = M;
    const int64_t m1 = std::max<int64_t>(M, 1);
    if (t.counted) {
        RELNN_TRY(b.hs.alloc_nosync(4 * m1, st));
        RELNN_TRY(b.hd.alloc_nosync(4 * m1, st));
        RELNN_TRY(b.seg.alloc_nosync(4 * (m1 + 1), st));
        RELNN_TRY(group_by_counting(p, b, t, st));
        t.key_tmp.release();
        t.val_tmp.release();
        return RELNN_OK;
    }
    // hs / er from the sorted payloads; hd and seg follow once the output rows are known
    if (t.pair) {
        RELNN_TRY(b.hs.alloc_nosync(4 * m1, st));
        RELNN_TRY(b.er.alloc_nosync(4 * m1, st));
        if (M > 0)
            { split_pair_kernel<<<grid_for(M), 256, 0, st>>>(t.sorted_val().as<int64_t>(), M, b.hs.as<int32_t>(),
                                                           b.er.as<int32_t>()); note_launch(); }
        t.val.release();
        t.val_tmp.release();
    } else {
        b.hs = std::move(t.sorted_val());
        b.hs.ordered = false;  // now a plan buffer: freed with the plan (after its work)
        b.hs.st = nullptr;
        t.val.release();
        t.val_tmp.release();
    }
    RELNN_TRY(b.hd.alloc_nosync(4 * m1, st));
    RELNN_TRY(b.seg.alloc_nosync(4 * (m1 + 1), st));
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

}  // namespace

relnn_status ensure_src_order(const Plan& p, BranchPlan& b, cudaStream_t st) {
    if (b.src_perm.p || b.m == 0) return RELNN_OK;
    const int64_t M = b.m;
    DevBuf key, key_tmp, val_tmp;
    RELNN_TRY(key.alloc_tmp(sizeof(uint32_t) * M, st));
    RELNN_TRY(key_tmp.alloc_tmp(sizeof(uint32_t) * M, st));
    RELNN_TRY(val_tmp.alloc_tmp(sizeof(int32_t) * M, st));
    RELNN_TRY(b.src_perm.alloc_nosync(sizeof(int32_t) * M, st));
    RELNN_TRY(b.hs_src.alloc_nosync(sizeof(int32_t) * M, st));
    RELNN_TRY(b.seg_src.alloc_nosync(sizeof(int32_t) * M, st));
    { src_pairs_kernel<<<grid_for(M), 256, 0, st>>>(b.hs.as<int32_t>(), M, key.as<uint32_t>(), b.src_perm.as<int32_t>()); note_launch(); }
    RELNN_TRY((radix_sort_pairs<uint32_t, int32_t>(key.as<uint32_t>(), b.src_perm.as<int32_t>(), key_tmp.as<uint32_t>(),
                                                    val_tmp.as<int32_t>(), M,
                                                    bit_length((uint64_t)std::max<int64_t>(p.n_h - 1, 0)), st)));
    RELNN_CUDA(cudaMemcpyAsync(b.hs_src.p, key.p, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st));
    { gather_i32_kernel<<<grid_for(M), 256, 0, st>>>(b.seg.as<int32_t>(), b.src_perm.as<int32_t>(), M, b.seg_src.as<int32_t>()); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    // the plan's buffers are used on other streams later
    RELNN_CUDA(cudaStreamSynchronize(st));
    return RELNN_OK;
}

relnn_status build_plan(Plan& p, const relnn_rule_desc* desc, cudaStream_t st) {
    RELNN_CHECK_ARG(desc, "rule plan: null descriptor");
    RELNN_CHECK_ARG(desc->key_type == RELNN_I32 || desc->key_type == RELNN_I64, "rule plan: bad key type");
    RELNN_CHECK_ARG(desc->n_branches >= 1 && desc->branches, "rule plan: need >= 1 branch");
    RELNN_CHECK_ARG(desc->d > 0 && desc->d <= 4096, "rule plan: bad embedding width d");
    RELNN_CHECK_ARG(desc->n_h >= 0 && (desc->n_h == 0 || desc->d_h_ids || p.Hx), "rule plan: bad H");
    RELNN_CHECK_ARG(desc->act == RELNN_ACT_NONE || desc->act == RELNN_ACT_RELU, "rule plan: bad act");
    p.kt = desc->key_type;
    p.flags = desc->flags;
    p.act = desc->act;
    p.d = desc->d;
    p.n_h = desc->n_h;
    p.join_dst = !(desc->flags & RELNN_FLAG_NO_JOIN_DST);
    p.concat_dst = p.join_dst && !(desc->flags & RELNN_FLAG_NO_CONCAT_DST);
    p.identity = (desc->flags & RELNN_FLAG_IDENTITY) != 0;
    p.bf16 = (desc->flags & RELNN_FLAG_BF16) != 0;
    p.kahan = (desc->flags & RELNN_FLAG_KAHAN) != 0;
    RELNN_CHECK_ARG(p.join_dst || desc->n_branches == 1, "rule plan: a union needs the dst join (shared key space)");
    if (desc->flags & RELNN_FLAG_MAX) {
        RELNN_CHECK_ARG(desc->n_branches == 1, "rule plan: MAX aggregator: single-branch rules only");
        RELNN_CHECK_ARG(!(desc->flags & (RELNN_FLAG_MEAN | RELNN_FLAG_PUSHDOWN)),
                        "rule plan: MAX aggregator excludes MEAN and PUSHDOWN");
    }
    const int d_r0 = desc->branches[0].d_r;
    for (int i = 0; i < desc->n_branches; ++i) {
        const relnn_branch_desc& b = desc->branches[i];
        RELNN_CHECK_ARG(b.n_tuples >= 0 && b.n_tuples < (1ll << 31) - 1, "rule plan: n_tuples out of range");
        RELNN_CHECK_ARG(b.n_tuples == 0 || (b.d_src && b.d_dst), "rule plan: null E column");
        RELNN_CHECK_ARG(b.d_r >= 0 && b.d_r <= 4096, "rule plan: bad d_r");
        RELNN_CHECK_ARG(b.d_r == d_r0, "rule plan: branches must share the Concat width");
        RELNN_CHECK_ARG(b.n_filters >= 0 && b.n_filters <= RELNN_MAX_FILTERS && (b.n_filters == 0 || b.filters),
                        "rule plan: bad filter list");
        for (int k = 0; k < b.n_filters; ++k) {
            const relnn_filter& f = b.filters[k];
            RELNN_CHECK_ARG(f.lhs >= RELNN_TERM_SRC && f.lhs <= RELNN_TERM_CONST && f.rhs >= RELNN_TERM_SRC &&
                                f.rhs <= RELNN_TERM_CONST && f.op >= RELNN_CMP_EQ && f.op <= RELNN_CMP_GE,
                            "rule plan: bad filter");
        }
    }
    p.d_in = p.d * (p.concat_dst ? 2 : 1) + d_r0;
    p.d_out = p.identity ? p.d_in : desc->d_out;
    RELNN_CHECK_ARG(p.d_out > 0 && p.d_out <= 4096, "rule plan: bad d_out");
    RELNN_TRY(p.status.alloc_nosync(sizeof(int) * kStatusInts, st));
    RELNN_CUDA(cudaMemsetAsync(p.status.p, 0, sizeof(int) * kStatusInts, st));

    // a1: build side over H.id
    if (!p.Hx) RELNN_TRY(join_table_build(p.H, desc->d_h_ids, desc->n_h, p.kt, st, false));
    const JoinTable& HT = p.Ht();
    const int64_t U = HT.n_unique;

    // a2: probe and emit per branch; a3: sort by group key
    p.br.clear();
    p.br.resize(desc->n_branches);
    std::vector<Tmp> tmp(desc->n_branches);
    for (int i = 0; i < desc->n_branches; ++i) {
        p.br[i].n_tuples = desc->branches[i].n_tuples;
        p.br[i].d_r = desc->branches[i].d_r;
        RELNN_TRY(emit_branch(p, p.br[i], desc->branches[i], tmp[i], st));
    }

    // output key set and output row of every matched tuple (sorted positions at or past pos_limit are
    // the sentinels of tuples that matched nothing)
    const uint32_t pos_limit = (uint32_t)std::min<int64_t>(HT.n, 0xffffffffll);
    int32_t nout_join = 0;
    int64_t counted_total = -1;
    if (p.join_dst && p.dense_out) {
        // stream chunk: output row = distinct index of the dst key; presence kept by the stream
        for (auto i = 0u; i < p.br.size(); ++i)
            if (p.br[i].m > 0) {
                { mark_present_kernel<<<ilp_grid(p.br[i].m), 256, 0, st>>>(
                    tmp[i].keys<uint32_t>(), p.br[i].m, HT.uid_of_pos.as<int32_t>(), p.present_ext, pos_limit); note_launch(); }
                { finalize_dst_kernel<<<ilp_grid(p.br[i].m), 256, 0, st>>>(
                    tmp[i].keys<uint32_t>(), p.br[i].m, HT.rows_sorted.as<int32_t>(), HT.uid_of_pos.as<int32_t>(),
                    p.iota_ext, p.br[i].hd.as<int32_t>(), p.br[i].seg.as<int32_t>(), pos_limit); note_launch(); }
            }
        RELNN_CUDA(cudaGetLastError());
        nout_join = (int32_t)U;
    } else if (p.join_dst && tmp.size() == 1 && tmp[0].counted) {
        // counting group-by: output keys, hd and seg are written; the output-row count is the high
        // half of the scanned total, read with the final synchronisation
        RELNN_CUDA(cudaMemcpyAsync(&counted_total, tmp[0].gpacked.as<int64_t>() + p.n_h, sizeof(int64_t),
                                   cudaMemcpyDeviceToHost, st));
    } else if (p.join_dst) {
        DevBuf present;
        RELNN_TRY(present.alloc_tmp(sizeof(int32_t) * (U + 1), st));
        RELNN_CUDA(cudaMemsetAsync(present.p, 0, sizeof(int32_t) * (U + 1), st));
        DevBuf out_row;
        RELNN_TRY(out_row.alloc_tmp(sizeof(int32_t) * (U + 1), st));
        for (auto i = 0u; i < p.br.size(); ++i)
            if (p.br[i].m > 0)
                { mark_present_kernel<<<ilp_grid(p.br[i].m), 256, 0, st>>>(
                    tmp[i].keys<uint32_t>(), p.br[i].m, HT.uid_of_pos.as<int32_t>(), present.as<int32_t>(), pos_limit); note_launch(); }
        RELNN_TRY(exclusive_scan<int32_t>(present.as<int32_t>(), out_row.as<int32_t>(), U, out_row.as<int32_t>() + U, st));
        RELNN_TRY(p.out_keys.alloc_nosync(sizeof(int64_t) * std::max<int64_t>(U, 1), st));
        if (U > 0)
            { out_keys_kernel<<<grid_for(U), 256, 0, st>>>(present.as<int32_t>(), out_row.as<int32_t>(),
                                                         HT.ukeys.as<int64_t>(), U, p.out_keys.as<int64_t>()); note_launch(); }
        for (auto i = 0u; i < p.br.size(); ++i)
            if (p.br[i].m > 0)
                { finalize_dst_kernel<<<ilp_grid(p.br[i].m), 256, 0, st>>>(
                    tmp[i].keys<uint32_t>(), p.br[i].m, HT.rows_sorted.as<int32_t>(), HT.uid_of_pos.as<int32_t>(),
                    out_row.as<int32_t>(), p.br[i].hd.as<int32_t>(), p.br[i].seg.as<int32_t>(), pos_limit); note_launch(); }
        RELNN_CUDA(cudaGetLastError());
        // the output-row count (U bounds it) is read with the final synchronisation; a copy to pageable
        // host memory returns only once it is done, so it is queued after the kernels above
        RELNN_CUDA(cudaMemcpyAsync(&nout_join, out_row.as<int32_t>() + U, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    } else {
        BranchPlan& b = p.br[0];
        Tmp& t = tmp[0];
        const int64_t M = b.m;
        DevBuf flags;
        RELNN_TRY(flags.alloc_tmp(sizeof(int32_t) * (M + 1), st));
        if (M > 0) {
            if (t.wide) { key_flags_kernel<uint64_t><<<grid_for(M), 256, 0, st>>>(t.keys<uint64_t>(), M, flags.as<int32_t>()); note_launch(); }
            else { key_flags_kernel<uint32_t><<<grid_for(M), 256, 0, st>>>(t.keys<uint32_t>(), M, flags.as<int32_t>()); note_launch(); }
        }
        RELNN_TRY(exclusive_scan<int32_t>(flags.as<int32_t>(), flags.as<int32_t>(), M, flags.as<int32_t>() + M, st));
        int32_t nout = 0;
        RELNN_CUDA(cudaMemcpyAsync(&nout, flags.as<int32_t>() + M, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        RELNN_CUDA(cudaStreamSynchronize(st));
        p.n_out = nout;
        RELNN_TRY(p.out_keys.alloc_nosync(sizeof(int64_t) * std::max<int64_t>(nout, 1), st));
        // without a dst join there is no dst H row
        RELNN_CUDA(cudaMemsetAsync(b.hd.p, 0xff, b.hd.bytes, st));
        if (M > 0) {
            if (t.wide)
                { raw_seg_kernel<uint64_t><<<grid_for(M), 256, 0, st>>>(t.keys<uint64_t>(), flags.as<int32_t>(), M,
                                                                      t.omin, b.seg.as<int32_t>(), p.out_keys.as<int64_t>()); note_launch(); }
            else
                { raw_seg_kernel<uint32_t><<<grid_for(M), 256, 0, st>>>(t.keys<uint32_t>(), flags.as<int32_t>(), M,
                                                                      t.omin, b.seg.as<int32_t>(), p.out_keys.as<int64_t>()); note_launch(); }
        }
        RELNN_CUDA(cudaGetLastError());
    }
    // device-side checks of the plan kernels (a look-back that gave up) and the deferred miss counts,
    // with the final sync
    int dev_status = 0;
    std::vector<unsigned long long> misses(p.br.size(), 0);
    for (size_t i = 0; i < p.br.size(); ++i)
        if (tmp[i].defer && tmp[i].miss.p)
            RELNN_CUDA(cudaMemcpyAsync(&misses[i], tmp[i].miss.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaMemcpyAsync(&dev_status, p.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < p.br.size(); ++i)
        if (tmp[i].defer) p.br[i].m -= (int64_t)std::min<unsigned long long>(misses[i], (unsigned long long)p.br[i].m);
    if (counted_total >= 0) nout_join = (int32_t)(counted_total >> 32);
    if (p.join_dst) p.n_out = nout_join;
    if (dev_status) {
        set_device_error(dev_status);
        set_error("rule plan: device check failed");
        return RELNN_EDEVICE;
    }
    return RELNN_OK;
}

}  // namespace relnn
