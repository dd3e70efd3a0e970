// BF16 form of the rule forward on tcgen05 tensor cores (sm_103a): gather -> Concat -> Linear
// (+ReLU) -> segmented SUM, fused in one persistent kernel.
//
// The Linear is computed transposed: D[o][t] = sum_k W[o][k] X[t][k], M = output features (a
// 128-row block of W), N = a tile of tile_n matched tuples, K = the Concat width in 64-element
// blocks. TMEM lane o then holds feature o of every tuple of the tile in consecutive columns, so the
// epilogue thread that owns feature o reads its tuples in output-key order and the SUM over a run of
// equal output rows is a walk in registers; each emitted row is a 128-byte coalesced store per warp.
//
// Roles (512 threads, one CTA per SM; 16 warps leave 128 registers per thread):
//   warps 0-6  producers: gather rows z[hs], z[hd], r[er] for one 64-column K block of a tile into
//              a 128B-swizzled stage (cp.async for bf16 sources, convert-and-store for f32 sources);
//              the tile's row indices are staged by cp.async two tiles ahead
//   warp 7     TMEM allocation; lane 0 issues tcgen05.mma (A = W block staged once by TMA,
//              B = the gathered stage) and tcgen05.commit
//   warps 8-15 epilogue, two warps per TMEM lane quarter, each owning one half of the tile's
//              columns (a half-tile is the unit of the SUM walk and of the boundary partials):
//              tcgen05.ld of the accumulator (double-buffered in TMEM so the next tile's MMAs
//              overlap), bias, ReLU, SUM walk, stores / unit-boundary partials.
// Narrow outputs (d_out <= 64) leave lane quarters empty, so W is replicated into them (2 or 4
// copies): every quarter then holds all features of the tile, and each of the rep warps sharing a
// feature quarter walks 1/rep of the half-tile's columns (the unit shrinks to half_n / rep).
#include "agg.cuh"
#include "fwd.cuh"
#include "maxagg.cuh"
#include "segscan.cuh"
#include "tc.cuh"

#include <algorithm>
#include <mutex>

namespace relnn {

namespace {

using namespace tc;

constexpr int kThreads = 512;
constexpr int kProducerThreads = 224;
constexpr int kMmaWarp = 7;     // warps 0-6 produce, 8-15 are the epilogue
constexpr int kEpiWarps = 8;
constexpr int kIdxSlots = 3;    // row-index ring: the tile in production and the next two
constexpr int kRowGroups = kProducerThreads / 8;                 // 28 rows per pass of the producers
constexpr int kMaxRows = (256 + kRowGroups - 1) / kRowGroups;    // rows per producer thread per stage
// Staged row indices: in row order (16-byte copies; each producer thread then reads its rows'
// indices one by one, once per Concat part), or transposed when every part is a single K block
// (entry (row group rg, k) = index of row rg + 28 k at rg * kIdxPitch + k, staged by 4-byte copies,
// so a producer thread reads its rows' indices with three 16-byte loads).
constexpr int kIdxPitch = 12;
constexpr int kIdxArr = kRowGroups * kIdxPitch;                  // ints per staged index array
static_assert(kMaxRows <= kIdxPitch && kIdxPitch % 4 == 0 && kIdxArr >= 256, "index layout");
constexpr int kMaxKb = 12;
constexpr int kSmemLimit = 227 * 1024;

struct TcArgs {
    const void* z;
    const void* r;
    const int32_t* hs;
    const int32_t* hd;
    const int32_t* er;
    const int32_t* seg;
    const float* bias;
    float* out;
    float* carry;
    int32_t* arg;         // MAX: [n_out][d_out] plan position of each maximum (-1: ReLU'd zero)
    int32_t* carry_pos;   // MAX: the positions of the boundary partials in `carry`
    int* status;
    uint32_t* relu_mask;
    int64_t m;
    int64_t n_tiles;
    int64_t z_rows, r_rows;  // rows of z and r (the checked build tests the gathered indices)
    int z_bf16, r_bf16, d, d_r;
    int d_out, act, kahan, accumulate;
    int n_kb, tile_n, m_blocks, stages, mask_words;
    int rep;              // copies of W in the 128 TMEM lanes (d_out <= 64: 2, <= 32: 4)
    uint32_t idesc, tmem_cols;
    int kb_src[kMaxKb];   // 0: z[hs], 1: z[hd], 2: r[er]
    int kb_col[kMaxKb];   // first element of the block within its part
    int kb_width[kMaxKb]; // width of that part
    int need_arr[3];      // which of hs, hd, er the K blocks read
};

// Aggregation of the epilogue: SUM walk, one row per tuple (dense product), or MAX with argmax.
constexpr int kAggSum = 0, kAggDense = 1, kAggMax = 2;

template <bool IDX_T, int AGG>
__global__ void __launch_bounds__(kThreads, 1)
fwd_tc_kernel(const __grid_constant__ CUtensorMap wmap, const __grid_constant__ TcArgs a) {
    extern __shared__ uint8_t dyn_smem[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~(uintptr_t)1023);
    const uint32_t w_bytes = (uint32_t)a.n_kb * a.m_blocks * 16384u;
    const uint32_t stage_bytes = (uint32_t)a.tile_n * 128u;
    uint8_t* w_smem = base;
    uint8_t* st_smem = base + w_bytes;
    // row indices of the tiles being gathered (kIdxSlots x {hs, hd, er} x tile_n)
    int32_t* idx_smem = reinterpret_cast<int32_t*>(st_smem + (size_t)a.stages * stage_bytes);
    // each epilogue warp walks the columns of one half of a tile (or 1/rep of it)
    const int half_n = a.tile_n / 2;
    uint64_t* bars = reinterpret_cast<uint64_t*>(idx_smem + kIdxSlots * 3 * kIdxArr);
    uint64_t* full = bars;
    uint64_t* empty = bars + a.stages;
    uint64_t* tfull = bars + 2 * a.stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* wbar = tempty + 2;
    uint64_t* drain = wbar + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(smem_u32(&full[s]), kProducerThreads);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&tfull[i]), 1);
            mbar_init(smem_u32(&tempty[i]), 32 * kEpiWarps);
        }
        mbar_init(smem_u32(wbar), 1);
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t acc_stride = (uint32_t)a.m_blocks * a.tile_n;

    if (warp < kProducerThreads / 32) {
        // ------------------------------------------------------------------ producers
        // Thread (row group rg, 16-byte chunk) copies chunk `chunk` of rows rg, rg + 28, rg + 56, ...
        // of every K block, so the 8 lanes of a row read its 128-byte segment together (4 rows per
        // warp instruction); the row indices of a stage are all loaded before the copies are issued.
        const int chunk = tid & 7;
        const int rg = tid >> 3;
        // cp.async of one tile's hs / hd / er entries (4 bytes each, zero-filled past m) into a slot
        // in the transposed layout; committed as one group
        auto issue_idx = [&](int64_t tile, int slot) {
            int32_t* dstb = idx_smem + slot * 3 * kIdxArr;
            if (!IDX_T) {
                const int q_per_arr = a.tile_n / 4;
                for (int e = tid; e < 3 * q_per_arr; e += kProducerThreads) {
                    const int r = e / q_per_arr, qq = e - r * q_per_arr;
                    if (!a.need_arr[r]) continue;
                    const int32_t* arr = r == 0 ? a.hs : (r == 1 ? a.hd : a.er);
                    const int64_t t = tile * a.tile_n + 4 * qq;
                    const int64_t left = (tile < a.n_tiles) ? a.m - t : 0;
                    const uint32_t bytes = left >= 4 ? 16u : (left > 0 ? (uint32_t)left * 4u : 0u);
                    cp_async_16_stream(smem_u32(dstb + r * kIdxArr + 4 * qq), bytes ? arr + t : arr, bytes);
                }
                cp_async_commit();
                return;
            }
            for (int e = tid; e < 3 * a.tile_n; e += kProducerThreads) {
                const int r = e >= 2 * a.tile_n ? 2 : (e >= a.tile_n ? 1 : 0);
                if (!a.need_arr[r]) continue;
                const int row = e - r * a.tile_n;
                const int32_t* arr = r == 0 ? a.hs : (r == 1 ? a.hd : a.er);
                const int64_t t = tile * a.tile_n + row;
                const bool valid = tile < a.n_tiles && t < a.m;
                cp_async_4(smem_u32(dstb + r * kIdxArr + (row % kRowGroups) * kIdxPitch + row / kRowGroups),
                           valid ? arr + t : arr, valid ? 4u : 0u);
            }
            cp_async_commit();
        };
        issue_idx(blockIdx.x, 0);
        issue_idx((int64_t)blockIdx.x + gridDim.x, 1);
        cp_async_wait<1>();
        named_bar_sync(1, kProducerThreads);
        int it = 0;
        bool ok = true;
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++lt) {
            const int64_t t0 = tile * a.tile_n;
            const int32_t* islot = idx_smem + (lt % kIdxSlots) * 3 * kIdxArr;
            // indices two tiles ahead (that slot was last read two tiles ago, before a barrier)
            issue_idx(tile + 2 * (int64_t)gridDim.x, (lt + 2) % kIdxSlots);
            // this thread's row indices, reloaded only when the K block reads another Concat part
            int32_t ridx[kMaxRows];
            int ridx_src = -1;
            for (int kb = 0; kb < a.n_kb; ++kb) {
                if (!ok) break;
                const int s = it % a.stages;
                const uint32_t ph = (uint32_t)((it / a.stages) & 1);
                if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, a.status, abort_flag)) { ok = false; break; }
                const int src = a.kb_src[kb];
                const int32_t* rows_idx = islot + src * kIdxArr;
                const void* tbl = src == 2 ? a.r : a.z;
                const int64_t tbl_rows = src == 2 ? a.r_rows : a.z_rows;
                const int tbl_bf16 = src == 2 ? a.r_bf16 : a.z_bf16;
                const int row_elems = src == 2 ? a.d_r : a.d;
                const uint32_t sbase = smem_u32(st_smem + (size_t)s * stage_bytes);
                const int col = a.kb_col[kb] + chunk * 8;
                const bool in_part = col < a.kb_width[kb];
                if (src != ridx_src && !IDX_T) {
#pragma unroll
                    for (int k = 0; k < kMaxRows; ++k) {
                        const int row = rg + k * kRowGroups;
                        ridx[k] = row < a.tile_n ? rows_idx[row] : 0;
                    }
                    ridx_src = src;
                } else if (src != ridx_src) {
                    const int4* rp = reinterpret_cast<const int4*>(rows_idx + rg * kIdxPitch);
                    const int4 i0 = rp[0], i1 = rp[1], i2 = rp[2];
                    const int32_t all[12] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w, i2.x, i2.y, i2.z, i2.w};
#pragma unroll
                    for (int k = 0; k < kMaxRows; ++k) ridx[k] = all[k];  // rows past tile_n are never copied
                    ridx_src = src;
                }
                // destination of row `row`: 128-byte line, 16-byte chunk swizzled by the row (SW128)
                auto dst_of = [&](int row) {
                    return sbase + (uint32_t)row * 128u + ((uint32_t)(chunk ^ (row & 7)) << 4);
                };
                if (tbl_bf16) {
                    const uint16_t* p = reinterpret_cast<const uint16_t*>(tbl);
                    if (src == 2) {
#pragma unroll
                        for (int k = 0; k < kMaxRows; ++k) {
                            const int row = rg + k * kRowGroups;
                            if (row >= a.tile_n) break;
                            const bool valid = (t0 + row < a.m) && in_part && in_bounds(ridx[k], tbl_rows, a.status);
                            cp_async_16_stream(dst_of(row), valid ? p + (int64_t)ridx[k] * row_elems + col : p,
                                               valid ? 16u : 0u);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < kMaxRows; ++k) {
                            const int row = rg + k * kRowGroups;
                            if (row >= a.tile_n) break;
                            const bool valid = (t0 + row < a.m) && in_part && in_bounds(ridx[k], tbl_rows, a.status);
                            cp_async_16(dst_of(row), valid ? p + (int64_t)ridx[k] * row_elems + col : p,
                                        valid ? 16u : 0u);
                        }
                    }
                } else {
                    // f32 rows: five rows' loads in flight before their convert-and-store
                    const float* pf32 = reinterpret_cast<const float*>(tbl);
#pragma unroll
                    for (int k0 = 0; k0 < kMaxRows; k0 += 5) {
                        float4 u[5], w[5];
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            const int row = rg + (k0 + k) * kRowGroups;
                            const bool valid = k0 + k < kMaxRows && row < a.tile_n && (t0 + row < a.m) && in_part &&
                                               in_bounds(ridx[k0 + k < kMaxRows ? k0 + k : 0], tbl_rows, a.status);
                            const float4* qp = reinterpret_cast<const float4*>(
                                pf32 + (valid ? (int64_t)ridx[k0 + k < kMaxRows ? k0 + k : 0] * row_elems + col : 0));
                            u[k] = valid ? __ldg(qp) : make_float4(0.f, 0.f, 0.f, 0.f);
                            w[k] = valid ? __ldg(qp + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            const int row = rg + (k0 + k) * kRowGroups;
                            if (k0 + k >= kMaxRows || row >= a.tile_n) break;
                            st_shared_v4(dst_of(row), pack_bf16x2(u[k].x, u[k].y), pack_bf16x2(u[k].z, u[k].w),
                                         pack_bf16x2(w[k].x, w[k].y), pack_bf16x2(w[k].z, w[k].w));
                        }
                    }
                }
                // The stage is complete for this thread when its copies have landed: cp.async sources
                // arrive asynchronously (the thread moves on to the next stage at once); converted f32
                // rows were stored by the thread itself and are published with a proxy fence.
                if (tbl_bf16) {
                    cp_async_mbar_arrive_noinc(smem_u32(&full[s]));
                } else {
                    fence_proxy_async();
                    mbar_arrive(smem_u32(&full[s]));
                }
                ++it;
            }
            // the next tile's indices (issued two tiles ago) have landed for every producer thread
            cp_async_wait<1>();
            named_bar_sync(1, kProducerThreads);
        }
        // no copy may still be writing shared memory when the CTA retires
        cp_async_wait<0>();
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = true;
            const uint32_t wb = smem_u32(wbar);
            mbar_arrive_expect_tx(wb, w_bytes);
            for (int kb = 0; kb < a.n_kb; ++kb)
                for (int mb = 0; mb < a.m_blocks; ++mb)
                    tma_load_2d(smem_u32(w_smem + (size_t)(kb * a.m_blocks + mb) * 16384u), &wmap, kb * 64,
                                mb * 128, wb);
            ok = mbar_wait(wb, 0, a.status, abort_flag);
            tc_fence_after();
            int it = 0;
            int lt = 0;
            for (int64_t tile = blockIdx.x; tile < a.n_tiles && ok; tile += gridDim.x, ++lt) {
                const int acc = lt & 1;
                const uint32_t use = (uint32_t)(lt >> 1);
                if (!mbar_wait(smem_u32(&tempty[acc]), (use & 1u) ^ 1u, a.status, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_acc = tmem_base + (uint32_t)acc * acc_stride;
                for (int kb = 0; kb < a.n_kb; ++kb, ++it) {
                    const int s = it % a.stages;
                    const uint32_t ph = (uint32_t)((it / a.stages) & 1);
                    if (!mbar_wait(smem_u32(&full[s]), ph, a.status, abort_flag)) { ok = false; break; }
                    // the stage was written through the generic proxy (cp.async): order it before the
                    // tensor core's reads
                    fence_proxy_async();
                    tc_fence_after();
                    const uint32_t b_base = smem_u32(st_smem + (size_t)s * stage_bytes);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t bdesc = sw128_kmajor_desc(b_base + k * 32);
                        for (int mb = 0; mb < a.m_blocks; ++mb) {
                            const uint64_t adesc = sw128_kmajor_desc(
                                smem_u32(w_smem + (size_t)(kb * a.m_blocks + mb) * 16384u) + k * 32);
                            mma_bf16(d_acc + (uint32_t)mb * a.tile_n, adesc, bdesc, a.idesc, (kb | k) != 0);
                        }
                    }
                    mma_commit(smem_u32(&empty[s]));
                }
                if (!ok) break;
                mma_commit(smem_u32(&tfull[acc]));
            }
            // make sure every issued MMA has finished before TMEM is released
            mma_commit(smem_u32(drain));
            mbar_wait(smem_u32(drain), 0, a.status, abort_flag);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------ epilogue
        const int q = warp & 3;                      // TMEM lane quarter this warp may access
        const int ew = warp - kMmaWarp - 1;          // 0..7 (quarters 0-3, then 0-3 again)
        const int hh = ew >> 2;                      // which half of the tile's columns
        const int n_fq = 4 / a.rep;                  // feature quarters (the rest are W replicas)
        const int fq = q % n_fq;                     // this warp's features: 32 * fq + lane
        const int unit = half_n / a.rep;             // columns per warp and tile
        const int ucol = hh * half_n + (q / n_fq) * unit;  // first column of this warp's unit
        const int n_unit_chunks = unit / 32;
        const bool relu = a.act == RELNN_ACT_RELU;
        const bool mask = relu && a.relu_mask != nullptr;
        float bias_r[2];
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
            const int o = mb * 128 + 32 * fq + lane;
            bias_r[mb] = (a.bias && mb < a.m_blocks && o < a.d_out) ? a.bias[o] : 0.f;
        }
        // output rows of this warp's unit of the next tile, loaded one tile ahead (up to 4 x 32)
        int pf[4];
        int pf_prev = -1, pf_after = -1;
        auto prefetch = [&](int64_t tile) {
            const int64_t h0 = tile * a.tile_n + ucol;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t t = h0 + 32 * c + lane;
                pf[c] = (tile < a.n_tiles && c < n_unit_chunks && t < a.m) ? __ldg(a.seg + t) : -1;
            }
            pf_prev = (tile < a.n_tiles && h0 > 0 && h0 - 1 < a.m) ? __ldg(a.seg + h0 - 1) : -1;
            pf_after = (tile < a.n_tiles && h0 + unit < a.m) ? __ldg(a.seg + h0 + unit) : -1;
        };
        prefetch(blockIdx.x);
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            // output rows of this warp's columns: chunk c, lane l -> row of column 32 c + l
            const int cs0 = pf[0], cs1 = pf[1], cs2 = pf[2], cs3 = pf[3];
            const int prev_seg = pf_prev;
            const int after_seg = pf_after;
            prefetch(tile + gridDim.x);
            // warp-uniform outcome of the bounded wait, so no lane runs the .sync.aligned loads alone
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[acc]), use & 1u, a.status, abort_flag))) break;
            tc_fence_after();
            const int64_t t0 = tile * a.tile_n + ucol;
            const int64_t vtile = t0 / unit;         // unit index (the boundary partials' slot)
            const int nt = (int)imin64(unit, a.m - t0);  // <= 0 for an empty unit
            for (int mb = 0; mb < a.m_blocks; ++mb) {
                const int obase = mb * 128 + 32 * fq;
                if (obase >= a.d_out) continue;
                const int o = obase + lane;
                const bool o_ok = o < a.d_out;
                const float bo = mb == 0 ? bias_r[0] : bias_r[1];
                float sum = 0.f, comp = 0.f;
                int rpos = 0;  // MAX: plan position of the running maximum
                bool first = true;
                unsigned prev_end = 1u;  // did the tuple before this chunk end a piece? (half start: yes)
                const uint32_t taddr = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)acc * acc_stride +
                                       (uint32_t)mb * a.tile_n + (uint32_t)ucol;
                for (int c = 0; c * 32 < nt; ++c) {
                    uint32_t v[32];
                    tmem_ld_32x32b_x32(taddr + (uint32_t)c * 32, v);
                    tmem_ld_wait();
                    if (AGG == kAggDense) {
                        // every tuple is its own output row (row t of a dense product): one
                        // coalesced 128-byte store per tuple, no SUM walk
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (c * 32 + j < nt && o_ok)
                                __stcg(a.out + (t0 + c * 32 + j) * a.d_out + o, __uint_as_float(v[j]) + bo);
                        continue;
                    }
                    const int li = c * 32 + lane;  // this lane's row in the half-tile
                    const bool tvalid = li < nt;
                    // a piece ends at row j if the next row has another output row or j is the
                    // half-tile's last row; it starts at j if row j-1 ended one
                    const int sg = c == 0 ? cs0 : (c == 1 ? cs1 : (c == 2 ? cs2 : cs3));
                    const int sgn = c == 0 ? cs1 : (c == 1 ? cs2 : cs3);  // next chunk's (lane 0 used)
                    int nx = __shfl_down_sync(0xffffffffu, sg, 1);
                    const int nx31 = __shfl_sync(0xffffffffu, sgn, 0);
                    if (lane == 31) nx = (li + 1 < unit) ? nx31 : after_seg;
                    const unsigned endmask = __ballot_sync(0xffffffffu, tvalid && (sg != nx || li == nt - 1));
                    const unsigned startmask = (endmask << 1) | prev_end;
                    prev_end = endmask >> 31;
                    uint32_t mword = 0;
                    unsigned takemask = 0;  // MAX: rows where the piece's running maximum was taken
                    // segmented running sum (maximum) over the chunk: v[j] <- sum (maximum) of its
                    // piece up to row j
                    if (AGG == kAggMax) {
                        if (relu) seg_scan_max<true>(v, bo, startmask, sum, takemask);
                        else seg_scan_max<false>(v, bo, startmask, sum, takemask);
                    } else if (a.kahan) {
                        if (mask) seg_scan<true, true, true>(v, bo, startmask, sum, comp, mword, lane);
                        else if (relu) seg_scan<true, true, false>(v, bo, startmask, sum, comp, mword, lane);
                        else seg_scan<false, true, false>(v, bo, startmask, sum, comp, mword, lane);
                    } else {
                        if (mask) seg_scan<true, false, true>(v, bo, startmask, sum, comp, mword, lane);
                        else if (relu) seg_scan<true, false, false>(v, bo, startmask, sum, comp, mword, lane);
                        else seg_scan<false, false, false>(v, bo, startmask, sum, comp, mword, lane);
                    }
                    // one store per piece end: the running sums go back to TMEM and each end's column is
                    // read back (four ends per round trip), instead of selecting registers by a run-time
                    // index
                    if (endmask) {
                        tmem_st_32x32b_x32(taddr + (uint32_t)c * 32, v);
                        tmem_st_wait();
                    }
                    for (unsigned em = endmask; em;) {
                        int jj[4];
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            jj[g] = em ? __ffs(em) - 1 : -1;
                            em &= em - 1u;
                        }
                        uint32_t vv[4];
#pragma unroll
                        for (int g = 0; g < 4; ++g)
                            vv[g] = jj[g] >= 0 ? tmem_ld_32x32b_x1(taddr + (uint32_t)(c * 32 + jj[g])) : 0u;
                        tmem_ld_wait();
#pragma unroll
                        for (int g = 0; g < 4; ++g) tmem_ld_after(vv[g]);
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            if (jj[g] < 0) break;
                            const int j = jj[g];
                            const float val = __uint_as_float(vv[g]);
                            const int s = __shfl_sync(0xffffffffu, sg, j);
                            const bool last = (c * 32 + j == nt - 1);
                            const int sn = last ? ((nt == unit) ? after_seg : -1) : s + 1;
                            const bool split = (first && prev_seg == s) || (last && sn == s);
                            if (AGG == kAggMax) {
                                // the piece's maximum was first reached at its last take up to row j
                                const unsigned tk = takemask & (0xffffffffu >> (31 - j));
                                const int pos = tk ? (int)(t0 + c * 32 + 31 - __clz(tk)) : rpos;
                                if (o_ok) {
                                    if (split) {
                                        const int64_t ci = (vtile * 2 + (first ? 0 : 1)) * a.d_out + o;
                                        __stcg(a.carry + ci, val);
                                        __stcg(a.carry_pos + ci, pos);
                                    } else {
                                        __stcs(a.out + (int64_t)s * a.d_out + o, val);
                                        __stcs(a.arg + (int64_t)s * a.d_out + o, (relu && !(val > 0.f)) ? -1 : pos);
                                    }
                                }
                            } else if (o_ok) {
                                if (split) __stcg(a.carry + (vtile * 2 + (first ? 0 : 1)) * a.d_out + o, val);
                                else emit_out(a.out + (int64_t)s * a.d_out + o, val, a.accumulate);
                            }
                            first = false;
                        }
                    }
                    // MAX: the open piece's position carried into the next chunk
                    if (AGG == kAggMax && takemask) rpos = (int)(t0 + c * 32 + 31 - __clz(takemask));
                    if (mask && tvalid) a.relu_mask[(t0 + li) * a.mask_words + mb * 4 + fq] = mword;
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&tempty[acc]));
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem_base, a.tmem_cols);
    }
}

// out[i] = bf16(z[i]) (round to nearest even), 4 elements per thread and step.
__global__ void z_to_bf16_kernel(const float4* __restrict__ z, int64_t n4, uint2* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(z + i);
        out[i] = make_uint2(pack_bf16x2(v.x, v.y), pack_bf16x2(v.z, v.w));
    }
}

// W_pad[mb*128 + o][kb*64 + kk] (bf16) = W[o][k(kb, kk)] with zero padding; with rep_rows < rows_pad
// the padded rows repeat W every rep_rows rows.
__global__ void pack_w_kernel(const void* W, int w_bf16, int d_out, int d_in, int rows_pad, int rep_rows, int n_kb,
                              const int* kb_kofs, const int* kb_width_left, uint16_t* wp) {
    const int cols = n_kb * 64;
    const int n = rows_pad * cols;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int prow = i / cols, cc = i - prow * cols;
        const int row = prow % rep_rows;  // replicated copies of W
        const int kb = cc >> 6, kk = cc & 63;
        uint16_t v = 0;
        if (row < d_out && kk < kb_width_left[kb]) {
            const int k = kb_kofs[kb] + kk;
            if (w_bf16) {
                v = reinterpret_cast<const uint16_t*>(W)[row * d_in + k];
            } else {
                const float f = reinterpret_cast<const float*>(W)[row * d_in + k];
                v = __bfloat16_as_ushort(__float2bfloat16_rn(f));
            }
        }
        wp[i] = v;
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

}  // namespace

relnn_status encode_bf16_tile_map(CUtensorMap* m, void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
    EncodeTiledFn enc = get_encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return RELNN_ECUDA;
    }
    cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
        return RELNN_ECUDA;
    }
    return RELNN_OK;
}

// Concat layout for the tensor-core path: every part (z_src, z_dst, r) starts on a 64-column
// K block; K blocks never straddle parts.
struct KbLayout {
    int n_kb = 0;
    int src[kMaxKb], col[kMaxKb], width[kMaxKb], kofs[kMaxKb], left[kMaxKb];
};

static bool make_layout(const Plan& p, KbLayout& L) {
    int kofs = 0;
    auto add_part = [&](int src, int width) {
        for (int c = 0; c < width; c += 64) {
            if (L.n_kb >= kMaxKb) return false;
            L.src[L.n_kb] = src;
            L.col[L.n_kb] = c;
            L.width[L.n_kb] = width;
            L.kofs[L.n_kb] = kofs + c;
            L.left[L.n_kb] = std::min(64, width - c);
            ++L.n_kb;
        }
        kofs += width;
        return true;
    };
    if (!add_part(0, p.d)) return false;
    if (p.concat_dst && !add_part(1, p.d)) return false;
    if (p.br[0].d_r > 0 && !add_part(2, p.br[0].d_r)) return false;
    return true;
}

void f32_to_bf16(const float* src, int64_t n, uint16_t* dst, cudaStream_t st) {
    const int64_t n4 = n / 4;
    if (n4 == 0) return;
    const int blocks = (int)std::min<int64_t>(ceil_div(n4, 256), (int64_t)num_sms() * 16);
    { z_to_bf16_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4*>(src), n4, reinterpret_cast<uint2*>(dst)); note_launch(); }
}

relnn_status with_bf16_z(Plan& p, const CallIO& io, CallIO& out, cudaStream_t st) {
    out = io;
    // (an f32 table that is not 16-byte aligned keeps the kernels' convert-as-you-gather path)
    if (io.z_bf16 || p.n_h == 0 || (reinterpret_cast<uintptr_t>(io.z) & 15u)) return RELNN_OK;
    const int64_t n = p.n_h * (int64_t)p.d;  // d % 8 == 0 on the tensor-core path
    out.z = p.zbf.p;
    out.z_bf16 = 1;
    if (p.z_version != 0 && p.zbf.p && p.zbf_src == io.z && p.zbf_version == p.z_version &&
        p.zbf.bytes >= sizeof(uint16_t) * (size_t)n)
        return RELNN_OK;  // the copy converted for this table version
    RELNN_TRY(p.zbf.alloc_nosync(sizeof(uint16_t) * n, st));
    p.zbf_src = io.z;
    p.zbf_version = p.z_version;
    const int64_t n4 = n / 4;
    const int blocks = (int)std::min<int64_t>(ceil_div(n4, 256), (int64_t)num_sms() * 16);
    { z_to_bf16_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4*>(io.z), n4, p.zbf.as<uint2>()); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    out.z = p.zbf.p;
    out.z_bf16 = 1;
    return RELNN_OK;
}

relnn_status forward_tc(Plan& p, const CallIO& io_in, float* out, cudaStream_t st) {
    // linear SUM / MEAN rules: sum each output row's Concat rows first, then one GEMM row (agg.cu)
    if (agg_forward_ok(p, io_in, out)) return forward_agg(p, io_in, out, st);
    if (p.identity) {
        set_error("BF16 form needs a Linear (identity rules run in the FP32 form)");
        return RELNN_ENOTSUP;
    }
    if (p.d % 8 != 0 || p.br[0].d_r % 8 != 0) {
        set_error("BF16 form: d and d_r must be multiples of 8");
        return RELNN_ENOTSUP;
    }
    if (p.d_out > 256) {
        set_error("BF16 form: d_out must be <= 256");
        return RELNN_ENOTSUP;
    }
    KbLayout L;
    if (!make_layout(p, L)) {
        set_error("BF16 form: Concat too wide");
        return RELNN_ENOTSUP;
    }
    CallIO io;
    RELNN_TRY(with_bf16_z(p, io_in, io, st));
    const int m_blocks = (p.d_out + 127) / 128;
    // 256 matched tuples per tile; 128 when d_out needs two TMEM blocks or the caller asks for
    // smaller tiles (more tiles per SM on small inputs)
    const int tile_n = (m_blocks == 1 && !(p.flags & RELNN_FLAG_TILE128)) ? 256 : 128;
    const uint32_t w_bytes = (uint32_t)L.n_kb * m_blocks * 16384u;
    const uint32_t stage_bytes = (uint32_t)tile_n * 128u;
    const int bar_bytes = 256;
    // staged row indices (kIdxSlots x 3 arrays)
    const int aux_bytes = 4 * (kIdxSlots * 3 * kIdxArr);
    int stages = (int)((kSmemLimit - 1024 - bar_bytes - aux_bytes - (int)w_bytes) / (int)stage_bytes);
    stages = std::min(stages, 8);
    if (stages < 2) {
        set_error("BF16 form: weights too large for shared memory");
        return RELNN_ENOTSUP;
    }
    const size_t smem = 1024 + w_bytes + (size_t)stages * stage_bytes + aux_bytes + bar_bytes;
    EncodeTiledFn enc = get_encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return RELNN_ECUDA;
    }
    // several branches add into one output; a stream chunk adds into the stream's accumulator
    const bool multi = p.br.size() > 1 || p.acc_out;
    if (p.br.size() > 1 && !p.acc_out) RELNN_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * p.n_out * p.d_out, st));
    // replicas of W in the lane quarters, and the column unit of the SUM walk / boundary partials
    const int half_n = tile_n / 2;
    int rep = m_blocks == 1 ? (p.d_out <= 32 ? 4 : (p.d_out <= 64 ? 2 : 1)) : 1;
    while (rep > 1 && half_n / rep < 32) rep /= 2;
    const int unit = half_n / rep;
    int64_t max_units = 1;
    for (auto& b : p.br) max_units = std::max<int64_t>(max_units, ceil_div(b.m, unit));
    RELNN_TRY(p.carry.alloc_nosync(sizeof(float) * 2 * p.d_out * max_units, st));
    const int rows_pad = m_blocks * 128;
    const size_t wp_elems = (size_t)rows_pad * L.n_kb * 64;
    RELNN_TRY(p.wpack.alloc_nosync(wp_elems * 2 + 256, st));
    int* d_meta = reinterpret_cast<int*>(p.wpack.as<uint8_t>() + wp_elems * 2);
    int meta[2 * kMaxKb];
    for (int i = 0; i < L.n_kb; ++i) {
        meta[i] = L.kofs[i];
        meta[kMaxKb + i] = L.left[i];
    }
    RELNN_CUDA(cudaMemcpyAsync(d_meta, meta, sizeof(meta), cudaMemcpyHostToDevice, st));
    CUtensorMap wmap;
    {
        cuuint64_t gdim[2] = {(cuuint64_t)L.n_kb * 64, (cuuint64_t)rows_pad};
        cuuint64_t gstride[1] = {(cuuint64_t)L.n_kb * 64 * 2};
        cuuint32_t box[2] = {64, 128};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p.wpack.p, gdim, gstride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
            return RELNN_ECUDA;
        }
    }
    static bool attr_set = false;
    if (!attr_set) {
        RELNN_CUDA(cudaFuncSetAttribute(fwd_tc_kernel<false, kAggSum>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        RELNN_CUDA(cudaFuncSetAttribute(fwd_tc_kernel<true, kAggSum>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        RELNN_CUDA(cudaFuncSetAttribute(fwd_tc_kernel<false, kAggDense>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        RELNN_CUDA(cudaFuncSetAttribute(fwd_tc_kernel<true, kAggDense>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        RELNN_CUDA(cudaFuncSetAttribute(fwd_tc_kernel<false, kAggMax>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        RELNN_CUDA(cudaFuncSetAttribute(fwd_tc_kernel<true, kAggMax>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        attr_set = true;
    }
    const bool maxagg = (p.flags & RELNN_FLAG_MAX) != 0;
    // MAX: the backward routes dOut through the recorded argmax instead of a ReLU mask
    const bool want_mask = p.act == RELNN_ACT_RELU && (p.flags & RELNN_FLAG_RELU_MASK) && !maxagg;
    if (maxagg) {
        RELNN_CHECK_ARG(!multi, "MAX aggregator: single-branch rules only");
        RELNN_TRY(p.carry_pos.alloc_nosync(sizeof(int32_t) * 2 * p.d_out * max_units, st));
        RELNN_TRY(p.max_arg.alloc_nosync(sizeof(int32_t) * (size_t)p.n_out * p.d_out, st));
    }
    const int mask_words = m_blocks * 4;
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        if (b.m == 0) continue;
        { pack_w_kernel<<<64, 256, 0, st>>>(io.br[i].W, io.w_bf16, p.d_out, p.d_in, rows_pad, rows_pad / rep, L.n_kb, d_meta,
                                          d_meta + kMaxKb, p.wpack.as<uint16_t>()); note_launch(); }
        RELNN_CUDA(cudaGetLastError());
        TcArgs a{};
        a.z = io.z;
        a.r = io.br[i].r;
        a.r_bf16 = io.r_bf16;
        a.hs = b.hs.as<int32_t>();
        a.hd = b.hd.as<int32_t>();
        a.er = b.er.as<int32_t>();
        a.seg = b.seg.as<int32_t>();
        a.bias = io.br[i].b;
        a.out = out;
        a.carry = p.carry.as<float>();
        if (maxagg) {
            a.carry_pos = p.carry_pos.as<int32_t>();
            a.arg = p.max_arg.as<int32_t>();
        }
        a.status = p.status.as<int>();
        if (want_mask) {
            RELNN_TRY(b.relu_mask.alloc_nosync(sizeof(uint32_t) * (size_t)b.m * mask_words, st));
            a.relu_mask = b.relu_mask.as<uint32_t>();
        }
        a.mask_words = mask_words;
        a.m = b.m;
        a.n_tiles = ceil_div(b.m, tile_n);
        a.z_rows = p.n_h;
        a.r_rows = b.n_tuples;
        a.z_bf16 = io.z_bf16;
        a.d = p.d;
        a.d_r = b.d_r;
        a.d_out = p.d_out;
        a.act = p.act;
        a.kahan = p.kahan;
        a.accumulate = multi;
        a.n_kb = L.n_kb;
        a.tile_n = tile_n;
        a.m_blocks = m_blocks;
        a.rep = rep;
        a.stages = stages;
        a.idesc = tc::idesc_bf16_f32(128, tile_n);
        a.tmem_cols = (uint32_t)(2 * m_blocks * tile_n) <= 256 ? 256u : 512u;
        a.need_arr[0] = a.need_arr[1] = a.need_arr[2] = 0;
        for (int k = 0; k < L.n_kb; ++k) {
            a.need_arr[L.src[k]] = 1;
            a.kb_src[k] = L.src[k];
            a.kb_col[k] = L.col[k];
            a.kb_width[k] = L.width[k];
        }
        const int grid = (int)std::min<int64_t>(a.n_tiles, num_sms());
        // every Concat part a single K block: indices staged transposed (see kIdxPitch)
        const bool idx_t = p.d <= 64 && b.d_r <= 64;
        {
            ProfToken pt = prof_begin(RELNN_PROF_FWD_TC, st);
            const bool dense = (p.flags & kPlanDense) != 0;
            if (dense) {
                if (idx_t) fwd_tc_kernel<true, kAggDense><<<grid, kThreads, smem, st>>>(wmap, a);
                else fwd_tc_kernel<false, kAggDense><<<grid, kThreads, smem, st>>>(wmap, a);
            } else if (maxagg) {
                if (idx_t) fwd_tc_kernel<true, kAggMax><<<grid, kThreads, smem, st>>>(wmap, a);
                else fwd_tc_kernel<false, kAggMax><<<grid, kThreads, smem, st>>>(wmap, a);
            } else {
                if (idx_t) fwd_tc_kernel<true, kAggSum><<<grid, kThreads, smem, st>>>(wmap, a);
                else fwd_tc_kernel<false, kAggSum><<<grid, kThreads, smem, st>>>(wmap, a);
            }
            note_launch();
            prof_end(pt, st);
        }
        RELNN_CUDA(cudaGetLastError());
        if (maxagg)
            RELNN_TRY(launch_fixup_max(a.seg, a.m, unit, ceil_div(a.m, unit), a.carry, a.carry_pos, out, a.arg, p.d_out,
                                       p.act == RELNN_ACT_RELU, p.fixjobs, st));
        else if (!(p.flags & kPlanDense))
            RELNN_TRY(launch_fixup(a.seg, a.m, unit, ceil_div(a.m, unit), a.carry, out, p.d_out, multi, p.kahan, p.fixjobs, st));
        RELNN_CUDA(cudaGetLastError());
    }
    return RELNN_OK;
}

}  // namespace relnn
