// Backward of the BF16 form on tcgen05 tensor cores (sm_103a), one persistent kernel per branch.
//
// For the dst-sorted matched tuples of a branch, with dY_t = dOut[seg_t] (masked by the ReLU mask
// the forward stored), the kernel computes per tile of N tuples
//   GEMM A (dX):  D2[k][t] = sum_o W^T[k][o] dY[t][o]   M = input feature k (128-row blocks of W^T,
//                 staged once by TMA), N = tuples, K = output features; both operands K-major.
//   GEMM B (dW):  D1[o][k] += sum_t dY[t][o] X[t][k]    M = output features, N = input features,
//                 K = tuples; both operands read MN-major from the same staged dY and X tiles.
// The gathered Concat X is regathered (not stored by the forward). The epilogue reads D2 (TMEM lane =
// input feature, columns = tuples) and adds dX into dz / dr. D1 accumulates over all tiles of the
// CTA; each CTA writes its partial dW and a reduction kernel adds them in CTA order.
//
// Two passes, so that dz receives one add per run of equal H rows rather than one per tuple:
//   dst pass (tuples in output order, as the forward): the dst slice of dX, added once per run of
//     equal dst rows (a segmented sum in registers), r per tuple, dW and db;
//   src pass (the same tuples sorted by src H row, an order the plan caches): only GEMM A, and the
//     src slice of dX added once per run of equal src rows.
//
// Roles (416 threads, one CTA per SM): warps 0-7 producers (dY: dOut rows -> mask -> bf16; X: rows
// of z / r as in the forward; db partial sums), warp 8 TMEM allocation + MMA issue, warps 9-12
// epilogue. 13 warps leave at most 128 registers per thread (four warps share one SM sub-partition).
#include <algorithm>
#include <mutex>

#include "agg.cuh"
#include "bwd.cuh"
#include "segscan.cuh"
#include "tc.cuh"

namespace relnn {

namespace {

using namespace tc;

constexpr int kThreads = 416;
constexpr int kProducerThreads = 256;
constexpr int kMmaWarp = 8;
constexpr int kMaxKb = 4;  // input-feature K blocks (d_in <= 256)
constexpr int kMaxMbk = 2; // GEMM A row blocks of 128 (d_in <= 256)
constexpr int kSmemLimit = 227 * 1024;

struct BwArgs {
    const void* z;
    const void* r;
    const float* dout;
    const uint16_t* dout_bf;  // bf16 copy of dout (src pass), or nullptr
    const uint32_t* mask;   // [m][mask_words] or nullptr (no ReLU)
    const int32_t* hs;
    const int32_t* hd;
    const int32_t* er;
    const int32_t* seg;
    float* dz;
    float* dr;
    float* db_part;         // [grid][d_out]: this CTA's db partial (summed in a fixed order)
    float* dw_part;         // [grid][d_out][d_in]
    const int* row_src;     // input feature of each padded K row (-1 = padding), [mbk * 128]
    int* status;
    int64_t m, n_tiles;
    int z_bf16, r_bf16, d, d_r, d_in, d_out, concat_dst, mask_words;
    int n_kb, d_in_pad, mbk, tile_n, stages;
    int x_blocks;           // K blocks of X staged per tile (n_kb in the dst pass, 0 in the src pass)
    int dy_blocks;          // blocks of 64 outputs in dY (d_out <= 64: 1; GEMM B then computes dW rows
                            // 64-127 from whatever follows the dY block and they are never read)
    int src_pass;           // 1: tuples in src order; hd then holds each tuple's row in output order
                            // (its ReLU mask row), hs the src H rows (non-decreasing), seg their output rows
    uint32_t idesc_dx, idesc_dw, tmem_cols, d2_col;
    int kb_src[kMaxKb], kb_col[kMaxKb], kb_width[kMaxKb];
    // GEMM A rows of this pass: TMEM lane quarter i (block i / 4) holds Concat part qpart[i] (0 z_src,
    // 1 z_dst, 2 r, -1 none) from column qcol0[i]; with rep > 1 the quarters repeat rep times and
    // the warps of equal rows share the tile's columns
    int qpart[4 * kMaxMbk], qcol0[4 * kMaxMbk];
    int rep;
    int need_arr[3];
};

// dY rows of one producer thread (rows row_base .. row_base + rpt - 1, 16-byte chunk `chunk` of each
// 64-output block): dOut[seg_t] masked by the ReLU mask of tuple t, rounded to bf16 into the
// 128B-swizzled dY blocks, and added to the thread's db partial. RB rows' loads are issued before
// any is used; OB = blocks of 64 outputs.
// The staged entries of rows row_base .. row_base + rpt - 1 (rpt = 2 or 4) with one shared load.
__device__ __forceinline__ void load_rows(const int32_t* p, int rpt, int32_t (&o)[4]) {
    if (rpt == 4) {
        const int4 v = *reinterpret_cast<const int4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        const int2 v = *reinterpret_cast<const int2*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = 0; o[3] = 0;
    }
}

template <int RB, int OB>
__device__ __forceinline__ void build_dy(const BwArgs& a, const int32_t* islot, int N, int64_t t0, int row_base,
                                         int rpt, int chunk, uint32_t dyb, float (&dbacc)[2][8]) {
    int32_t sgv[4], mrv[4];
    load_rows(islot + 3 * N + row_base, rpt, sgv);
    if (a.src_pass) load_rows(islot + N + row_base, rpt, mrv);
#pragma unroll
    for (int j0 = 0; j0 < 4; j0 += RB) {
        if (j0 >= rpt) break;
        float4 u[RB][OB][2];
        uint32_t bits[RB][OB];
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
            const int row = row_base + j0 + jj;
            const bool in = j0 + jj < rpt;
            const bool tv = in && (t0 + row < a.m);
            const int sg = tv ? sgv[j0 + jj] : 0;
            const int64_t mrow = a.src_pass ? (int64_t)(in ? mrv[j0 + jj] : 0) : t0 + row;
#pragma unroll
            for (int ob = 0; ob < OB; ++ob) {
                const int o0 = ob * 64 + chunk * 8;
                const bool ld = tv && o0 < a.d_out;
                const float4* q = reinterpret_cast<const float4*>(a.dout + (int64_t)sg * a.d_out + o0);
                u[jj][ob][0] = ld ? __ldg(q) : make_float4(0.f, 0.f, 0.f, 0.f);
                u[jj][ob][1] = ld ? __ldg(q + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
                bits[jj][ob] = (ld && a.mask) ? __ldg(a.mask + mrow * a.mask_words + (o0 >> 5)) >> (o0 & 31)
                                              : 0xffffffffu;
            }
        }
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
            if (j0 + jj >= rpt) break;
            const int row = row_base + j0 + jj;
#pragma unroll
            for (int ob = 0; ob < OB; ++ob) {
                float v[8] = {u[jj][ob][0].x, u[jj][ob][0].y, u[jj][ob][0].z, u[jj][ob][0].w,
                              u[jj][ob][1].x, u[jj][ob][1].y, u[jj][ob][1].z, u[jj][ob][1].w};
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    v[k] = ((bits[jj][ob] >> k) & 1u) ? v[k] : 0.f;
                    dbacc[ob][k] += v[k];
                }
                const uint32_t dst = dyb + (uint32_t)ob * N * 128u + (uint32_t)row * 128u +
                                     ((uint32_t)(chunk ^ (row & 7)) << 4);
                st_shared_v4(dst, pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                             pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
            }
        }
    }
}

// The same dY rows from the bf16 copy of dOut (the rounding dY gets anyway; no db partial): one
// 16-byte load per row and block, the ReLU mask applied to the packed pairs.
template <int RB, int OB>
__device__ __forceinline__ void build_dy_bf(const BwArgs& a, const int32_t* islot, int N, int64_t t0, int row_base,
                                            int rpt, int chunk, uint32_t dyb) {
    int32_t sgv[4], mrv[4];
    load_rows(islot + 3 * N + row_base, rpt, sgv);
    if (a.src_pass) load_rows(islot + N + row_base, rpt, mrv);
#pragma unroll
    for (int j0 = 0; j0 < 4; j0 += RB) {
        if (j0 >= rpt) break;
        uint4 u[RB][OB];
        uint32_t bits[RB][OB];
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
            const int row = row_base + j0 + jj;
            const bool in = j0 + jj < rpt;
            const bool tv = in && (t0 + row < a.m);
            const int sg = tv ? sgv[j0 + jj] : 0;
            const int64_t mrow = a.src_pass ? (int64_t)(in ? mrv[j0 + jj] : 0) : t0 + row;
#pragma unroll
            for (int ob = 0; ob < OB; ++ob) {
                const int o0 = ob * 64 + chunk * 8;
                const bool ld = tv && o0 < a.d_out;
                u[jj][ob] = ld ? __ldg(reinterpret_cast<const uint4*>(a.dout_bf + (int64_t)sg * a.d_out + o0))
                               : make_uint4(0u, 0u, 0u, 0u);
                bits[jj][ob] = (ld && a.mask) ? __ldg(a.mask + mrow * a.mask_words + (o0 >> 5)) >> (o0 & 31)
                                              : 0xffffffffu;
            }
        }
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
            if (j0 + jj >= rpt) break;
            const int row = row_base + j0 + jj;
#pragma unroll
            for (int ob = 0; ob < OB; ++ob) {
                const uint32_t b = bits[jj][ob];
                auto keep = [&](int k) { return ((b >> k) & 1u ? 0x0000ffffu : 0u) | ((b >> (k + 1)) & 1u ? 0xffff0000u : 0u); };
                const uint32_t dst = dyb + (uint32_t)ob * N * 128u + (uint32_t)row * 128u +
                                     ((uint32_t)(chunk ^ (row & 7)) << 4);
                st_shared_v4(dst, u[jj][ob].x & keep(0), u[jj][ob].y & keep(2), u[jj][ob].z & keep(4),
                             u[jj][ob].w & keep(6));
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
bwd_tc_kernel(const __grid_constant__ CUtensorMap wtmap, const __grid_constant__ BwArgs a) {
    extern __shared__ uint8_t dyn_smem[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~(uintptr_t)1023);
    const int N = a.tile_n;
    const uint32_t wt_bytes = (uint32_t)(a.mbk * a.dy_blocks) * 16384u;   // W^T: mbk x dy_blocks of 128 x 64
    const uint32_t dy_bytes = (uint32_t)a.dy_blocks * N * 128u;             // dY: blocks of 64 outputs
    const uint32_t x_bytes = (uint32_t)a.x_blocks * (uint32_t)N * 128u; // X: x_blocks blocks of 64 inputs
    const uint32_t stage_bytes = dy_bytes + x_bytes;
    uint8_t* wt_smem = base;
    uint8_t* st_smem = base + wt_bytes;
    int32_t* idx_smem = reinterpret_cast<int32_t*>(st_smem + (size_t)a.stages * stage_bytes);  // 2 x 4 x N
    int32_t* epi_smem = idx_smem + 8 * N;                                                      // 4 warps x 3 x N
    float* db_smem = reinterpret_cast<float*>(epi_smem + 12 * N);  // producer warps x 128 outputs
    uint64_t* bars = reinterpret_cast<uint64_t*>(db_smem + (kProducerThreads / 32) * 128);
    uint64_t* full = bars;
    uint64_t* empty = bars + a.stages;
    uint64_t* tfull = bars + 2 * a.stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* wbar = tempty + 2;
    uint64_t* dwdone = wbar + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dwdone + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(smem_u32(&full[s]), 2 * kProducerThreads);  // a plain and a cp.async arrive per thread
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&tfull[i]), 1);
            mbar_init(smem_u32(&tempty[i]), 128);
        }
        mbar_init(smem_u32(wbar), 1);
        mbar_init(smem_u32(dwdone), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t d2_stride = (uint32_t)a.mbk * N;

    if (warp < kProducerThreads / 32) {
        // ------------------------------------------------------------------ producers
        // thread = (row group of rpt consecutive rows, 16-byte chunk); the tile's hs / hd / er / seg
        // entries (4N) are staged in shared memory one tile ahead, at most 2 per thread
        const int chunk = tid & 7;
        const int rpt = N / (kProducerThreads / 8);
        const int row_base = (tid >> 3) * rpt;
        auto idx_load = [&](int64_t tile, int k) -> int32_t {
            const int e = tid + k * kProducerThreads;
            const int r = e / N, qq = e - r * N;
            const int64_t t = tile * N + qq;
            if (e >= 4 * N || (r < 3 && !a.need_arr[r]) || tile >= a.n_tiles || t >= a.m) return 0;
            const int32_t* arr = r == 0 ? a.hs : (r == 1 ? a.hd : (r == 2 ? a.er : a.seg));
            return __ldg(arr + t);
        };
        auto idx_store = [&](int32_t* slot, int k, int32_t v) {
            const int e = tid + k * kProducerThreads;
            if (e < 4 * N) slot[e] = v;
        };
        idx_store(idx_smem, 0, idx_load(blockIdx.x, 0));
        idx_store(idx_smem, 1, idx_load(blockIdx.x, 1));
        named_bar_sync(1, kProducerThreads);
        float dbacc[2][8];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < 8; ++k) dbacc[i][k] = 0.f;
        int it = 0, lt = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++lt) {
            const int64_t t0 = tile * N;
            const int32_t* islot = idx_smem + (lt & 1) * 4 * N;
            // the next tile's indices, stored after this tile's copies are issued
            const int32_t nxt0 = idx_load(tile + gridDim.x, 0), nxt1 = idx_load(tile + gridDim.x, 1);
            if (ok) {
                const int s = it % a.stages;
                const uint32_t ph = (uint32_t)((it / a.stages) & 1);
                if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, a.status, abort_flag)) ok = false;
                if (ok) {
                    uint8_t* stg = st_smem + (size_t)s * stage_bytes;
                    const uint32_t dyb = smem_u32(stg);
                    const uint32_t xb = smem_u32(stg + dy_bytes);
                    // dY rows: dOut[seg_t] masked by the stored ReLU mask, as bf16, in blocks of 64
                    // outputs; up to 4 rows' loads in flight before any is used
                    if (a.dout_bf) {
                        if (a.dy_blocks == 1) build_dy_bf<4, 1>(a, islot, N, t0, row_base, rpt, chunk, dyb);
                        else build_dy_bf<4, 2>(a, islot, N, t0, row_base, rpt, chunk, dyb);
                    } else if (a.dy_blocks == 1) {
                        build_dy<4, 1>(a, islot, N, t0, row_base, rpt, chunk, dyb, dbacc);
                    } else {
                        build_dy<2, 2>(a, islot, N, t0, row_base, rpt, chunk, dyb, dbacc);
                    }
                    // X rows, K-block by K-block (as in the forward); the src pass needs no dW. The
                    // rows' indices are loaded once per Concat part.
                    int32_t rix[4];
                    int rix_src = -1;
                    for (int kb = 0; kb < a.x_blocks; ++kb) {
                        const int src = a.kb_src[kb];
                        const int col = a.kb_col[kb] + chunk * 8;
                        const bool in_part = col < a.kb_width[kb];
                        if (src != rix_src) {
                            load_rows(islot + src * N + row_base, rpt, rix);
                            rix_src = src;
                        }
                        const void* tbl = src == 2 ? a.r : a.z;
                        const int tbl_bf16 = src == 2 ? a.r_bf16 : a.z_bf16;
                        const int row_elems = src == 2 ? a.d_r : a.d;
                        const uint32_t kbase = xb + (uint32_t)kb * N * 128u;
                        if (tbl_bf16) {
                            const uint16_t* p = reinterpret_cast<const uint16_t*>(tbl);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                if (j >= rpt) break;
                                const int row = row_base + j;
                                const uint32_t dst = kbase + (uint32_t)row * 128u + ((uint32_t)(chunk ^ (row & 7)) << 4);
                                const bool valid = (t0 + row < a.m) && in_part;
                                const int64_t ridx = rix[j];
                                cp_async_16(dst, valid ? p + ridx * row_elems + col : p, valid ? 16u : 0u);
                            }
                        } else {
                            // f32 rows: all (up to 4) rows' loads in flight before the convert-and-store
                            float4 u[4], w[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int row = row_base + j;
                                const bool valid = j < rpt && (t0 + row < a.m) && in_part;
                                const int64_t ridx = valid ? rix[j] : 0;
                                const float4* q = reinterpret_cast<const float4*>(
                                    reinterpret_cast<const float*>(tbl) + ridx * row_elems + col);
                                u[j] = valid ? __ldg(q) : make_float4(0.f, 0.f, 0.f, 0.f);
                                w[j] = valid ? __ldg(q + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
                            }
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                if (j >= rpt) break;
                                const int row = row_base + j;
                                const uint32_t dst = kbase + (uint32_t)row * 128u + ((uint32_t)(chunk ^ (row & 7)) << 4);
                                st_shared_v4(dst, pack_bf16x2(u[j].x, u[j].y), pack_bf16x2(u[j].z, u[j].w),
                                             pack_bf16x2(w[j].x, w[j].y), pack_bf16x2(w[j].z, w[j].w));
                            }
                        }
                    }
                    // dY and converted f32 rows were stored by this thread: publish them now; the
                    // cp.async rows arrive on their own once they have landed (no waiting here)
                    fence_proxy_async();
                    mbar_arrive(smem_u32(&full[s]));
                    cp_async_mbar_arrive_noinc(smem_u32(&full[s]));
                    ++it;
                }
            }
            // indices of this CTA's next tile into the other slot
            idx_store(idx_smem + ((lt + 1) & 1) * 4 * N, 0, nxt0);
            idx_store(idx_smem + ((lt + 1) & 1) * 4 * N, 1, nxt1);
            named_bar_sync(1, kProducerThreads);
        }
        // no copy may still be writing shared memory when the CTA retires
        cp_async_wait<0>();
        // db: this CTA's partial, summed in a fixed order (lanes of equal chunk, then warps)
        if (a.db_part) {
#pragma unroll
            for (int ob = 0; ob < 2; ++ob)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    float v = ob < a.dy_blocks ? dbacc[ob][k] : 0.f;
                    v += __shfl_xor_sync(0xffffffffu, v, 8);
                    v += __shfl_xor_sync(0xffffffffu, v, 16);
                    if (lane < 8) db_smem[warp * 128 + ob * 64 + chunk * 8 + k] = v;
                }
            named_bar_sync(1, kProducerThreads);
            for (int o = tid; o < a.d_out; o += kProducerThreads) {
                float v = 0.f;
                for (int w = 0; w < kProducerThreads / 32; ++w) v += db_smem[w * 128 + o];
                a.db_part[(int64_t)blockIdx.x * a.d_out + o] = v;
            }
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t wb = smem_u32(wbar);
            mbar_arrive_expect_tx(wb, wt_bytes);
            for (int mb = 0; mb < a.mbk; ++mb)
                for (int kk = 0; kk < a.dy_blocks; ++kk)
                    tma_load_2d(smem_u32(wt_smem + (size_t)(mb * a.dy_blocks + kk) * 16384u), &wtmap, kk * 64, mb * 128, wb);
            bool ok = mbar_wait(wb, 0, a.status, abort_flag);
            tc_fence_after();
            int lt = 0;
            for (int64_t tile = blockIdx.x; tile < a.n_tiles && ok; tile += gridDim.x, ++lt) {
                const int s = lt % a.stages;
                const uint32_t ph = (uint32_t)((lt / a.stages) & 1);
                const int acc = lt & 1;
                const uint32_t use = (uint32_t)(lt >> 1);
                if (!mbar_wait(smem_u32(&full[s]), ph, a.status, abort_flag)) { ok = false; break; }
                if (!mbar_wait(smem_u32(&tempty[acc]), (use & 1u) ^ 1u, a.status, abort_flag)) { ok = false; break; }
                fence_proxy_async();  // cp.async rows of the stage, before the tensor core reads them
                tc_fence_after();
                const uint32_t dyb = smem_u32(st_smem + (size_t)s * stage_bytes);
                const uint32_t xb = dyb + dy_bytes;
                // GEMM A: dX^T for this tile
                const uint32_t d2 = tmem_base + a.d2_col + (uint32_t)acc * d2_stride;
                for (int mb = 0; mb < a.mbk; ++mb)
                    for (int kk = 0; kk < a.dy_blocks; ++kk)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint64_t ad = sw128_kmajor_desc(smem_u32(wt_smem + (size_t)(mb * a.dy_blocks + kk) * 16384u) + k * 32);
                            const uint64_t bd = sw128_kmajor_desc(dyb + (uint32_t)kk * N * 128u + k * 32);
                            mma_bf16(d2 + (uint32_t)mb * N, ad, bd, a.idesc_dx, (kk | k) != 0);
                        }
                mma_commit(smem_u32(&tfull[acc]));
                // GEMM B: dW += dY^T X, 16 tuples per instruction (dst pass only)
                for (int step = 0; step < (a.src_pass ? 0 : N / 16); ++step) {
                    const uint64_t ad = sw128_mnmajor_desc(dyb + (uint32_t)step * 2048u, (uint32_t)N * 128u);
                    const uint64_t bd = sw128_mnmajor_desc(xb + (uint32_t)step * 2048u, (uint32_t)N * 128u);
                    mma_bf16(tmem_base, ad, bd, a.idesc_dw, (lt > 0 || step > 0) ? 1u : 0u);
                }
                mma_commit(smem_u32(&empty[s]));
            }
            mma_commit(smem_u32(dwdone));
            // every issued MMA must finish before TMEM is released (also when another role aborted)
            mbar_wait(smem_u32(dwdone), 0, a.status, abort_flag);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------ epilogue
        const int q = warp & 3;
        const int span = N / a.rep;                     // columns of each tile this warp reduces
        const int c0 = (q / (4 / a.rep)) * span;        // the first of them
        int32_t* wix = epi_smem + (warp - kMmaWarp - 1) * 3 * N;  // hs, hd, er of those columns
        int lt = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++lt) {
            const int64_t t0 = tile * N + c0;
            const int ntl = (int)imin64(span, a.m - t0);  // <= 0: nothing in this warp's columns
            __syncwarp();
            for (int rr = lane; rr < span; rr += 32) {
                const bool v = rr < ntl;
                wix[rr] = v ? __ldg(a.hs + t0 + rr) : 0;
                wix[N + rr] = (v && a.concat_dst && !a.src_pass) ? __ldg(a.hd + t0 + rr) : -1;
                wix[2 * N + rr] = (v && a.dr) ? __ldg(a.er + t0 + rr) : 0;
            }
            __syncwarp();
            const int acc = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[acc]), use & 1u, a.status, abort_flag))) {
                ok = false;
                break;
            }
            tc_fence_after();
            for (int mb = 0; mb < a.mbk; ++mb) {
                const int part = a.qpart[mb * 4 + q];  // warp-uniform
                if (part < 0) continue;
                const int kk = a.qcol0[mb * 4 + q] + lane;  // this lane's column of the part
                const bool k_ok = kk < (part == 2 ? a.d_r : a.d);
                const uint32_t taddr = tmem_base + ((uint32_t)(32 * q) << 16) + a.d2_col + (uint32_t)acc * d2_stride +
                                       (uint32_t)(mb * N + c0);
                for (int c = 0; c * 32 < ntl; ++c) {
                    uint32_t v[32];
                    tmem_ld_32x32b_x32(taddr + (uint32_t)c * 32, v);
                    tmem_ld_wait();
                    const int cnt = min(32, ntl - c * 32);
                    if (part != 2) {
                        // runs of equal dst (dst pass) or src (src pass) H rows inside the chunk (the
                        // tuples are sorted by it): a segmented running sum in registers, then one
                        // add per run end
                        const int32_t* keyv = (part == 1 ? wix + N : wix) + c * 32;
                        const int h = keyv[lane];
                        const bool tvalid = lane < cnt;
                        const bool nx_diff = (lane == cnt - 1) || (lane + 1 < cnt && keyv[lane + 1] != h);
                        const unsigned endmask = __ballot_sync(0xffffffffu, tvalid && nx_diff);
                        const unsigned startmask = (endmask << 1) | 1u;
                        float sum = 0.f, comp = 0.f;
                        uint32_t mword = 0;
                        seg_scan<false, false, false>(v, 0.f, startmask, sum, comp, mword, lane);
                        float* dzc = a.dz + kk;
                        // one add per run end, four ends at a time (independent selects and adds)
                        for (unsigned em = endmask; em;) {
                            int jj[4];
#pragma unroll
                            for (int g = 0; g < 4; ++g) {
                                jj[g] = em ? __ffs(em) - 1 : -1;
                                em &= em - 1u;
                            }
#pragma unroll
                            for (int g = 0; g < 4; ++g) {
                                const uint32_t val = select32(v, jj[g] & 31);
                                const int hj = keyv[jj[g] & 31];
                                if (jj[g] >= 0 && k_ok) atomicAdd(dzc + (int64_t)hj * a.d, __uint_as_float(val));
                            }
                        }
                    } else {
                        const int32_t* erv = wix + 2 * N + c * 32;
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < cnt && k_ok)
                                atomicAdd(a.dr + (int64_t)erv[j] * a.d_r + kk, __uint_as_float(v[j]));
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&tempty[acc]));
        }
        // this CTA's dW partial: TMEM lane o (output feature), columns k (input features)
        if (ok && a.dw_part && __all_sync(0xffffffffu, mbar_wait(smem_u32(dwdone), 0, a.status, abort_flag))) {
            tc_fence_after();
            const int o = 32 * q + lane;
            float* dst = a.dw_part + ((int64_t)blockIdx.x * a.d_out + o) * a.d_in;
            for (int c = 0; c * 32 < a.d_in_pad; ++c) {
                uint32_t v[32];
                tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)c * 32, v);
                tmem_ld_wait();
                if (o < a.d_out) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int k = a.row_src[c * 32 + j];  // padded column -> input feature
                        if (k >= 0) dst[k] = __uint_as_float(v[j]);
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem_base, a.tmem_cols);
    }
}

// W^T padded to [mbk*128 rows (input features)][128 cols (output features)] in bf16.
__global__ void pack_wt_kernel(const void* W, int w_bf16, int d_out, int d_in, int rows_pad, const int* row_src,
                               uint16_t* wt) {
    const int n = rows_pad * 128;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int kr = i >> 7, o = i & 127;
        const int k = row_src[kr];  // input feature of padded row kr, or -1
        uint16_t v = 0;
        if (k >= 0 && o < d_out) {
            if (w_bf16) v = reinterpret_cast<const uint16_t*>(W)[o * d_in + k];
            else v = __bfloat16_as_ushort(__float2bfloat16_rn(reinterpret_cast<const float*>(W)[o * d_in + k]));
        }
        wt[i] = v;
    }
}

// out[i] = sum over parts of part[c][i], compensated, in part order (deterministic).
__global__ void reduce_parts_kahan_kernel(const float* part, int nparts, int64_t n, float* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float sum = 0.f, c = 0.f;
        for (int p = 0; p < nparts; ++p) kahan_add(sum, c, part[(int64_t)p * n + i]);
        out[i] = sum;
    }
}

__global__ void reduce_parts_kernel(const float* part, int nparts, int64_t n, float* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * n + i];
        out[i] = s;
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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

// Whether the tensor-core backward covers this plan (else the FP32-form backward runs).
static bool tc_backward_supported(const Plan& p) {
    if (p.identity || p.d_out > 128 || p.d_out % 8 || p.d % 8 || p.br[0].d_r % 8) return false;
    int kb = 0;
    kb += (p.d + 63) / 64;
    if (p.concat_dst) kb += (p.d + 63) / 64;
    if (p.br[0].d_r) kb += (p.br[0].d_r + 63) / 64;
    return kb <= kMaxKb;
}

relnn_status backward_tc(Plan& p, const CallIO& io_in, const GradIO& g, cudaStream_t st) {
    // linear SUM / MEAN rules: per-H-row sums of dOut, then dense GEMM rows (agg.cu)
    if (agg_backward_ok(p, io_in, g)) return backward_agg(p, io_in, g, st);
    if (!tc_backward_supported(p)) return backward_fp32(p, io_in, g, st);
    RELNN_CHECK_ARG(g.dout, "backward: null output gradient");
    const bool relu = p.act == RELNN_ACT_RELU;
    // K-block layout of the Concat (each part starts on a 64-column block)
    int n_kb = 0, kb_src[kMaxKb], kb_col[kMaxKb], kb_width[kMaxKb];
    std::vector<int> row_src;  // input feature of each padded K row (-1 = padding)
    auto add_part = [&](int src, int width, int kofs) {
        for (int c = 0; c < width; c += 64) {
            kb_src[n_kb] = src;
            kb_col[n_kb] = c;
            kb_width[n_kb] = width;
            for (int i = 0; i < 64; ++i) row_src.push_back(c + i < width ? kofs + c + i : -1);
            ++n_kb;
        }
    };
    add_part(0, p.d, 0);
    if (p.concat_dst) add_part(1, p.d, p.d);
    if (p.br[0].d_r) add_part(2, p.br[0].d_r, p.d * (p.concat_dst ? 2 : 1));
    const int d_in_pad = n_kb * 64;
    const uint32_t d2_col = (uint32_t)((d_in_pad + 31) / 32 * 32);
    // GEMM A rows of each pass: the dst pass needs dX for the z_dst and r slices, the src pass for
    // the z_src slice. Each part fills whole 32-row lane quarters; one or two quarters are repeated
    // to fill the 128 lanes (so every epilogue warp has work).
    struct PassMap {
        std::vector<int> rows;  // input feature of each GEMM A row (-1 = padding), mbk * 128
        int mbk = 1, rep = 1;
        int qpart[4 * kMaxMbk], qcol0[4 * kMaxMbk];
    };
    auto make_map = [&](bool src_slice) {
        PassMap m;
        std::vector<std::pair<int, int>> qs;  // (part, first column) per quarter
        std::vector<int> rows;
        auto add = [&](int part, int width, int kofs) {
            for (int c = 0; c < width; c += 32) {
                qs.push_back({part, c});
                for (int i = 0; i < 32; ++i) rows.push_back(c + i < width ? kofs + c + i : -1);
            }
        };
        if (src_slice) add(0, p.d, 0);
        else {
            if (p.concat_dst) add(1, p.d, p.d);
            if (p.br[0].d_r) add(2, p.br[0].d_r, p.d * (p.concat_dst ? 2 : 1));
        }
        if (qs.empty()) {
            qs.push_back({-1, 0});
            rows.assign(32, -1);
        }
        const int nq = (int)qs.size();
        m.rep = nq == 1 ? 4 : (nq == 2 ? 2 : 1);
        const int per = m.rep > 1 ? 4 / m.rep : 4 * ((nq + 3) / 4);  // quarters of one copy
        while ((int)qs.size() < per) {
            qs.push_back({-1, 0});
            rows.insert(rows.end(), 32, -1);
        }
        for (int r = 1; r < m.rep; ++r)
            for (int i = 0; i < per; ++i) {
                qs.push_back(qs[i]);
                rows.insert(rows.end(), rows.begin() + 32 * i, rows.begin() + 32 * (i + 1));
            }
        m.mbk = (int)qs.size() / 4;
        for (int i = 0; i < 4 * kMaxMbk; ++i) {
            m.qpart[i] = i < (int)qs.size() ? qs[i].first : -1;
            m.qcol0[i] = i < (int)qs.size() ? qs[i].second : 0;
        }
        m.rows = rows;
        return m;
    };
    const PassMap dmap = make_map(false), smap = make_map(true);
    const int dy_blocks = (p.d_out + 63) / 64;
    // quarter table of a pass at the tile's replication (copies beyond it are switched off, so no
    // two warps reduce the same rows over the same columns)
    auto fill_quarters = [](BwArgs& a, const PassMap& pm, int rep) {
        for (int k = 0; k < 4 * kMaxMbk; ++k) {
            const bool on = (k % 4) % (4 / rep) < 4 / pm.rep;
            a.qpart[k] = on ? pm.qpart[k] : -1;
            a.qcol0[k] = pm.qcol0[k];
        }
        a.rep = rep;
    };
    if (dmap.mbk > kMaxMbk || smap.mbk > kMaxMbk) return backward_fp32(p, io_in, g, st);
    // Tile size per pass: 128 tuples when three stages and the TMEM columns fit, else 64. The src
    // pass stages only dY.
    struct PassCfg {
        int N = 0, stages = 0, rep = 1;
        uint32_t tmem_cols = 0, wt_bytes = 0;
        size_t smem = 0;
    };
    auto pass_cfg = [&](int x_blocks, const PassMap& pm) {
        PassCfg c;
        c.wt_bytes = (uint32_t)(pm.mbk * dy_blocks) * 16384u;
        auto stage_of = [&](int N) { return (uint32_t)dy_blocks * N * 128u + (uint32_t)x_blocks * N * 128u; };
        auto aux_of = [&](int N) { return (uint32_t)(20 * N * 4 + (kProducerThreads / 32) * 128 * 4); };
        auto stages_at = [&](int N) {
            return (int)((kSmemLimit - 1024 - 256 - (int)c.wt_bytes - (int)aux_of(N)) / (int)stage_of(N));
        };
        c.N = 128;
        c.stages = stages_at(128);
        if (c.stages < 3 || d2_col + 2u * pm.mbk * 128u > 512u) {
            c.N = 64;
            c.stages = stages_at(64);
        }
        c.stages = std::min(c.stages, 6);
        c.rep = std::min(pm.rep, c.N / 32);
        const uint32_t cols_needed = d2_col + 2u * pm.mbk * c.N;
        if (c.stages < 2 || cols_needed > 512) c.stages = 0;  // not runnable
        c.tmem_cols = cols_needed <= 256 ? 256u : 512u;
        c.smem = 1024 + c.wt_bytes + (size_t)c.stages * stage_of(c.N) + aux_of(c.N) + 256;
        return c;
    };
    const PassCfg dcfg = pass_cfg(n_kb, dmap), scfg = pass_cfg(0, smap);
    if (dcfg.stages == 0 || scfg.stages == 0) return backward_fp32(p, io_in, g, st);
    const int N = dcfg.N;

    // f32 z is gathered as a bf16 copy (the rounding the kernel applies anyway), by cp.async
    CallIO io;
    RELNN_TRY(with_bf16_z(p, io_in, io, st));
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return RELNN_ECUDA;
    }
    static bool attr_set = false;
    if (!attr_set) {
        RELNN_CUDA(cudaFuncSetAttribute(bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        attr_set = true;
    }
    if (g.dz && !g.accumulate_dz) RELNN_CUDA(cudaMemsetAsync(g.dz, 0, sizeof(float) * p.n_h * p.d, st));
    // the src pass gathers dOut rows in H-row order: from a bf16 copy (half the bytes, the rounding
    // dY gets anyway)
    const uint16_t* dout_bf = nullptr;
    if (g.dz && (reinterpret_cast<uintptr_t>(g.dout) & 15u) == 0 && p.n_out > 0) {
        RELNN_TRY(p.doutbf.alloc_nosync(sizeof(uint16_t) * (size_t)p.n_out * p.d_out, st));
        f32_to_bf16(g.dout, p.n_out * (int64_t)p.d_out, p.doutbf.as<uint16_t>(), st);
        RELNN_CUDA(cudaGetLastError());
        dout_bf = p.doutbf.as<uint16_t>();
    }
    const int grid_max = num_sms();
    const size_t wt_d_elems = (size_t)dmap.mbk * 128 * 128, wt_s_elems = (size_t)smap.mbk * 128 * 128;
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        float* dW = g.dW.size() > i ? g.dW[i] : nullptr;
        float* db = g.db.size() > i ? g.db[i] : nullptr;
        float* dr = (g.dr.size() > i && b.d_r > 0) ? g.dr[i] : nullptr;
        if (dr) RELNN_CUDA(cudaMemsetAsync(dr, 0, sizeof(float) * b.n_tuples * b.d_r, st));
        if (db) RELNN_CUDA(cudaMemsetAsync(db, 0, sizeof(float) * p.d_out, st));
        if (b.m == 0) {
            if (dW) RELNN_CUDA(cudaMemsetAsync(dW, 0, sizeof(float) * p.d_out * p.d_in, st));
            continue;
        }
        // MAX: the winner mask (argmax and ReLU' in one) replaces the ReLU mask
        const bool maxagg = (p.flags & RELNN_FLAG_MAX) != 0;
        if (relu && !maxagg && !b.relu_mask.p) {
            set_error("BF16 backward with ReLU needs the forward's mask (plan flag RELNN_FLAG_RELU_MASK)");
            return RELNN_EINVAL;
        }
        const int64_t n_tiles = ceil_div(b.m, N);
        const int grid = (int)std::min<int64_t>(n_tiles, grid_max);
        // scratch: W^T row blocks of the two passes (bf16), their row maps, the X column map, and
        // the dW / db partials
        const size_t part_elems = (size_t)grid * p.d_out * p.d_in;
        const size_t dbp_elems = (size_t)grid * p.d_out;
        const size_t n_maps = dmap.rows.size() + smap.rows.size() + row_src.size();
        const size_t head = ((wt_d_elems + wt_s_elems) * 2 + sizeof(int) * n_maps + 255) & ~(size_t)255;
        RELNN_TRY(p.scratch.alloc_nosync(head + sizeof(float) * (part_elems + dbp_elems), st));
        uint16_t* wt_d = p.scratch.as<uint16_t>();
        uint16_t* wt_s = wt_d + wt_d_elems;
        int* d_maps = reinterpret_cast<int*>(wt_s + wt_s_elems);
        int* d_rows = d_maps + dmap.rows.size() + smap.rows.size();
        float* part = reinterpret_cast<float*>(p.scratch.as<uint8_t>() + head);
        float* db_part = part + part_elems;
        {
            std::vector<int> maps(dmap.rows);
            maps.insert(maps.end(), smap.rows.begin(), smap.rows.end());
            maps.insert(maps.end(), row_src.begin(), row_src.end());
            RELNN_CUDA(cudaMemcpyAsync(d_maps, maps.data(), sizeof(int) * maps.size(), cudaMemcpyHostToDevice, st));
        }
        { pack_wt_kernel<<<64, 256, 0, st>>>(io.br[i].W, io.w_bf16, p.d_out, p.d_in, dmap.mbk * 128, d_maps, wt_d); note_launch(); }
        if (g.dz) { pack_wt_kernel<<<64, 256, 0, st>>>(io.br[i].W, io.w_bf16, p.d_out, p.d_in, smap.mbk * 128,
                                                       d_maps + dmap.rows.size(), wt_s); note_launch(); }
        auto make_tmap = [&](CUtensorMap& m, uint16_t* wt, int mbk) -> relnn_status {
            cuuint64_t gdim[2] = {128, (cuuint64_t)mbk * 128};
            cuuint64_t gstride[1] = {128 * 2};
            cuuint32_t box[2] = {64, 128};
            cuuint32_t estr[2] = {1, 1};
            CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, wt, gdim, gstride, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                set_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
                return RELNN_ECUDA;
            }
            return RELNN_OK;
        };
        CUtensorMap wtmap_d, wtmap_s;
        RELNN_TRY(make_tmap(wtmap_d, wt_d, dmap.mbk));
        RELNN_TRY(make_tmap(wtmap_s, wt_s, smap.mbk));
        BwArgs a{};
        a.z = io.z;
        a.r = io.br[i].r;
        a.dout = g.dout;
        a.mask = maxagg ? p.win_mask.as<uint32_t>() : (relu ? b.relu_mask.as<uint32_t>() : nullptr);
        a.hs = b.hs.as<int32_t>();
        a.hd = b.hd.as<int32_t>();
        a.er = b.er.as<int32_t>();
        a.seg = b.seg.as<int32_t>();
        a.dz = g.dz;
        a.dr = dr;
        a.db_part = db ? db_part : nullptr;
        a.dw_part = part;
        a.row_src = d_rows;
        a.status = p.status.as<int>();
        a.m = b.m;
        a.n_tiles = n_tiles;
        a.z_bf16 = io.z_bf16;
        a.r_bf16 = io.r_bf16;
        a.d = p.d;
        a.d_r = b.d_r;
        a.d_in = p.d_in;
        a.d_out = p.d_out;
        a.concat_dst = p.concat_dst;
        a.mask_words = ((p.d_out + 127) / 128) * 4;
        a.n_kb = n_kb;
        a.d_in_pad = d_in_pad;
        a.mbk = dmap.mbk;
        fill_quarters(a, dmap, dcfg.rep);
        a.tile_n = N;
        a.stages = dcfg.stages;
        a.x_blocks = n_kb;
        a.dy_blocks = dy_blocks;
        a.idesc_dx = tc::idesc_bf16_f32(128, N);
        a.idesc_dw = tc::idesc_bf16_f32(128, d_in_pad, true, true);
        a.tmem_cols = dcfg.tmem_cols;
        a.d2_col = d2_col;
        a.need_arr[0] = a.need_arr[1] = a.need_arr[2] = 0;
        for (int k = 0; k < n_kb; ++k) {
            a.kb_src[k] = kb_src[k];
            a.kb_col[k] = kb_col[k];
            a.kb_width[k] = kb_width[k];
            a.need_arr[kb_src[k]] = 1;
        }
        { ProfToken pt = prof_begin(RELNN_PROF_BWD_TC, st); bwd_tc_kernel<<<grid, kThreads, dcfg.smem, st>>>(wtmap_d, a); note_launch(); prof_end(pt, st); }
        RELNN_CUDA(cudaGetLastError());
        if (g.dz) {
            // src pass: the src slice of dX over the tuples in src order, one add per run
            RELNN_TRY(ensure_src_order(p, b, st));
            BwArgs s2 = a;
            s2.src_pass = 1;
            s2.x_blocks = 0;
            s2.tile_n = scfg.N;
            s2.stages = scfg.stages;
            s2.mbk = smap.mbk;
            fill_quarters(s2, smap, scfg.rep);
            s2.n_tiles = ceil_div(b.m, scfg.N);
            s2.idesc_dx = tc::idesc_bf16_f32(128, scfg.N);
            s2.tmem_cols = scfg.tmem_cols;
            const int sgrid = (int)std::min<int64_t>(s2.n_tiles, grid_max);
            s2.hs = b.hs_src.as<int32_t>();
            s2.hd = b.src_perm.as<int32_t>();
            s2.seg = b.seg_src.as<int32_t>();
            s2.dr = nullptr;
            s2.db_part = nullptr;
            s2.dout_bf = dout_bf;
            s2.dw_part = nullptr;
            s2.need_arr[0] = 1;
            s2.need_arr[1] = a.mask ? 1 : 0;  // each tuple's mask row (its position in output order)
            s2.need_arr[2] = 0;
            { ProfToken pt = prof_begin(RELNN_PROF_BWD_TC, st); bwd_tc_kernel<<<sgrid, kThreads, scfg.smem, st>>>(wtmap_s, s2); note_launch(); prof_end(pt, st); }
            RELNN_CUDA(cudaGetLastError());
        }
        if (dW) {
            const int64_t nw = (int64_t)p.d_out * p.d_in;
            { reduce_parts_kernel<<<(int)std::min<int64_t>(ceil_div(nw, 256), 1024), 256, 0, st>>>(part, grid, nw, dW); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
        }
        if (db) {
            { reduce_parts_kahan_kernel<<<1, 128, 0, st>>>(db_part, grid, p.d_out, db); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
        }
    }
    return RELNN_OK;
}

}  // namespace relnn
