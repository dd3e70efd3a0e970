// Aggregate-first evaluation of linear SUM rules on tcgen05 tensor cores (sm_103a).
//
// A join rule without an activation, H'(dst; SUM(W Concat(z_src, z_dst) + b)) (Sec. 3.1 join rule:
// T_tau with tau = Linear, then alpha = SUM over the tuples B_t of a key, Sec. 2.2), is linear in its
// Concat rows, so the SUM commutes with the transformation:
//     Out[k] = sum_{t in B_k} (W X_t + b) = W S[k] + n_k b,     S[k] = sum_{t in B_k} X_t,
// with S[k] = [sum z[hs_t] | sum z[hd_t]]. It is one of the hybrid content/embedding rewrites the
// paper lists as future work (Sec. 6: transformations applied once per node instead of once per
// edge): the tensor cores run once per output row instead of once per matched tuple, and the
// per-tuple work is a gather-sum of bf16 rows. The BF16 form's precision is kept: the f32 sums are
// split into a bf16 pair S = S_hi + S_lo (about 16 significant bits) and both halves are multiplied
// by the bf16 W with f32 accumulation.
//
// The same kernel evaluates the linear backward (the fit of Sec. 2.3; embeddings are parameters,
// Sec. 3.6). With dY_t = dOut[seg_t] (SUM broadcasts the row gradient to its tuples):
//     dz[h] = G_s[h] W_s + G_d[h] W_d,    G_s[h] = sum_{t: hs_t = h} dOut[seg_t]
//                                         G_d[h] = sum_{t: hd_t = h} dOut[seg_t]
//     dW_s = G_s^T Z,  dW_d = G_d^T Z,    db = sum_k n_k dOut[k]
// (W_s, W_d: the column blocks of W that multiply z_src and z_dst). A pass takes the tuples in src
// order (G_s; every H row, so dz is written once) or in dst order (G_d; runs of equal dst H rows,
// added): per H row a gather-sum of dOut rows and one GEMM row of dz; G^T Z is a second GEMM whose
// K dimension is the H rows, accumulated over all tiles of the CTA in TMEM. db is summed in f32 from
// the unrounded dOut by the pass that makes its bf16 copy.
//
// Virtual rows: the tuples of a destination row are cut into chunks of at most kChunk tuples (one
// virtual row each), which bounds a producer warp's unit of work; a row cut into several chunks
// leaves one partial per chunk, added in chunk order by the fix-up (two levels for rows with many
// chunks). Summation order: a chunk's tuples are summed in L-strided groups (fixed), the groups by a
// butterfly, the chunks in order: results are deterministic.
//
// Roles (512 threads, one CTA per SM, persistent over tiles of N virtual rows):
//   warps 0-6, 12-15  producers: take the tile's virtual rows one at a time from a shared counter,
//                     gather-sum the rows' Concat parts in f32, write S_hi / S_lo into 128B-swizzled
//                     K-major stages; in a backward pass also the row's z (B operand of G^T Z)
//   warp 7            TMEM allocation; lane 0 stages A (W, or a W^T block) once by TMA and issues
//                     tcgen05.mma: D[f][row] = sum_k A[f][k] S[row][k] over both halves
//   warps 8-11        epilogue (TMEM lane quarter = warp % 4): Out row = D + n b (or the chunk's
//                     partial); after the last tile of a backward pass, the CTA's dW and db partials
#include "agg.cuh"
#include "primitives.cuh"
#include "tc.cuh"

#include <algorithm>
#include <vector>

namespace relnn {

namespace {

using namespace tc;

constexpr int kThreads = 512;
constexpr int kMmaWarp = 7;
constexpr int kEpiWarp0 = 8;
constexpr int kEpiWarps = 4;
constexpr int kProdWarps = 11;                 // warps 0-6 and 12-15
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kMaxParts = 2;
constexpr int kMaxMeta = 4;                    // tile rows / 32 (N <= 128)
constexpr int kUnroll = 8;                     // row loads in flight per lane
constexpr int kChunk = 32;                     // tuples per virtual row (one index per lane)
constexpr int kMaxG = 8;                       // rows per warp in group mode (row width >= 4 chunks)
constexpr int kRound = 16;                     // tuples of a row loaded together (two rounds per row)
constexpr int kMaxZ = 2;                       // z-row chunks per lane loaded with the row (the rest after)
constexpr int kFixChunk = 256;                 // chunk partials one fix-up block adds
constexpr int kSmemLimit = 227 * 1024;

struct AggArgs {
    const int4* vr;                            // virtual rows {t0, n, row, part}
    int64_t nv, n_tiles;
    // Concat parts, in processing order: gather index per tuple, bf16 table, width, kind (0: a
    // different row per tuple; 1: few distinct rows per virtual row, summed as count x row), and
    // the part's first column in A's K dimension (a multiple of 64)
    const int32_t* gidx[kMaxParts];
    const uint16_t* tbl[kMaxParts];
    int64_t tbl_rows[kMaxParts];
    int width[kMaxParts], kind[kMaxParts], kofs[kMaxParts];
    int n_parts, n_kb, m_blocks, n_feat;
    const float* bias;                         // forward: + n * bias[f]
    float* out;                                // [rows][n_feat] (nullptr: no output rows)
    float* vpart;                              // [partials][n_feat]
    int accumulate, tile_n, stages;
    uint32_t idesc, tmem_cols;
    int* status;
    // backward pass: dW_part += G^T Z[row]
    const uint16_t* zrows;                     // bf16 [rows][d_z]
    int d_z, z_blocks, m_dw;
    float* dw_part;                            // [grid][n_g][d_z]
    int n_g;
    uint32_t idesc_dw, dw_col;
};

// a0 += low bf16 of w, a1 += high bf16 of w, by the mixed-precision add (sm_100+): the bf16 operand
// is widened inside the add, so no separate unpack; the widening is exact, so the sums equal the
// unpack-then-add.rn.f32 results
__device__ __forceinline__ void add_bf16x2(float& a0, float& a1, uint32_t w) {
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "add.rn.f32.bf16 %0, l, %0;\n\tadd.rn.f32.bf16 %1, h, %1;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "r"(w));
}

__device__ __forceinline__ void add8(float (&acc)[8], float (&cmp)[8], const uint4& u, bool kahan) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (kahan) {
            kahan_add(acc[2 * i], cmp[2 * i], __uint_as_float(w[i] << 16));
            kahan_add(acc[2 * i + 1], cmp[2 * i + 1], __uint_as_float(w[i] & 0xffff0000u));
        } else {
            add_bf16x2(acc[2 * i], acc[2 * i + 1], w[i]);
        }
    }
}

// Sum over the virtual row's tuples of table rows (bf16, `w` elements) for this lane's 16-byte
// chunk: `ix` holds lane j's tuple index (j < n). Returns the f32 sums of the chunk's 8 elements in
// every lane of the chunk (groups of w / 8 lanes share nothing but the final butterfly).
template <bool KAHAN>
__device__ __forceinline__ void part_sum(const uint16_t* __restrict__ tbl, int64_t rows, int* status, int w, int kind,
                                         int ix, int n, int lane, float (&acc)[8]) {
    const int L = w >> 3;  // lanes per table row (a power of two <= 32)
    const int G = 32 / L;  // tuples per warp step
    const int grp = lane / L, ch = lane - grp * L;
    const uint4* __restrict__ base = reinterpret_cast<const uint4*>(tbl) + ch;
    float cmp[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = cmp[i] = 0.f;
    if (kind == 0) {
        for (int j0 = 0; j0 < n; j0 += kUnroll * G) {
            uint4 u[kUnroll];
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                const int j = j0 + q * G + grp;
                const int r = __shfl_sync(0xffffffffu, ix, j & 31);
                u[q] = (j < n && in_bounds(r, rows, status)) ? __ldg(base + (int64_t)r * L) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) add8(acc, cmp, u[q], KAHAN);
        }
    } else {
        // distinct rows among the tuples, each loaded once and weighted by its multiplicity
        const bool valid = lane < n;
        unsigned rem = __ballot_sync(0xffffffffu, valid);
        while (rem) {
            const int r = __shfl_sync(0xffffffffu, ix, __ffs(rem) - 1);
            const unsigned mm = __ballot_sync(0xffffffffu, valid && ix == r);
            rem &= ~mm;
            if (grp == 0 && in_bounds(r, rows, status)) {
                const uint4 u = __ldg(base + (int64_t)r * L);
                const float c = (float)__popc(mm);
                const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    // c <= 32 times a bf16 value is exact in f32
                    const float lo = c * __uint_as_float(wd[i] << 16), hi = c * __uint_as_float(wd[i] & 0xffff0000u);
                    if (KAHAN) {
                        kahan_add(acc[2 * i], cmp[2 * i], lo);
                        kahan_add(acc[2 * i + 1], cmp[2 * i + 1], hi);
                    } else {
                        acc[2 * i] += lo;
                        acc[2 * i + 1] += hi;
                    }
                }
            }
        }
    }
    // groups of the warp: butterfly (each pairwise add is commutative, so every lane of a chunk
    // ends with the same value)
    for (int off = L; off < 32; off <<= 1) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (KAHAN) {
                const float s2 = __shfl_xor_sync(0xffffffffu, acc[i], off);
                const float c2 = __shfl_xor_sync(0xffffffffu, cmp[i], off);
                // (s1 - c1) + (s2 - c2), compensated; symmetric in the two operands
                const float a1 = acc[i] - cmp[i], a2 = s2 - c2;
                acc[i] = a1 + a2;
                cmp[i] = 0.f;
            } else {
                acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
            }
        }
    }
    if (KAHAN) {
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] -= cmp[i];
    }
}

// S = S_hi + S_lo of one 8-element chunk into the stage (lanes < L of the part write).
__device__ __forceinline__ void store_pair(uint32_t sb, uint32_t blk, int n_kb, int kofs, int r, int lane,
                                           const float (&acc)[8]) {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        hi[i] = pack_bf16x2(acc[2 * i], acc[2 * i + 1]);
        const float h0 = __uint_as_float(hi[i] << 16), h1 = __uint_as_float(hi[i] & 0xffff0000u);
        lo[i] = pack_bf16x2(acc[2 * i] - h0, acc[2 * i + 1] - h1);
    }
    const int k = kofs + 8 * lane;  // first element of this lane's chunk in K
    const uint32_t off = (uint32_t)(k >> 6) * blk + (uint32_t)r * 128u +
                         ((((uint32_t)(k >> 3) & 7u) ^ ((uint32_t)r & 7u)) << 4);
    st_shared_v4(sb + off, hi[0], hi[1], hi[2], hi[3]);
    st_shared_v4(sb + (uint32_t)n_kb * blk + off, lo[0], lo[1], lo[2], lo[3]);
}

template <bool BWD, bool KAHAN, int K1, int K0>
__global__ void __launch_bounds__(kThreads, 1)
agg_tc_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ AggArgs a) {
    extern __shared__ uint8_t dyn_smem[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~(uintptr_t)1023);
    const int N = a.tile_n;
    const uint32_t a_bytes = (uint32_t)a.n_kb * a.m_blocks * 16384u;
    const uint32_t blk = (uint32_t)N * 128u;  // one 64-column block of a stage
    const uint32_t stage_bytes = (uint32_t)(2 * a.n_kb + a.z_blocks) * blk;
    uint8_t* a_smem = base;
    uint8_t* st_smem = base + a_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(st_smem + (size_t)a.stages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + a.stages;
    uint64_t* tfull = bars + 2 * a.stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* wbar = tempty + 2;
    uint64_t* drain = wbar + 1;
    int* ctr = reinterpret_cast<int*>(drain + 1);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctr + a.stages);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(smem_u32(&full[s]), kProdThreads);
            mbar_init(smem_u32(&empty[s]), 1);
            ctr[s] = 0;
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
    // zero the stages (columns a part does not fill stay zero)
    for (uint32_t i = tid; i < (uint32_t)a.stages * stage_bytes / 16u; i += kThreads)
        st_shared_v4(smem_u32(st_smem) + i * 16u, 0u, 0u, 0u, 0u);
    fence_proxy_async();
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t acc_stride = (uint32_t)a.m_blocks * N;
    const bool producer = warp < kMmaWarp || warp >= kEpiWarp0 + kEpiWarps;

    if (producer) {
        // ------------------------------------------------------------------ producers
        // Group mode (every part L = width / 8 >= 4 lanes wide): a warp takes G = 32 / L rows at once
        // and lane group g sums row g alone (lane = one 16-byte chunk of the row), so a row needs no
        // cross-group reduction and the per-row work is shared by G rows. Other widths: one row at a
        // time with the general part sums.
        const int Lw = a.width[0] >> 3;  // a power of two
        const int lsh = 31 - __clz(Lw);   // log2(Lw): no integer division in the loops below
        const bool gmode = Lw >= 4 && (a.n_parts == 1 || a.width[1] == a.width[0]);
        const int G = gmode ? 32 >> lsh : 1;
        const int grp = gmode ? lane >> lsh : 0, ch = gmode ? (lane & (Lw - 1)) : lane;
        const int zch = BWD ? a.d_z >> 3 : 0;  // 16-byte chunks of a z row
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++lt) {
            const int s = lt % a.stages;
            const uint32_t use = (uint32_t)(lt / a.stages);
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&empty[s]), (use & 1u) ^ 1u, a.status, abort_flag))) break;
            const uint32_t sb = smem_u32(st_smem + (size_t)s * stage_bytes);
            const int64_t v0 = tile * N;
            // rows are taken G at a time from the stage's counter; each warp's last take fails, so a
            // tile use consumes exactly G * (ceil(N / G) + kProdWarps) values
            const int cbase = (int)use * G * ((N + G - 1) / G + kProdWarps);
            bool done = false;
            auto take = [&]() {
                if (done) return N;
                int r = 0;
                if (lane == 0) r = atomicAdd(ctr + s, G) - cbase;
                r = __shfl_sync(0xffffffffu, r, 0);
                if (r >= N) done = true;
                return r;
            };
            auto meta_of = [&](int r) {
                return (r < N && v0 + r < a.nv) ? __ldg(a.vr + v0 + r) : make_int4(0, 0, -1, -1);
            };
            // past the last virtual row: zero the row's S blocks (stale rows would add into dW)
            auto zero_row = [&](int r, int l0, int nl) {
                for (int i = l0; i < 2 * a.n_kb * 8; i += nl)
                    st_shared_v4(sb + (uint32_t)(i >> 3) * blk + (uint32_t)r * 128u + (uint32_t)(i & 7) * 16u, 0u, 0u, 0u, 0u);
            };
            auto z_store = [&](int r, int c, const uint4& zc) {
                st_shared_v4(sb + (uint32_t)(2 * a.n_kb + (c >> 3)) * blk + (uint32_t)r * 128u +
                                 ((((uint32_t)c & 7u) ^ ((uint32_t)r & 7u)) << 4),
                             zc.x, zc.y, zc.z, zc.w);
            };
            if (!gmode) {
                // ---------------------------------------------------------------- one row at a time
                for (int r = take(); r < N; r = take()) {
                    const int4 m = meta_of(r);
                    if (m.z < 0) {
                        zero_row(r, lane, 32);
                        continue;
                    }
                    int ix[kMaxParts];
#pragma unroll
                    for (int p = 0; p < kMaxParts; ++p)
                        ix[p] = (p < a.n_parts && lane < m.y) ? __ldg(a.gidx[p] + m.x + lane) : -1;
                    for (int c = lane; c < zch; c += 32)
                        z_store(r, c, __ldg(reinterpret_cast<const uint4*>(a.zrows + (int64_t)m.z * a.d_z) + c));
#pragma unroll
                    for (int p = 0; p < kMaxParts; ++p) {
                        if (p >= a.n_parts) break;
                        float acc[8];
                        part_sum<KAHAN>(a.tbl[p], a.tbl_rows[p], a.status, a.width[p], a.kind[p], ix[p], m.y, lane, acc);
                        if (lane < (a.width[p] >> 3)) store_pair(sb, blk, a.n_kb, a.kofs[p], r, lane, acc);
                    }
                }
            } else {
                // ---------------------------------------------------------------- G rows at a time
                // lane (g, c) holds tuple c + L i of row g's part indices, i < G (rows <= 32 tuples)
                int r_n = take();
                int4 m_n = meta_of(r_n + grp);
                int ix_n[kMaxParts][kMaxG];
                auto load_idx = [&](const int4& m, int (&ix)[kMaxParts][kMaxG]) {
#pragma unroll
                    for (int p = 0; p < kMaxParts; ++p)
#pragma unroll
                        for (int i = 0; i < kMaxG; ++i) {
                            const int t = ch + Lw * i;
                            ix[p][i] = (p < a.n_parts && i < G && m.z >= 0 && t < m.y) ? __ldg(a.gidx[p] + m.x + t) : -1;
                        }
                };
                load_idx(m_n, ix_n);
                while (r_n < N) {
                    const int r0 = r_n;
                    const int4 m = m_n;
                    int ix[kMaxParts][kMaxG];
#pragma unroll
                    for (int p = 0; p < kMaxParts; ++p)
#pragma unroll
                        for (int i = 0; i < kMaxG; ++i) ix[p][i] = ix_n[p][i];
                    const int rr = r0 + grp;  // this lane group's row
                    const bool row_ok = rr < N && m.z >= 0;
                    const int nmax = __reduce_max_sync(0xffffffffu, row_ok ? m.y : 0);
                    // the single-row part: every tuple of a row names the same table row (else the
                    // warp takes the general path for its rows)
                    int first1 = -1;
                    bool single = true;
                    if (K1) {
                        first1 = __shfl_sync(0xffffffffu, ix[0][0], grp << lsh);
#pragma unroll
                        for (int i = 0; i < kMaxG; ++i)
                            single = single && (i >= G || ix[0][i] < 0 || ix[0][i] == first1);
                        single = __all_sync(0xffffffffu, single);
                    }
                    // the next rows' descriptors and indices load while these rows are summed
                    r_n = take();
                    m_n = meta_of(r_n + grp);
                    load_idx(m_n, ix_n);
                    if (!single) {
                        // general path, row by row (indices reloaded in row layout)
                        for (int g = 0; g < G; ++g) {
                            const int r = r0 + g;
                            if (r >= N) break;
                            const int4 mg = meta_of(r);
                            if (mg.z < 0) {
                                zero_row(r, lane, 32);
                                continue;
                            }
                            int ixr[kMaxParts];
#pragma unroll
                            for (int p = 0; p < kMaxParts; ++p)
                                ixr[p] = (p < a.n_parts && lane < mg.y) ? __ldg(a.gidx[p] + mg.x + lane) : -1;
                            for (int c = lane; c < zch; c += 32)
                                z_store(r, c, __ldg(reinterpret_cast<const uint4*>(a.zrows + (int64_t)mg.z * a.d_z) + c));
#pragma unroll
                            for (int p = 0; p < kMaxParts; ++p) {
                                if (p >= a.n_parts) break;
                                float acc[8];
                                part_sum<KAHAN>(a.tbl[p], a.tbl_rows[p], a.status, a.width[p], a.kind[p], ixr[p], mg.y, lane, acc);
                                if (lane < (a.width[p] >> 3)) store_pair(sb, blk, a.n_kb, a.kofs[p], r, lane, acc);
                            }
                        }
                        continue;
                    }
                    // every load of the rows' first 16 tuples (and the single-row part, and z) in flight
                    // before any is summed
                    uint4 zc[kMaxZ];
#pragma unroll
                    for (int i = 0; i < kMaxZ; ++i) {
                        const int c = ch + Lw * i;
                        zc[i] = (BWD && row_ok && c < zch)
                                    ? __ldg(reinterpret_cast<const uint4*>(a.zrows + (int64_t)m.z * a.d_z) + c)
                                    : make_uint4(0u, 0u, 0u, 0u);
                    }
                    uint4 d1 = make_uint4(0u, 0u, 0u, 0u);
                    if (K1 && row_ok && m.y > 0 && in_bounds(first1, a.tbl_rows[0], a.status))
                        d1 = __ldg(reinterpret_cast<const uint4*>(a.tbl[0]) + (int64_t)first1 * Lw + ch);
                    float acc[8], cmp[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) acc[i] = cmp[i] = 0.f;
                    if (K0) {
                        const uint4* __restrict__ base = reinterpret_cast<const uint4*>(a.tbl[K1]) + ch;
                        // round 0: tuples 0..15, round 1: 16..31 (rows of more than 16 tuples)
#pragma unroll
                        for (int round = 0; round < 2; ++round) {
                            if (round == 1 && nmax <= kRound) break;
                            uint4 u[kRound];
#pragma unroll
                            for (int q = 0; q < kRound; ++q) {
                                const int j = round * kRound + q;  // compile-time
                                const int src = (grp << lsh) + (j & (Lw - 1));
                                // register j / L of the group's lanes holds tuple j
                                const int jr = j >> lsh;
                                int v = -1;
#pragma unroll
                                for (int i = 0; i < kMaxG; ++i)
                                    if (i == jr) v = ix[K1][i];
                                const int r = __shfl_sync(0xffffffffu, v, src);
                                u[q] = (row_ok && j < m.y && in_bounds(r, a.tbl_rows[K1], a.status))
                                           ? __ldg(base + (int64_t)r * Lw)
                                           : make_uint4(0u, 0u, 0u, 0u);
                            }
#pragma unroll
                            for (int q = 0; q < kRound; ++q) {
                                if (round * kRound + q >= nmax) break;
                                add8(acc, cmp, u[q], KAHAN);
                            }
                        }
                    }
                    if (rr < N) {
                        if (!row_ok) {
                            zero_row(rr, ch, Lw);
                        } else {
                            if (K1) {
                                // count x a bf16 value is exact in f32 (count <= 32)
                                float a1[8];
                                const float c1 = (float)m.y;
                                const uint32_t w[4] = {d1.x, d1.y, d1.z, d1.w};
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    a1[2 * i] = c1 * __uint_as_float(w[i] << 16);
                                    a1[2 * i + 1] = c1 * __uint_as_float(w[i] & 0xffff0000u);
                                }
                                store_pair(sb, blk, a.n_kb, a.kofs[0], rr, ch, a1);
                            }
                            if (K0) {
                                if (KAHAN) {
#pragma unroll
                                    for (int i = 0; i < 8; ++i) acc[i] -= cmp[i];
                                }
                                store_pair(sb, blk, a.n_kb, a.kofs[K1], rr, ch, acc);
                            }
#pragma unroll
                            for (int i = 0; i < kMaxZ; ++i) {
                                const int c = ch + Lw * i;
                                if (BWD && c < zch) z_store(rr, c, zc[i]);
                            }
                            for (int c = ch + Lw * kMaxZ; BWD && c < zch; c += Lw)
                                z_store(rr, c, __ldg(reinterpret_cast<const uint4*>(a.zrows + (int64_t)m.z * a.d_z) + c));
                        }
                    }
                }
            }
            fence_proxy_async();
            mbar_arrive(smem_u32(&full[s]));
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t wb = smem_u32(wbar);
            mbar_arrive_expect_tx(wb, a_bytes);
            for (int kb = 0; kb < a.n_kb; ++kb)
                for (int mb = 0; mb < a.m_blocks; ++mb)
                    tma_load_2d(smem_u32(a_smem + (size_t)(kb * a.m_blocks + mb) * 16384u), &amap, kb * 64, mb * 128, wb);
            bool ok = mbar_wait(wb, 0, a.status, abort_flag);
            tc_fence_after();
            int lt = 0;
            for (int64_t tile = blockIdx.x; tile < a.n_tiles && ok; tile += gridDim.x, ++lt) {
                const int s = lt % a.stages;
                const uint32_t use = (uint32_t)(lt / a.stages);
                const int acc = lt & 1;
                const uint32_t ause = (uint32_t)(lt >> 1);
                if (!mbar_wait(smem_u32(&tempty[acc]), (ause & 1u) ^ 1u, a.status, abort_flag)) { ok = false; break; }
                if (!mbar_wait(smem_u32(&full[s]), use & 1u, a.status, abort_flag)) { ok = false; break; }
                fence_proxy_async();
                tc_fence_after();
                const uint32_t sb = smem_u32(st_smem + (size_t)s * stage_bytes);
                const uint32_t d_acc = tmem_base + (uint32_t)acc * acc_stride;
                for (int mb = 0; mb < a.m_blocks; ++mb) {
                    uint32_t accum = 0;
                    for (int kb = 0; kb < a.n_kb; ++kb) {
                        const uint32_t ab = smem_u32(a_smem + (size_t)(kb * a.m_blocks + mb) * 16384u);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint64_t adesc = sw128_kmajor_desc(ab + k * 32);
#pragma unroll
                            for (int hl = 0; hl < 2; ++hl) {
                                const uint64_t bdesc = sw128_kmajor_desc(sb + (uint32_t)(hl * a.n_kb + kb) * blk + k * 32);
                                mma_bf16(d_acc + (uint32_t)mb * N, adesc, bdesc, a.idesc, accum);
                                accum = 1;
                            }
                        }
                    }
                }
                if (BWD) {
                    // G^T Z: K = the tile's rows (16 per instruction), both operands read MN-major
                    // from the staged rows
                    const uint32_t zb = sb + (uint32_t)(2 * a.n_kb) * blk;
                    for (int step = 0; step < N / 16; ++step) {
                        for (int mbw = 0; mbw < a.m_dw; ++mbw) {
#pragma unroll
                            for (int hl = 0; hl < 2; ++hl) {
                                const uint32_t accw = (lt > 0 || step > 0 || hl > 0) ? 1u : 0u;
                                const uint64_t ad = sw128_mnmajor_desc(
                                    sb + (uint32_t)(hl * a.n_kb + 2 * mbw) * blk + (uint32_t)step * 2048u, blk);
                                const uint64_t bd = sw128_mnmajor_desc(zb + (uint32_t)step * 2048u, blk);
                                mma_bf16(tmem_base + a.dw_col + (uint32_t)mbw * a.d_z, ad, bd, a.idesc_dw, accw);
                            }
                        }
                    }
                }
                mma_commit(smem_u32(&empty[s]));
                mma_commit(smem_u32(&tfull[acc]));
            }
            // every issued MMA has finished before the dW read-out and the TMEM release
            mma_commit(smem_u32(drain));
            mbar_wait(smem_u32(drain), 0, a.status, abort_flag);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------ epilogue
        const int q = warp & 3;
        float bias_r[2];
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
            const int o = mb * 128 + 32 * q + lane;
            bias_r[mb] = (a.bias && mb < a.m_blocks && o < a.n_feat) ? a.bias[o] : 0.f;
        }
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            const uint32_t ause = (uint32_t)(lt >> 1);
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[acc]), ause & 1u, a.status, abort_flag))) break;
            tc_fence_after();
            const int64_t v0 = tile * N;
            for (int c = 0; c < N / 32; ++c) {
                const int64_t vb = v0 + 32 * c;
                if (vb >= a.nv) break;
                const int4 mt = vb + lane < a.nv ? __ldg(a.vr + vb + lane) : make_int4(0, 0, -1, -1);
                for (int mb = 0; mb < a.m_blocks; ++mb) {
                    if (mb * 128 + 32 * q >= a.n_feat) continue;
                    const int o = mb * 128 + 32 * q + lane;
                    const bool o_ok = o < a.n_feat && a.out != nullptr;
                    const float bo = mb == 0 ? bias_r[0] : bias_r[1];
                    uint32_t v[32];
                    tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)acc * acc_stride +
                                           (uint32_t)mb * N + (uint32_t)(32 * c), v);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int row = __shfl_sync(0xffffffffu, mt.z, j);
                        const int part = __shfl_sync(0xffffffffu, mt.w, j);
                        const int nj = __shfl_sync(0xffffffffu, mt.y, j);
                        if (row < 0) break;  // past the last virtual row (warp-uniform)
                        if (o_ok) {
                            const float y = __uint_as_float(v[j]) + (float)nj * bo;
                            if (part >= 0) __stcg(a.vpart + (int64_t)part * a.n_feat + o, y);
                            else emit_out(a.out + (int64_t)row * a.n_feat + o, y, a.accumulate);
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&tempty[acc]));
        }
        if (BWD) {
            // this CTA's dW (TMEM lane = G feature, columns = z features)
            if (__all_sync(0xffffffffu, mbar_wait(smem_u32(drain), 0, a.status, abort_flag))) {
                tc_fence_after();
                for (int mbw = 0; mbw < a.m_dw; ++mbw) {
                    const int g = mbw * 128 + 32 * q + lane;
                    float* dst = a.dw_part + ((int64_t)blockIdx.x * a.n_g + g) * a.d_z;
                    for (int c = 0; c < a.d_z / 32; ++c) {
                        uint32_t v[32];
                        tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(32 * q) << 16) + a.dw_col + (uint32_t)mbw * a.d_z +
                                               (uint32_t)(32 * c), v);
                        tmem_ld_wait();
                        if (g < a.n_g) {
#pragma unroll
                            for (int j = 0; j < 32; j += 4)
                                *reinterpret_cast<float4*>(dst + 32 * c + j) =
                                    make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
                        }
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

// ------------------------------------------------------------------------------ two-kernel forward
// For a plan whose H keys are unique, the forward runs as two kernels:
//   seg_sum_kernel  S_src[v] = sum over virtual row v's tuples of z[hs_t] (f32 on CUDA cores, high
//                   occupancy, the next row's tuple indices loading while a row is summed), stored
//                   as a bf16 pair S_hi | S_lo per row;
//   agg_gemm_kernel D1 = W_src [S_hi; S_lo] with S staged by TMA, D2 = W_dst z[hd(v)] with the dst rows
//                   (exact bf16) copied by cp.async, and Out = D1 + n_v (D2 + b) in the epilogue (the
//                   dst part of S is n_v z[hd(v)], so scaling D2 gives it exactly).

// S[v][0, w) = S_hi, S[v][kpad, kpad + w) = S_lo of the sum of the tuples' table rows; the other
// columns of the row zero. A warp takes 32 virtual rows at a time (their descriptors in one load);
// their tuples are one contiguous range of gidx (at most 32 x 32 indices), staged in shared memory.
// Lane groups of L = w / 8 lanes each own one row at a time (a lane = one 16-byte chunk of the row,
// so a group needs no reduction across lanes): G = 32 / L rows are summed side by side, each group
// walking its row's tuples in order with up to kSegUnroll row loads in flight.
// SINGLE: every tuple of a virtual row names the same table row (the backward's runs of equal dst
// rows): the row is loaded once and multiplied by the tuple count (exact in f32, count <= 32).
constexpr int kSegWarps = 8;
// row loads in flight per lane of the gather-sum: 6 with four blocks per SM (at most 64 registers)
// measured 4 % faster on the single-rule workload than 8 with three
constexpr int kSegUnroll = 6;

// MASK (the backward of a ReLU rule): every tuple's row is taken through its ReLU mask bits (the
// forward's per-tuple mask, uint32 [m][mask_words], bit o of word o / 32 = feature o active). The
// src pass reads the mask already permuted into its tuple order; the dst pass (SINGLE) counts,
// per feature, the active tuples of the run (plan positions x .. x + n - 1) and also sums its rows,
// from the f32 table tbl_f32 (16-byte aligned rows), into this block's db partial db_part[block][w]
// (the warps' sums added in warp order).
template <bool KAHAN, bool SINGLE, bool MASK = false>
__global__ void __launch_bounds__(32 * kSegWarps, 4) seg_sum_kernel(const int4* __restrict__ vr, int64_t nv,
                                                                 const int32_t* __restrict__ gidx,
                                                                 const uint16_t* __restrict__ tbl, int64_t tbl_rows,
                                                                 int w, int kpad, uint16_t* __restrict__ S,
                                                                 int* status, int kahan_min,
                                                                 const uint32_t* __restrict__ mask = nullptr,
                                                                 int mask_words = 0,
                                                                 float* __restrict__ db_part = nullptr,
                                                                 const float* __restrict__ tbl_f32 = nullptr) {
    // MASK (src pass): batches of 16 rows, whose mask words are staged in shared memory with their
    // indices (one contiguous copy per batch instead of a second load per tuple)
    constexpr bool SMASK = MASK && !SINGLE;
    constexpr int kBR = SMASK ? 16 : 32;  // virtual rows per batch
    constexpr int kBI = kBR * kChunk;     // their tuple indices at most
    __shared__ int32_t s_idx[SINGLE ? 1 : kSegWarps][SINGLE ? 1 : kBI];
    __shared__ uint32_t s_mk[SMASK ? kSegWarps : 1][SMASK ? 2 * kBI : 1];
    __shared__ float s_db[MASK && SINGLE ? kSegWarps : 1][MASK && SINGLE ? 256 : 1];
    // src pass of a ReLU rule: the AND mask of 8 bf16 elements for each byte of mask bits
    __shared__ uint4 s_lut[MASK && !SINGLE ? 256 : 1];
    if (MASK && !SINGLE) {
        for (int v = threadIdx.x; v < 256; v += blockDim.x) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                w[i] = ((v >> (2 * i)) & 1 ? 0x0000ffffu : 0u) | ((v >> (2 * i + 1)) & 1 ? 0xffff0000u : 0u);
            s_lut[v] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int L = w >> 3, lsh = 31 - __clz(L), G = 32 >> lsh;
    const int grp = lane >> lsh, ch = lane & (L - 1);
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint4* __restrict__ base = reinterpret_cast<const uint4*>(tbl) + ch;
    const int pitch = 2 * kpad, nck = kpad >> 3;
    int32_t* sidx = s_idx[SINGLE ? 0 : threadIdx.x >> 5];
    uint32_t* smk = s_mk[SMASK ? threadIdx.x >> 5 : 0];
    const bool stage_mask = SMASK && mask_words <= 2;
    const int mword = (8 * ch) >> 5, msh = (8 * ch) & 31;  // this lane's 8 features in the mask
    float dbacc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) dbacc[i] = 0.f;
    for (int64_t vb = warp0 * kBR; vb < nv; vb += nw * kBR) {
        const int4 mine = (lane < kBR && vb + lane < nv) ? __ldg(vr + vb + lane) : make_int4(0, 0, -1, -1);
        const int nrows = (int)imin64(kBR, nv - vb);
        const int myn = mine.y > 0 ? mine.y : 0;
        int x0 = 0;
        bool ok = true;
        if (!SINGLE) {
            x0 = (int)__reduce_min_sync(0xffffffffu, (unsigned)(myn > 0 ? mine.x : INT_MAX));
            const int cnt = (int)__reduce_add_sync(0xffffffffu, (unsigned)myn);
            const int x1 = (int)__reduce_max_sync(0xffffffffu, (unsigned)(myn > 0 ? mine.x + myn : 0));
            // the non-empty rows' tuples must tile [x0, x0 + cnt) (virtual rows are in tuple order)
            ok = cnt == 0 || (x1 - x0 == cnt && cnt <= kBI);
            if (!ok && lane == 0) raise_status(status, RELNN_DEV_BOUNDS);
            __syncwarp();
            if (ok)
                for (int i = lane; i < cnt; i += 32) sidx[i] = __ldg(gidx + x0 + i);
            if (ok && stage_mask)
                for (int i = lane; i < cnt * mask_words; i += 32) smk[i] = __ldg(mask + (int64_t)x0 * mask_words + i);
            __syncwarp();
        }
        for (int j0 = 0; j0 < nrows; j0 += G) {
            const int j = j0 + grp;  // this group's row of the batch
            const int jj = j < nrows ? j : 0;
            // every lane takes part in every shuffle (none under a condition)
            const int n_j = __shfl_sync(0xffffffffu, myn, jj);
            const int x_j = __shfl_sync(0xffffffffu, mine.x, jj);
            const int p_j = __shfl_sync(0xffffffffu, mine.w, jj);
            const int n = (j < nrows && ok) ? n_j : 0;
            const int xo = x_j - x0;
            // KAHAN: compensated for rows of at least kahan_min tuples and for chunks of cut rows
            const bool kh = KAHAN && (n >= kahan_min || p_j >= 0);
            float acc[8], cmp[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = cmp[i] = 0.f;
            if (SINGLE) {
                const int r = n > 0 ? __ldg(gidx + xo) : -1;
                if (n > 0 && in_bounds(r, tbl_rows, status)) {
                    const uint4 u = __ldg(base + (int64_t)r * L);
                    float c[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) c[i] = (float)n;
                    if (MASK) {
                        // per feature, the run's tuples whose ReLU was active
                        int ci[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                        for (int t = 0; t < n; ++t) {
                            const uint32_t mw = __ldg(mask + (int64_t)(xo + t) * mask_words + mword) >> msh;
#pragma unroll
                            for (int i = 0; i < 8; ++i) ci[i] += (mw >> i) & 1u;
                        }
#pragma unroll
                        for (int i = 0; i < 8; ++i) c[i] = (float)ci[i];
                    }
                    const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        acc[2 * i] = c[2 * i] * __uint_as_float(wd[i] << 16);
                        acc[2 * i + 1] = c[2 * i + 1] * __uint_as_float(wd[i] & 0xffff0000u);
                    }
                    if (MASK) {
                        // db from the f32 rows (the bf16 copy feeds only the tensor cores)
                        const float4* fr = reinterpret_cast<const float4*>(tbl_f32 + (int64_t)r * w + 8 * ch);
                        const float4 f0 = __ldg(fr), f1 = __ldg(fr + 1);
                        dbacc[0] += c[0] * f0.x;
                        dbacc[1] += c[1] * f0.y;
                        dbacc[2] += c[2] * f0.z;
                        dbacc[3] += c[3] * f0.w;
                        dbacc[4] += c[4] * f1.x;
                        dbacc[5] += c[5] * f1.y;
                        dbacc[6] += c[6] * f1.z;
                        dbacc[7] += c[7] * f1.w;
                    }
                }
            } else {
                const int nmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)n);
                for (int t0 = 0; t0 < nmax; t0 += kSegUnroll) {
                    const int slots = min(kSegUnroll, nmax - t0);  // warp-uniform
                    uint4 u[kSegUnroll];
                    uint32_t mk[kSegUnroll];
#pragma unroll
                    for (int q = 0; q < kSegUnroll; ++q) {
                        if (q >= slots) break;
                        u[q] = make_uint4(0u, 0u, 0u, 0u);
                        mk[q] = 0u;
                        if (t0 + q < n) {
                            const int r = sidx[xo + t0 + q];
                            if (in_bounds(r, tbl_rows, status)) u[q] = __ldg(base + (int64_t)r * L);
                            if (MASK)
                                mk[q] = (stage_mask ? smk[(xo + t0 + q) * mask_words + mword]
                                                    : __ldg(mask + (int64_t)(x0 + xo + t0 + q) * mask_words + mword)) >> msh;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kSegUnroll; ++q) {
                        if (q >= slots) break;
                        if (MASK) {
                            // a bf16 element whose ReLU was inactive becomes +0 (bit j of the byte
                            // selects element j; the byte's AND mask comes from the table)
                            const uint4 am = s_lut[mk[q] & 0xffu];
                            u[q].x &= am.x;
                            u[q].y &= am.y;
                            u[q].z &= am.z;
                            u[q].w &= am.w;
                        }
                        add8(acc, cmp, u[q], kh);
                    }
                }
            }
            if (KAHAN) {
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] -= cmp[i];
            }
            if (j < nrows) {
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    hi[i] = pack_bf16x2(acc[2 * i], acc[2 * i + 1]);
                    const float h0 = __uint_as_float(hi[i] << 16), h1 = __uint_as_float(hi[i] & 0xffff0000u);
                    lo[i] = pack_bf16x2(acc[2 * i] - h0, acc[2 * i + 1] - h1);
                }
                uint16_t* row = S + (vb + j) * pitch;
                for (int c = ch; c < nck; c += L) {
                    const bool data = c < L;  // chunks past w are the zero padding of each half
                    *reinterpret_cast<uint4*>(row + 8 * c) =
                        data ? make_uint4(hi[0], hi[1], hi[2], hi[3]) : make_uint4(0u, 0u, 0u, 0u);
                    *reinterpret_cast<uint4*>(row + kpad + 8 * c) =
                        data ? make_uint4(lo[0], lo[1], lo[2], lo[3]) : make_uint4(0u, 0u, 0u, 0u);
                }
            }
        }
    }
    if (MASK && SINGLE) {
        // db partial of this block: groups of the warp in group order (butterfly over lanes with the
        // same column chunk), then warps in warp order
        for (int off = L; off < 32; off <<= 1) {
#pragma unroll
            for (int i = 0; i < 8; ++i) dbacc[i] += __shfl_xor_sync(0xffffffffu, dbacc[i], off);
        }
        const int wib = threadIdx.x >> 5;
        if (lane < L) {
#pragma unroll
            for (int i = 0; i < 8; ++i) s_db[wib][8 * lane + i] = dbacc[i];
        }
        __syncthreads();
        for (int f = threadIdx.x; f < w; f += blockDim.x) {
            float sacc = 0.f;
            for (int k = 0; k < kSegWarps; ++k) sacc += s_db[k][f];
            db_part[(int64_t)blockIdx.x * w + f] = sacc;
        }
    }
}

// The ReLU mask rows in the src pass's tuple order, keeping only the words that hold features:
// out[i][w] = mask[perm[i]][w] for w < out_words (= ceil(d_out / 32) <= mask_words).
__global__ void permute_mask_kernel(const uint32_t* __restrict__ mask, const int32_t* __restrict__ perm, int64_t m,
                                    int mask_words, int out_words, uint32_t* __restrict__ out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t* row = mask + (int64_t)__ldg(perm + t) * mask_words;
        for (int w = 0; w < out_words; ++w) out[t * out_words + w] = __ldg(row + w);
    }
}

// Grid of the gather-sum: every block resident (the warps stride over the 32-row batches).
template <bool KAHAN, bool SINGLE, bool MASK = false>
int seg_sum_grid(int64_t nv) {
    static int per_sm = 0;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, seg_sum_kernel<KAHAN, SINGLE, MASK>, 32 * kSegWarps, 0) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            per_sm = 0;
        }
        per_sm = std::max(1, per_sm);
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nv, 32 * kSegWarps), (int64_t)num_sms() * per_sm));
}

// The plain gather-sum (no compensation, no mask) with 32-byte lane chunks, for rows of w = 16 .. 256
// elements (a power of two) in a 32-byte aligned table: a lane owns 16 elements of its row
// (one 256-bit load per tuple), so each tuple's index, address and load serve 16 adds instead of 8.
// The same sums in the same order as seg_sum_kernel<false, false>, so the same S bit for bit.
template <int U>
__global__ void __launch_bounds__(32 * kSegWarps, 4) seg_sum_wide_kernel(const int4* __restrict__ vr, int64_t nv,
                                                                      const int32_t* __restrict__ gidx,
                                                                      const uint16_t* __restrict__ tbl, int64_t tbl_rows,
                                                                      int w, int kpad, uint16_t* __restrict__ S,
                                                                      int* status) {
    // batches of 16 virtual rows: 16 KB of staged indices per block instead of 32 leave more of the
    // SM's shared storage to L1 (the backward's src pass over a 256 MB dOut table: 0.489 -> 0.438 ms)
    constexpr int kBR = 16;
    constexpr int kBI = kBR * kChunk;
    __shared__ int32_t s_idx[kSegWarps][kBI];
    const int lane = threadIdx.x & 31;
    const int L = w >> 4, lsh = 31 - __clz(L), G = 32 >> lsh;
    const int grp = lane >> lsh, ch = lane & (L - 1);
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint16_t* __restrict__ base = tbl + 16 * ch;
    const int pitch = 2 * kpad, nck = kpad >> 3;
    int32_t* sidx = s_idx[threadIdx.x >> 5];
    for (int64_t vb = warp0 * kBR; vb < nv; vb += nw * kBR) {
        const int4 mine = (lane < kBR && vb + lane < nv) ? __ldg(vr + vb + lane) : make_int4(0, 0, -1, -1);
        const int nrows = (int)imin64(kBR, nv - vb);
        const int myn = mine.y > 0 ? mine.y : 0;
        const int x0 = (int)__reduce_min_sync(0xffffffffu, (unsigned)(myn > 0 ? mine.x : INT_MAX));
        const int cnt = (int)__reduce_add_sync(0xffffffffu, (unsigned)myn);
        const int x1 = (int)__reduce_max_sync(0xffffffffu, (unsigned)(myn > 0 ? mine.x + myn : 0));
        // the non-empty rows' tuples must tile [x0, x0 + cnt) (virtual rows are in tuple order)
        const bool ok = cnt == 0 || (x1 - x0 == cnt && cnt <= kBI);
        if (!ok && lane == 0) raise_status(status, RELNN_DEV_BOUNDS);
        __syncwarp();
        if (ok)
            for (int i = lane; i < cnt; i += 32) sidx[i] = __ldg(gidx + x0 + i);
        __syncwarp();
        for (int j0 = 0; j0 < nrows; j0 += G) {
            const int j = j0 + grp;
            const int jj = j < nrows ? j : 0;
            const int n_j = __shfl_sync(0xffffffffu, myn, jj);
            const int x_j = __shfl_sync(0xffffffffu, mine.x, jj);
            const int n = (j < nrows && ok) ? n_j : 0;
            const int xo = x_j - x0;
            float acc[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = 0.f;
            const int nmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)n);
            for (int t0 = 0; t0 < nmax; t0 += U) {
                const int slots = min(U, nmax - t0);  // warp-uniform
                uint32_t u[U][8];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    if (q >= slots) break;
#pragma unroll
                    for (int i = 0; i < 8; ++i) u[q][i] = 0u;
                    if (t0 + q < n) {
                        const int r = sidx[xo + t0 + q];
                        if (in_bounds(r, tbl_rows, status))
                            asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                                : "=r"(u[q][0]), "=r"(u[q][1]), "=r"(u[q][2]), "=r"(u[q][3]), "=r"(u[q][4]),
                                  "=r"(u[q][5]), "=r"(u[q][6]), "=r"(u[q][7])
                                : "l"(base + (int64_t)r * w));
                    }
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    if (q >= slots) break;
#pragma unroll
                    for (int i = 0; i < 8; ++i) add_bf16x2(acc[2 * i], acc[2 * i + 1], u[q][i]);
                }
            }
            if (j < nrows) {
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    hi[i] = pack_bf16x2(acc[2 * i], acc[2 * i + 1]);
                    const float h0 = __uint_as_float(hi[i] << 16), h1 = __uint_as_float(hi[i] & 0xffff0000u);
                    lo[i] = pack_bf16x2(acc[2 * i] - h0, acc[2 * i + 1] - h1);
                }
                uint16_t* row = S + (vb + j) * pitch;
                uint4* ph = reinterpret_cast<uint4*>(row + 16 * ch);
                uint4* pl = reinterpret_cast<uint4*>(row + kpad + 16 * ch);
                ph[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                ph[1] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
                pl[0] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                pl[1] = make_uint4(lo[4], lo[5], lo[6], lo[7]);
                // 8-element chunks past w: the zero padding of each half
                for (int c = 2 * L + ch; c < nck; c += L) {
                    *reinterpret_cast<uint4*>(row + 8 * c) = make_uint4(0u, 0u, 0u, 0u);
                    *reinterpret_cast<uint4*>(row + kpad + 8 * c) = make_uint4(0u, 0u, 0u, 0u);
                }
            }
        }
    }
}

constexpr int kSegUnrollWide = 3;  // 256-bit row loads in flight per lane (the same bytes as 6 x 16)

// The wide gather-sum is taken for rows of 64 .. 256 elements in a 32-byte aligned table. Narrower
// rows keep the 16-byte form: with twice the rows side by side in a warp, the warp-uniform loop over
// the longest row's tuples leaves more lanes idle (rows of 32: 16 % slower, measured).
bool seg_sum_wide_ok(int w, const void* tbl) {
    return w >= 64 && w <= 256 && (w & (w - 1)) == 0 && ((uintptr_t)tbl & 31) == 0;
}

int seg_sum_wide_grid(int64_t nv) {
    static int per_sm = 0;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, seg_sum_wide_kernel<kSegUnrollWide>, 32 * kSegWarps,
                                                          0) != cudaSuccess) {
            (void)cudaGetLastError();
            per_sm = 0;
        }
        per_sm = std::max(1, per_sm);
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nv, 32 * kSegWarps), (int64_t)num_sms() * per_sm));
}

// Dst H row of every virtual row (the first tuple's; all tuples of a row share it when H keys are
// unique), or -1 for an empty row.
__global__ void vr_first_kernel(const int4* __restrict__ vr, int64_t nv, const int32_t* __restrict__ hd, int32_t* d1) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        const int4 m = vr[v];
        d1[v] = m.y > 0 ? hd[m.x] : -1;
    }
}

// ------------------------------------------------------------------------------ FP32 form
// Aggregate-first forward of the FP32 form (f32 arithmetic on CUDA cores, no tensor cores) for linear
// rules with narrow rows: lane = one virtual row. The lane sums its tuples' src rows in f32 in tuple
// order (compensated with KAHAN), then applies the Linear once:
//     y = W_src S + n (W_dst z_dst + b)
// with W and b in shared memory (every lane reads the same element: a broadcast). A row cut into
// chunks leaves one partial per chunk, added in chunk order by the fix-up. The per-tuple FP32 form
// computes the same rule; the two differ by the order of f32 additions only.
constexpr int kF32Batch = 4;  // tuples of a lane whose row loads are in flight together

template <int D, bool CDST, bool KAHAN>
__global__ void __launch_bounds__(256) fwd_fp32_agg_kernel(const int4* __restrict__ vr, int64_t nv,
                                                        const int32_t* __restrict__ hs,
                                                        const int32_t* __restrict__ d1,
                                                        const float* __restrict__ z, int64_t z_rows,
                                                        const float* __restrict__ W, const float* __restrict__ bias,
                                                        int d_out, float* __restrict__ out, int64_t out_rows,
                                                        float* __restrict__ vpart, int accumulate, int* status) {
    constexpr int D4 = D / 4;
    constexpr int DIN4 = CDST ? 2 * D4 : D4;
    extern __shared__ float4 s_w4[];  // W [d_out][d_in / 4] (the src part, then the dst part), then b
    float* s_b = reinterpret_cast<float*>(s_w4 + (size_t)d_out * DIN4);
    for (int i = threadIdx.x; i < d_out * DIN4; i += blockDim.x) s_w4[i] = __ldg(reinterpret_cast<const float4*>(W) + i);
    for (int i = threadIdx.x; i < d_out; i += blockDim.x) s_b[i] = bias ? __ldg(bias + i) : 0.f;
    __syncthreads();
    const float4* __restrict__ z4 = reinterpret_cast<const float4*>(z);
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        const int4 m = __ldg(vr + v);  // {first tuple, tuples, output row, chunk slot or -1}
        const int n = m.y > 0 ? m.y : 0;
        // the dst row's index and row are loaded with the first tuples' (one round trip each)
        const int rd = CDST && n > 0 ? __ldg(d1 + v) : -1;
        float sx[D], cx[D];
#pragma unroll
        for (int k = 0; k < D; ++k) sx[k] = cx[k] = 0.f;
        float4 g[CDST ? D4 : 1];
        for (int t0 = 0; t0 < n; t0 += kF32Batch) {
            int r[kF32Batch];
#pragma unroll
            for (int q = 0; q < kF32Batch; ++q) r[q] = t0 + q < n ? __ldg(hs + m.x + t0 + q) : -1;
            if (CDST && t0 == 0) {
                const bool ok = rd >= 0 && in_bounds(rd, z_rows, status);
#pragma unroll
                for (int c = 0; c < D4; ++c) g[c] = ok ? __ldg(z4 + (int64_t)rd * D4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            float4 f[kF32Batch][D4];
#pragma unroll
            for (int q = 0; q < kF32Batch; ++q) {
                const bool ok = r[q] >= 0 && in_bounds(r[q], z_rows, status);
#pragma unroll
                for (int c = 0; c < D4; ++c)
                    f[q][c] = ok ? __ldg(z4 + (int64_t)r[q] * D4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < kF32Batch; ++q) {
                if (t0 + q >= n) break;
#pragma unroll
                for (int c = 0; c < D4; ++c) {
                    const float e[4] = {f[q][c].x, f[q][c].y, f[q][c].z, f[q][c].w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (KAHAN) kahan_add(sx[4 * c + j], cx[4 * c + j], e[j]);
                        else sx[4 * c + j] += e[j];
                    }
                }
            }
        }
        if (KAHAN) {
#pragma unroll
            for (int k = 0; k < D; ++k) sx[k] -= cx[k];
        }
        float zd[CDST ? D : 1];
        if (CDST) {
#pragma unroll
            for (int c = 0; c < D4; ++c) {
                const float4 gg = n > 0 ? g[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                zd[4 * c] = gg.x;
                zd[4 * c + 1] = gg.y;
                zd[4 * c + 2] = gg.z;
                zd[4 * c + 3] = gg.w;
            }
        }
        const bool part = m.w >= 0;
        if (!part && !in_bounds(m.z, out_rows, status)) continue;
        float* dst = part ? vpart + (int64_t)m.w * d_out : out + (int64_t)m.z * d_out;
        const float fn = (float)n;
        // four outputs at a time, stored as one 16-byte write (d_out is a multiple of 4)
        for (int o0 = 0; o0 < d_out; o0 += 4) {
            float y[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4* wr = s_w4 + (size_t)(o0 + j) * DIN4;
                float ys = 0.f, yd = 0.f;
#pragma unroll
                for (int c = 0; c < D4; ++c) {
                    const float4 w = wr[c];
                    ys = fmaf(w.x, sx[4 * c], ys);
                    ys = fmaf(w.y, sx[4 * c + 1], ys);
                    ys = fmaf(w.z, sx[4 * c + 2], ys);
                    ys = fmaf(w.w, sx[4 * c + 3], ys);
                    if (CDST) {
                        const float4 u = wr[D4 + c];
                        yd = fmaf(u.x, zd[4 * c], yd);
                        yd = fmaf(u.y, zd[4 * c + 1], yd);
                        yd = fmaf(u.z, zd[4 * c + 2], yd);
                        yd = fmaf(u.w, zd[4 * c + 3], yd);
                    }
                }
                y[j] = fmaf(fn, yd + s_b[o0 + j], ys);
            }
            if (part || !accumulate) {
                *reinterpret_cast<float4*>(dst + o0) = make_float4(y[0], y[1], y[2], y[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) emit_out(dst + o0 + j, y[j], 1);
            }
        }
    }
}

// warps 0-2 loaders, 3 MMA, 4.. epilogue: EPI = 4 (one per TMEM lane quarter) or 8 (two per quarter,
// each on every other 32-row chunk of a tile)
constexpr int kGemmLoaders = 96;
constexpr int kGemmMma = 3;
constexpr int kGemmEpi0 = 4;
constexpr int gemm_threads(int epi, int prod = 0) { return 32 * (kGemmEpi0 + epi + prod); }

struct GemmArgs {
    const int4* vr;
    int64_t nv, n_tiles;
    const int32_t* ridx;      // per virtual row v: ridx[v * ridx_stride] = the R-part table row (-1: zeros)
    int ridx_stride;
    const uint16_t* rtbl;     // R-part table (forward: the dst rows z; backward: the rows z of dW), bf16
    int64_t rtbl_rows, out_rows;
    int w_r;                  // R-part width (0: none)
    // backward pass: dW_part += S^T R over all rows of the CTA
    float* dw_part;           // [grid][n_g][w_r]
    int n_g, m_dw;
    uint32_t idesc_dw, dw_col;
    int n_kb_s, n_kb_r, kpad_s, m_blocks, n_feat;
    const float* bias;
    float* out;
    float* vpart;
    int accumulate, tile_n, stages;
    uint32_t idesc, tmem_cols;
    int* status;
    // fused forward (PROD > 0): the S pairs are not read from a buffer but summed by the producer
    // warps: row v's tuples are gidx[vr[v].x ..) (rows of gtbl, width w_s)
    const int32_t* gidx;
    const uint16_t* gtbl;
    int64_t gtbl_rows;
    int w_s;
};

// Forward: D1 = A_src [S_hi; S_lo], D2 = A_dst R (the dst rows), Out = D1 + n (D2 + b).
// Backward pass: D1 = A [S_hi; S_lo] is a dz row (A = a W^T block), and dW += S^T R with R = the
// rows' z, both operands read MN-major from the staged rows, accumulated in TMEM over the CTA's tiles.
// PROD > 0 (forward only): PROD producer warps after the epilogue warps compute each tile's S pairs
// (the gather-sum of seg_sum_kernel: lane groups of w_s / 8 lanes own a row, up to kUnroll row loads
// in flight per lane) and write them straight into the stage (128B swizzle), so the pairs never
// touch global memory.
template <bool BWD, int EPI, int PROD = 0>
__global__ void __launch_bounds__(gemm_threads(EPI, PROD), 1)
agg_gemm_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap smap,
                const __grid_constant__ GemmArgs a) {
    extern __shared__ uint8_t dyn_smem[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~(uintptr_t)1023);
    const int N = a.tile_n;
    const int n_kb = a.n_kb_s + (BWD ? 0 : a.n_kb_r);  // K blocks of A (the backward's R feeds dW only)
    const uint32_t a_bytes = (uint32_t)n_kb * a.m_blocks * 16384u;
    const uint32_t blk = (uint32_t)N * 128u;
    const uint32_t stage_bytes = (uint32_t)(2 * a.n_kb_s + a.n_kb_r) * blk;
    const uint32_t s_bytes = (uint32_t)(2 * a.n_kb_s) * blk;  // TMA bytes of one stage
    uint8_t* a_smem = base;
    uint8_t* st_smem = base + a_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(st_smem + (size_t)a.stages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + a.stages;
    uint64_t* tfull = bars + 2 * a.stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* wbar = tempty + 2;
    uint64_t* drain = wbar + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) {
            // the loaders' copies + the TMA's bytes, or + every producer thread (fused)
            mbar_init(smem_u32(&full[s]), kGemmLoaders + (PROD > 0 ? 32 * PROD : 1));
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&tfull[i]), 1);
            mbar_init(smem_u32(&tempty[i]), 32 * EPI);
        }
        mbar_init(smem_u32(wbar), 1);
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (PROD > 0 && a.w_s < a.kpad_s) {
        // fused: the K padding of the S blocks (columns w_s .. kpad_s of each half) is never written
        // by the producers and must read as zeros
        const int pc0 = a.w_s >> 3, pcn = (a.kpad_s - a.w_s) >> 3;  // 16-byte chunks per row
        const int per_stage = 2 * N * pcn;
        for (int i = tid; i < a.stages * per_stage; i += blockDim.x) {
            const int s = i / per_stage, rem = i - s * per_stage;
            const int hl = rem / (N * pcn), rem2 = rem - hl * N * pcn;
            const int r = rem2 / pcn, c = pc0 + (rem2 - r * pcn);
            const uint32_t off = (uint32_t)(hl * a.n_kb_s + (c >> 3)) * blk + (uint32_t)r * 128u +
                                 ((((uint32_t)c & 7u) ^ ((uint32_t)r & 7u)) << 4);
            st_shared_v4(smem_u32(st_smem + (size_t)s * stage_bytes) + off, 0u, 0u, 0u, 0u);
        }
        fence_proxy_async();
    }
    if (a.w_r > 0 && a.w_r < 64 * a.n_kb_r) {
        // the columns w_r .. 64 n_kb_r of the R block are never copied and must read as zeros (the
        // forward's K padding: stale shared memory of an earlier kernel could hold NaN patterns, and
        // 0 x NaN is NaN)
        const int rc0 = a.w_r >> 3, rcn = 8 * a.n_kb_r - rc0;  // 16-byte chunks per row
        const int per_stage = N * rcn;
        for (int i = tid; i < a.stages * per_stage; i += blockDim.x) {
            const int s = i / per_stage, rem = i - s * per_stage;
            const int r = rem / rcn, c = rc0 + (rem - r * rcn);
            const uint32_t off = (uint32_t)(2 * a.n_kb_s + (c >> 3)) * blk + (uint32_t)r * 128u +
                                 ((((uint32_t)c & 7u) ^ ((uint32_t)r & 7u)) << 4);
            st_shared_v4(smem_u32(st_smem + (size_t)s * stage_bytes) + off, 0u, 0u, 0u, 0u);
        }
        fence_proxy_async();
    }
    if (warp == kGemmMma) tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t buf_cols = (BWD ? 1u : 2u) * a.m_blocks * N;  // D1 (and D2) of one accumulator buffer

    if (tid < kGemmLoaders) {
        // ------------------------------------------------------------------ loaders
        // dst rows: a row is copied by rch = w_r / 8 lanes (16 bytes each, at most 32); the tile's
        // dst row indices are loaded for the next tile while this one's copies are issued
        const int rch = a.w_r >> 3;
        const int rsh = rch > 0 ? 31 - __clz(rch) : 0;  // rch is a power of two
        const int lw = tid >> 5;                         // loader warp 0..2
        const int rpw = rch > 0 ? 32 >> rsh : 0;         // rows per warp instruction
        const int rsub = rch > 0 ? lane >> rsh : 0, c = rch > 0 ? lane & (rch - 1) : 0;
        int hrow_n[kMaxMeta];                            // lane l: dst row of tile row 32 i + l
        auto load_rows = [&](int64_t tile) {
#pragma unroll
            for (int i = 0; i < kMaxMeta; ++i) {
                const int64_t v = tile * N + 32 * i + lane;
                hrow_n[i] = (rch > 0 && tile < a.n_tiles && 32 * i < N && v < a.nv) ? __ldg(a.ridx + v * a.ridx_stride) : -1;
            }
        };
        load_rows(blockIdx.x);
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++lt) {
            const int s = lt % a.stages;
            const uint32_t use = (uint32_t)(lt / a.stages);
            int hrow[kMaxMeta];
#pragma unroll
            for (int i = 0; i < kMaxMeta; ++i) hrow[i] = hrow_n[i];
            load_rows(tile + gridDim.x);
            if (!mbar_wait(smem_u32(&empty[s]), (use & 1u) ^ 1u, a.status, abort_flag)) break;
            const uint32_t sb = smem_u32(st_smem + (size_t)s * stage_bytes);
            const int64_t v0 = tile * N;
            if (PROD == 0 && tid == 0) {
                mbar_arrive_expect_tx(smem_u32(&full[s]), s_bytes);
                for (int hl = 0; hl < 2; ++hl)
                    for (int kb = 0; kb < a.n_kb_s; ++kb)
                        tma_load_2d(sb + (uint32_t)(hl * a.n_kb_s + kb) * blk, &smap, hl * a.kpad_s + kb * 64, (int)v0,
                                    smem_u32(&full[s]));
            }
            // rows past the end and empty rows are zero-filled by the copy
            const uint32_t rb = sb + (uint32_t)(2 * a.n_kb_s) * blk;
            if (rch > 0) {
                for (int r0 = lw * rpw; r0 < N; r0 += 3 * rpw) {
                    const int r = r0 + rsub;
                    int hr = -1;
#pragma unroll
                    for (int i = 0; i < kMaxMeta; ++i) {
                        const int h = __shfl_sync(0xffffffffu, hrow[i], r & 31);
                        if (i == (r >> 5)) hr = h;
                    }
                    const uint32_t dst = rb + (uint32_t)(c >> 3) * blk + (uint32_t)r * 128u +
                                         ((((uint32_t)c & 7u) ^ ((uint32_t)r & 7u)) << 4);
                    const bool ok = hr >= 0 && in_bounds(hr, a.rtbl_rows, a.status);
                    const uint16_t* src = ok ? a.rtbl + (int64_t)hr * a.w_r + 8 * c : a.rtbl;
                    cp_async_16(dst, src, ok ? 16u : 0u);
                }
            }
            cp_async_mbar_arrive_noinc(smem_u32(&full[s]));
        }
        cp_async_wait<0>();
    } else if (warp == kGemmMma) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t wb = smem_u32(wbar);
            mbar_arrive_expect_tx(wb, a_bytes);
            for (int kb = 0; kb < n_kb; ++kb)
                for (int mb = 0; mb < a.m_blocks; ++mb)
                    tma_load_2d(smem_u32(a_smem + (size_t)(kb * a.m_blocks + mb) * 16384u), &amap, kb * 64, mb * 128, wb);
            bool ok = mbar_wait(wb, 0, a.status, abort_flag);
            tc_fence_after();
            int lt = 0;
            for (int64_t tile = blockIdx.x; tile < a.n_tiles && ok; tile += gridDim.x, ++lt) {
                const int s = lt % a.stages;
                const uint32_t use = (uint32_t)(lt / a.stages);
                const int acc = lt & 1;
                const uint32_t ause = (uint32_t)(lt >> 1);
                if (!mbar_wait(smem_u32(&tempty[acc]), (ause & 1u) ^ 1u, a.status, abort_flag)) { ok = false; break; }
                if (!mbar_wait(smem_u32(&full[s]), use & 1u, a.status, abort_flag)) { ok = false; break; }
                fence_proxy_async();  // the cp.async rows were written through the generic proxy
                tc_fence_after();
                const uint32_t sb = smem_u32(st_smem + (size_t)s * stage_bytes);
                const uint32_t d1 = tmem_base + (uint32_t)acc * buf_cols;
                for (int mb = 0; mb < a.m_blocks; ++mb) {
                    uint32_t acc1 = 0, acc2 = 0;
                    for (int kb = 0; kb < n_kb; ++kb) {
                        const uint32_t ab = smem_u32(a_smem + (size_t)(kb * a.m_blocks + mb) * 16384u);
                        const bool src = kb < a.n_kb_s;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint64_t adesc = sw128_kmajor_desc(ab + k * 32);
                            if (src) {
#pragma unroll
                                for (int hl = 0; hl < 2; ++hl) {
                                    const uint64_t bdesc =
                                        sw128_kmajor_desc(sb + (uint32_t)(hl * a.n_kb_s + kb) * blk + k * 32);
                                    mma_bf16(d1 + (uint32_t)mb * N, adesc, bdesc, a.idesc, acc1);
                                    acc1 = 1;
                                }
                            } else {
                                const uint64_t bdesc = sw128_kmajor_desc(
                                    sb + (uint32_t)(2 * a.n_kb_s + kb - a.n_kb_s) * blk + k * 32);
                                mma_bf16(d1 + (uint32_t)(a.m_blocks + mb) * N, adesc, bdesc, a.idesc, acc2);
                                acc2 = 1;
                            }
                        }
                    }
                }
                if (BWD) {
                    // dW += S^T R: K = the tile's rows (16 per instruction), M = S features (128 per
                    // block: two 64-column blocks of S), N = the R width
                    const uint32_t rb = sb + (uint32_t)(2 * a.n_kb_s) * blk;
                    for (int step = 0; step < N / 16; ++step)
                        for (int mbw = 0; mbw < a.m_dw; ++mbw)
#pragma unroll
                            for (int hl = 0; hl < 2; ++hl) {
                                const uint32_t accw = (lt > 0 || step > 0 || hl > 0) ? 1u : 0u;
                                const uint64_t ad = sw128_mnmajor_desc(
                                    sb + (uint32_t)(hl * a.n_kb_s + 2 * mbw) * blk + (uint32_t)step * 2048u, blk);
                                const uint64_t bd = sw128_mnmajor_desc(rb + (uint32_t)step * 2048u, blk);
                                mma_bf16(tmem_base + a.dw_col + (uint32_t)mbw * a.w_r, ad, bd, a.idesc_dw, accw);
                            }
                }
                mma_commit(smem_u32(&empty[s]));
                mma_commit(smem_u32(&tfull[acc]));
            }
            mma_commit(smem_u32(drain));
            mbar_wait(smem_u32(drain), 0, a.status, abort_flag);
        }
        __syncwarp();
    } else if (PROD > 0 && warp >= kGemmEpi0 + EPI) {
        // ------------------------------------------------------------------ producers (fused)
        const int pw = warp - (kGemmEpi0 + EPI);
        const int L = a.w_s >> 3, lsh = 31 - __clz(L), G = 32 >> lsh;
        const int grp = lane >> lsh, ch = lane & (L - 1);
        const uint4* __restrict__ gbase = reinterpret_cast<const uint4*>(a.gtbl) + ch;
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++lt) {
            const int s = lt % a.stages;
            const uint32_t use = (uint32_t)(lt / a.stages);
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&empty[s]), (use & 1u) ^ 1u, a.status, abort_flag))) break;
            const uint32_t sb = smem_u32(st_smem + (size_t)s * stage_bytes);
            const int64_t v0 = tile * N;
            // steps of G rows, every PROD-th step to this warp
            for (int k = pw; k * G < N; k += PROD) {
                const int j = k * G + grp;
                const int64_t v = v0 + j;
                const int4 m = (j < N && v < a.nv) ? __ldg(a.vr + v) : make_int4(0, 0, -1, -1);
                const int n = m.y > 0 ? m.y : 0;
                const int nmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)n);
                float acc[8], cmp[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = cmp[i] = 0.f;
                for (int t0 = 0; t0 < nmax; t0 += kUnroll) {
                    const int slots = min(kUnroll, nmax - t0);  // warp-uniform
                    uint4 u[kUnroll];
#pragma unroll
                    for (int q = 0; q < kUnroll; ++q) {
                        if (q >= slots) break;
                        u[q] = make_uint4(0u, 0u, 0u, 0u);
                        if (t0 + q < n) {
                            const int r = __ldg(a.gidx + m.x + t0 + q);
                            if (in_bounds(r, a.gtbl_rows, a.status)) u[q] = __ldg(gbase + (int64_t)r * L);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kUnroll; ++q) {
                        if (q >= slots) break;
                        add8(acc, cmp, u[q], false);
                    }
                }
                if (j < N) store_pair(sb, blk, a.n_kb_s, 0, j, ch, acc);
            }
            // the stage's rows were written through the generic proxy: visible to the tensor cores
            fence_proxy_async();
            mbar_arrive(smem_u32(&full[s]));
        }
    } else if (warp >= kGemmEpi0) {
        // ------------------------------------------------------------------ epilogue
        // EH warps per TMEM lane quarter, warp eh taking 32-row chunks eh, eh + EH, ... of a tile
        constexpr int EH = EPI / 4;
        const int q = warp & 3;
        const int eh = (warp - kGemmEpi0) >> 2;
        const bool has_r = !BWD && a.n_kb_r > 0;
        float bias_r[2];
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
            const int o = mb * 128 + 32 * q + lane;
            bias_r[mb] = (a.bias && mb < a.m_blocks && o < a.n_feat) ? a.bias[o] : 0.f;
        }
        // this warp's chunks of the next tile (lane l of register c: row 32 (EH c + eh) + l) load
        // during this one
        int4 meta_n[kMaxMeta / EH];
        auto load_meta = [&](int64_t tile) {
#pragma unroll
            for (int c = 0; c < kMaxMeta / EH; ++c) {
                const int rr = 32 * (EH * c + eh);
                const int64_t v = tile * N + rr + lane;
                meta_n[c] = (tile < a.n_tiles && rr < N && v < a.nv) ? __ldg(a.vr + v) : make_int4(0, 0, -1, -1);
            }
        };
        load_meta(blockIdx.x);
        int lt = 0;
        for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++lt) {
            const int acc = lt & 1;
            const uint32_t ause = (uint32_t)(lt >> 1);
            int4 meta[kMaxMeta / EH];
#pragma unroll
            for (int c = 0; c < kMaxMeta / EH; ++c) meta[c] = meta_n[c];
            load_meta(tile + gridDim.x);
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[acc]), ause & 1u, a.status, abort_flag))) break;
            tc_fence_after();
            const int64_t v0 = tile * N;
#pragma unroll
            for (int c = 0; c < kMaxMeta / EH; ++c) {
                const int rr = 32 * (EH * c + eh);
                const int64_t vb = v0 + rr;
                if (rr >= N || vb >= a.nv) break;
                const int4 mt = meta[c];
                // chunks of 32 consecutive whole rows, or of 32 consecutive chunk partials (the chunks of
                // one long row), store row after row without per-row bookkeeping
                const int row0 = __shfl_sync(0xffffffffu, mt.z, 0);
                const int part0 = __shfl_sync(0xffffffffu, mt.w, 0);
                const bool whole = __all_sync(0xffffffffu, mt.w < 0 && mt.z == row0 + lane);
                const bool parts = !whole && __all_sync(0xffffffffu, mt.w >= 0 && mt.w == part0 + lane);
                // each lane's row as one word for the general path: the output row, -(slot + 1) for a
                // chunk partial, or INT_MIN for none
                const int myoff = (mt.z < 0 || !a.out) ? INT_MIN : (mt.w >= 0 ? -(mt.w + 1) : mt.z);
                const bool whole_ok = whole && a.out && in_bounds(row0 + 31, a.out_rows, a.status) &&
                                      in_bounds(row0, a.out_rows, a.status);
                for (int mb = 0; mb < a.m_blocks; ++mb) {
                    if (mb * 128 + 32 * q >= a.n_feat) continue;
                    const int o = mb * 128 + 32 * q + lane;
                    const bool o_ok = o < a.n_feat;
                    const float bo = mb == 0 ? bias_r[0] : bias_r[1];
                    const uint32_t ta = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)acc * buf_cols +
                                        (uint32_t)mb * N + (uint32_t)rr;
                    // eight rows (TMEM columns) at a time in a loop that is not unrolled: the three store
                    // paths stay small enough for the instruction cache (fully unrolled, chunks mixing
                    // whole rows and chunk partials stalled on instruction fetch)
#pragma unroll 1
                    for (int jp = 0; jp < 32; jp += 8) {
                        uint32_t v1[8], v2[8];
                        tmem_ld_32x32b_x8(ta + (uint32_t)jp, v1);
                        if (has_r) tmem_ld_32x32b_x8(ta + (uint32_t)a.m_blocks * N + (uint32_t)jp, v2);
                        tmem_ld_wait();
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            tmem_ld_after(v1[u]);
                            if (has_r) tmem_ld_after(v2[u]);
                        }
                        float y[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            y[u] = __uint_as_float(v1[u]);
                            if (!BWD) {
                                const float nj = (float)__shfl_sync(0xffffffffu, mt.y, jp + u);
                                y[u] += nj * ((has_r ? __uint_as_float(v2[u]) : 0.f) + bo);
                            }
                        }
                        if (whole_ok) {
                            float* dst = a.out + (int64_t)(row0 + jp) * a.n_feat + o;
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (o_ok) emit_out(dst + (int64_t)u * a.n_feat, y[u], a.accumulate);
                        } else if (parts && a.out) {
                            float* dst = a.vpart + (int64_t)(part0 + jp) * a.n_feat + o;
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (o_ok) __stcg(dst + (int64_t)u * a.n_feat, y[u]);
                        } else {
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const int off = __shfl_sync(0xffffffffu, myoff, jp + u);
                                if (o_ok && a.out && off != INT_MIN) {
                                    if (off < 0) __stcg(a.vpart + (int64_t)(-off - 1) * a.n_feat + o, y[u]);
                                    else if (in_bounds(off, a.out_rows, a.status))
                                        emit_out(a.out + (int64_t)off * a.n_feat + o, y[u], a.accumulate);
                                }
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&tempty[acc]));
        }
        if (BWD && eh == 0) {
            // this CTA's dW partial (TMEM lane = S feature, columns = R features)
            if (__all_sync(0xffffffffu, mbar_wait(smem_u32(drain), 0, a.status, abort_flag))) {
                tc_fence_after();
                for (int mbw = 0; mbw < a.m_dw; ++mbw) {
                    const int g = mbw * 128 + 32 * q + lane;
                    float* dst = a.dw_part + ((int64_t)blockIdx.x * a.n_g + g) * a.w_r;
                    for (int c = 0; c < a.w_r / 32; ++c) {
                        uint32_t v[32];
                        tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(32 * q) << 16) + a.dw_col + (uint32_t)mbw * a.w_r +
                                               (uint32_t)(32 * c), v);
                        tmem_ld_wait();
                        if (g < a.n_g) {
#pragma unroll
                            for (int j = 0; j < 32; j += 4)
                                *reinterpret_cast<float4*>(dst + 32 * c + j) =
                                    make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kGemmMma) {
        tc_fence_after();
        tmem_dealloc(tmem_base, a.tmem_cols);
    }
}

// ------------------------------------------------------------------------------ virtual rows
// Sorted keys (values in [0, R)): beg[k] / end[k] = the tuple range of row k (0 / 0 when absent).
// One thread per 4 tuples, all loads issued before the first store (one memory round trip).
__global__ void vr_bounds_kernel(const int32_t* __restrict__ key, int64_t m, int32_t* __restrict__ beg,
                                 int32_t* __restrict__ end) {
    const int64_t t0 = (blockIdx.x * (int64_t)blockDim.x) * 4 + threadIdx.x;
    int32_t k[4], kp[4], kn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t t = t0 + (int64_t)i * blockDim.x;
        k[i] = t < m ? __ldg(key + t) : 0;
        kp[i] = (t < m && t > 0) ? __ldg(key + t - 1) : ~k[i];
        kn[i] = t + 1 < m ? __ldg(key + t + 1) : ~k[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t t = t0 + (int64_t)i * blockDim.x;
        if (t >= m) continue;
        if (kp[i] != k[i]) beg[k[i]] = (int32_t)t;
        if (kn[i] != k[i]) end[k[i]] = (int32_t)(t + 1);
    }
}

// Unsorted keys: 1 at the first tuple of every run of equal keys.
__global__ void vr_run_flags_kernel(const int32_t* __restrict__ key, int64_t m, int32_t* flag) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
        flag[t] = (t == 0 || key[t - 1] != key[t]) ? 1 : 0;
}

// Run r (exclusive scan of the flags gives the run of each start): its tuple range and key.
__global__ void vr_runs_kernel(const int32_t* __restrict__ key, int64_t m, const int32_t* __restrict__ rid_excl,
                               int32_t* beg, int32_t* end, int32_t* rkey) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = key[t];
        const bool start = t == 0 || key[t - 1] != k;
        const int32_t r = rid_excl[t] - (start ? 0 : 1);
        if (start) {
            beg[r] = (int32_t)t;
            rkey[r] = k;
        }
        if (t == m - 1 || key[t + 1] != k) end[r] = (int32_t)(t + 1);
    }
}

// Chunks per row (every row of a sorted list gets one, empty or not), chunk partials per row (rows
// of one chunk need none), and the split flag.
__global__ void vr_count_kernel(const int32_t* __restrict__ beg, const int32_t* __restrict__ end, int64_t R,
                                int32_t* nch, int32_t* npart, int32_t* split, int32_t* cnt_out, int32_t* long_rows) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t cnt = end[r] - beg[r];
        if (cnt_out) cnt_out[r] = cnt;
        const int32_t c = cnt > kChunk ? (cnt + kChunk - 1) / kChunk : 1;
        nch[r] = c;
        npart[r] = c > 1 ? c : 0;
        split[r] = c > 1 ? 1 : 0;
        if (c > kFixChunk) *long_rows = 1;  // a row the fix-up cuts again (host-built jobs)
    }
}

__global__ void vr_fill_kernel(const int32_t* __restrict__ beg, const int32_t* __restrict__ end,
                               const int32_t* __restrict__ rkey, int64_t R, const int32_t* __restrict__ voff,
                               const int32_t* __restrict__ poff, const int32_t* __restrict__ soff, int4* vr, int4* splits) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = beg[r], cnt = end[r] - b;
        const int32_t c = cnt > kChunk ? (cnt + kChunk - 1) / kChunk : 1;
        const int32_t row = rkey ? rkey[r] : (int32_t)r;
        for (int32_t i = 0; i < c; ++i)
            vr[voff[r] + i] = make_int4(b + i * kChunk, max(0, min(kChunk, cnt - i * kChunk)), row, c > 1 ? poff[r] + i : -1);
        if (c > 1) splits[soff[r]] = make_int4(row, poff[r], c, -1);
    }
}

// ------------------------------------------------------------------------------ fix-up
// One block per job {row, first partial, count, level-2 slot or -1}: the partials are added in
// order (8 warps take every 8th, then the warps' sums are added in warp order), into the level-2
// slot or the output row. A warp fetches its next four partials together (one round trip for four:
// a 256-partial job took 32 dependent round trips per warp, about 25 us per launch).
__global__ void __launch_bounds__(256) agg_fix_kernel(const int4* __restrict__ jobs, int64_t n_jobs,
                                                      const float* __restrict__ part, float* part2, float* out, int F,
                                                      int accumulate, int kahan, int64_t out_rows, int* status) {
    __shared__ float4 red[8][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int F4 = F >> 2;
    for (int64_t jb = blockIdx.x; jb < n_jobs; jb += gridDim.x) {
        const int4 j = jobs[jb];
        for (int c4 = lane; c4 < F4; c4 += 32) {
            float s[4] = {0.f, 0.f, 0.f, 0.f}, cm[4] = {0.f, 0.f, 0.f, 0.f};
            const float4* src = reinterpret_cast<const float4*>(part + (int64_t)j.y * F) + c4;
            for (int i0 = warp; i0 < j.z; i0 += 32) {
                float4 v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    v[q] = i0 + 8 * q < j.z ? __ldcg(src + (int64_t)(i0 + 8 * q) * F4) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (i0 + 8 * q >= j.z) break;
                    const float vv[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (kahan) kahan_add(s[e], cm[e], vv[e]);
                        else s[e] += vv[e];
                    }
                }
            }
            red[warp][c4] = make_float4(s[0] - cm[0], s[1] - cm[1], s[2] - cm[2], s[3] - cm[3]);
        }
        __syncthreads();
        for (int c4 = threadIdx.x; c4 < F4; c4 += blockDim.x) {
            float s[4] = {0.f, 0.f, 0.f, 0.f}, cm[4] = {0.f, 0.f, 0.f, 0.f};
            for (int w = 0; w < 8; ++w) {
                const float4 v = red[w][c4];
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (kahan) kahan_add(s[e], cm[e], vv[e]);
                    else s[e] += vv[e];
                }
            }
            float4 res = make_float4(s[0] - cm[0], s[1] - cm[1], s[2] - cm[2], s[3] - cm[3]);
            if (j.w >= 0) {
                reinterpret_cast<float4*>(part2 + (int64_t)j.w * F)[c4] = res;
            } else if (in_bounds(j.x, out_rows, status)) {
                float4* dst = reinterpret_cast<float4*>(out + (int64_t)j.x * F) + c4;
                if (accumulate) {
                    const float4 o = *dst;
                    res = make_float4(o.x + res.x, o.y + res.y, o.z + res.z, o.w + res.w);
                }
                *dst = res;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------ operands
// A of the forward: A[o][k] = W[o][col(k)] with every Concat part padded to `kpad` columns.
__global__ void pack_a_fwd_kernel(const void* W, int w_bf16, int d_out, int d_in, int d, int kpad, int rows_pad,
                                  int cols, uint16_t* out) {
    const int n = rows_pad * cols;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = i / cols, k = i - o * cols;
        const int part = k / kpad, kk = k - part * kpad;
        uint16_t v = 0;
        if (o < d_out && kk < d && part * d + kk < d_in) {
            const int col = part * d + kk;
            v = w_bf16 ? reinterpret_cast<const uint16_t*>(W)[o * d_in + col]
                       : __bfloat16_as_ushort(__float2bfloat16_rn(reinterpret_cast<const float*>(W)[o * d_in + col]));
        }
        out[i] = v;
    }
}

// A of a backward pass: A[i][o] = W[o][col0 + i] (i < d, o < d_out), zero-padded.
__global__ void pack_a_bwd_kernel(const void* W, int w_bf16, int d_out, int d_in, int col0, int d, int rows_pad,
                                  int cols, uint16_t* out) {
    const int n = rows_pad * cols;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = i / cols, o = i - r * cols;
        uint16_t v = 0;
        if (r < d && o < d_out) {
            const int idx = o * d_in + col0 + r;
            v = w_bf16 ? reinterpret_cast<const uint16_t*>(W)[idx]
                       : __bfloat16_as_ushort(__float2bfloat16_rn(reinterpret_cast<const float*>(W)[idx]));
        }
        out[i] = v;
    }
}

// dW[g][col0 + i] = sum over CTAs (in order) of part[c][g][i].
// dW slice = sum over the CTAs' partials, in CTA order: 32 elements per block, warp w adds CTAs w,
// w + 8, ... (8 independent chains of loads), then the 8 warps' sums are added in warp order.
__global__ void __launch_bounds__(256) agg_reduce_dw_kernel(const float* __restrict__ part, int grid, int n_g,
                                                            int d_z, float* dW, int d_in, int col0) {
    __shared__ float red[8][32];
    const int64_t n = (int64_t)n_g * d_z;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = blockIdx.x * 32ll + lane;
    float s = 0.f;
    if (i < n)
        for (int c = w; c < grid; c += 8) s += part[(int64_t)c * n + i];
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && i < n) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += red[k][lane];
        const int64_t g = i / d_z, k = i - g * d_z;
        dW[g * d_in + col0 + k] = t;
    }
}


// dOut -> its bf16 copy (round to nearest even), and per block the partial of
// db_b = sum_k cnt_b[k] dOut[k] (the SUM backward's bias gradient, f32 from the unrounded dOut) for up
// to kDbBranches branches. Block i takes a contiguous range of rows; lanes hold float4 columns; the
// warps' partials are added in warp order, the blocks' later in block order (deterministic).
constexpr int kDbBranches = 4;
struct CntSet {
    const int32_t* c[kDbBranches];
    int n;
};

__global__ void __launch_bounds__(256) dout_prep_kernel(const float* __restrict__ dout, int64_t n_out, int d_out,
                                                        CntSet cs, int64_t rows_per_block, uint16_t* __restrict__ out_bf,
                                                        float* __restrict__ db_part) {
    __shared__ float4 red[8][kDbBranches][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int F4 = d_out >> 2;               // float4 per row (2..64)
    const int LR = F4 < 32 ? F4 : 32;        // lanes per row
    const int RPW = 32 / LR;                 // rows per warp step
    const int FPL = F4 / LR;                 // float4 per lane (1 or 2)
    const int g = lane / LR, c0 = lane - g * LR;
    float4 acc[kDbBranches][2];
#pragma unroll
    for (int b = 0; b < kDbBranches; ++b) acc[b][0] = acc[b][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t r0 = blockIdx.x * rows_per_block, r1 = imin64(n_out, r0 + rows_per_block);
    for (int64_t r = r0 + warp * RPW + g; r < r1; r += 8 * RPW) {
        int32_t cnt[kDbBranches];
#pragma unroll
        for (int b = 0; b < kDbBranches; ++b) cnt[b] = b < cs.n ? __ldg(cs.c[b] + r) : 0;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (j >= FPL) break;
            const int c = c0 + j * LR;
            const float4 v = __ldg(reinterpret_cast<const float4*>(dout + r * d_out) + c);
            *reinterpret_cast<uint2*>(out_bf + r * d_out + 4 * c) = make_uint2(tc::pack_bf16x2(v.x, v.y), tc::pack_bf16x2(v.z, v.w));
#pragma unroll
            for (int b = 0; b < kDbBranches; ++b) {
                const float w = (float)cnt[b];
                acc[b][j].x = fmaf(w, v.x, acc[b][j].x);
                acc[b][j].y = fmaf(w, v.y, acc[b][j].y);
                acc[b][j].z = fmaf(w, v.z, acc[b][j].z);
                acc[b][j].w = fmaf(w, v.w, acc[b][j].w);
            }
        }
    }
    // the row groups of the warp, then the warps
    for (int off = LR; off < 32; off <<= 1) {
#pragma unroll
        for (int b = 0; b < kDbBranches; ++b)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                acc[b][j].x += __shfl_xor_sync(0xffffffffu, acc[b][j].x, off);
                acc[b][j].y += __shfl_xor_sync(0xffffffffu, acc[b][j].y, off);
                acc[b][j].z += __shfl_xor_sync(0xffffffffu, acc[b][j].z, off);
                acc[b][j].w += __shfl_xor_sync(0xffffffffu, acc[b][j].w, off);
            }
    }
    if (g == 0) {
#pragma unroll
        for (int b = 0; b < kDbBranches; ++b)
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if (j < FPL) red[warp][b][c0 + j * LR] = acc[b][j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cs.n * F4; i += blockDim.x) {
        const int b = i / F4, c = i - b * F4;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int w = 0; w < 8; ++w) {
            const float4 v = red[w][b][c];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        reinterpret_cast<float4*>(db_part + ((int64_t)blockIdx.x * kDbBranches + b) * d_out)[c] = s;
    }
}

// db_b[f] = sum over blocks (in order, compensated) of the partials ([block][branch][d_out], or
// [block][d_out] for b = -1).
// (32 features per block; warp w takes blocks w, w + 8, ... compensated, then the 8 warps' sums are
// added in warp order, compensated)
__global__ void __launch_bounds__(256) db_reduce_kernel(const float* __restrict__ part, int blocks, int d_out, int b,
                                                        float* db) {
    __shared__ float red[8][32][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int f = blockIdx.x * 32 + lane;
    float s = 0.f, c = 0.f;
    if (f < d_out)
        for (int k = w; k < blocks; k += 8)
            kahan_add(s, c, part[(b < 0 ? (int64_t)k : ((int64_t)k * kDbBranches + b)) * d_out + f]);
    red[w][lane][0] = s;
    red[w][lane][1] = c;
    __syncthreads();
    if (w == 0 && f < d_out) {
        float t = 0.f, tc = 0.f;
        for (int k = 0; k < 8; ++k) kahan_add(t, tc, red[k][lane][0] - red[k][lane][1]);
        db[f] = t - tc;
    }
}

inline int grid_for(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 16));
}

inline bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

// Fix-up jobs of the split rows {row, first partial, chunks} (host copy): one job per row of at most
// kFixChunk chunks, otherwise one per kFixChunk chunks into level-2 slots plus one level-2 job.
relnn_status make_fix_jobs(VRows& V, const int4* d_splits, int64_t n_split, cudaStream_t st) {
    V.n_fix1 = V.n_fix2 = V.n_l2 = 0;
    if (n_split == 0) return RELNN_OK;
    std::vector<int4> sp((size_t)n_split);
    RELNN_CUDA(cudaMemcpyAsync(sp.data(), d_splits, sizeof(int4) * n_split, cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaStreamSynchronize(st));
    std::vector<int4> j1, j2;
    int64_t l2 = 0;
    for (const int4& sj : sp) {
        if (sj.z <= kFixChunk) {
            j1.push_back(make_int4(sj.x, sj.y, sj.z, -1));
        } else {
            const int nc = (sj.z + kFixChunk - 1) / kFixChunk;
            for (int c = 0; c < nc; ++c)
                j1.push_back(make_int4(sj.x, sj.y + c * kFixChunk, std::min(kFixChunk, sj.z - c * kFixChunk), (int)(l2 + c)));
            j2.push_back(make_int4(sj.x, (int)l2, nc, -1));
            l2 += nc;
        }
    }
    RELNN_TRY(V.fix1.alloc_nosync(sizeof(int4) * j1.size(), st));
    RELNN_CUDA(cudaMemcpyAsync(V.fix1.p, j1.data(), sizeof(int4) * j1.size(), cudaMemcpyHostToDevice, st));
    if (!j2.empty()) {
        RELNN_TRY(V.fix2.alloc_nosync(sizeof(int4) * j2.size(), st));
        RELNN_CUDA(cudaMemcpyAsync(V.fix2.p, j2.data(), sizeof(int4) * j2.size(), cudaMemcpyHostToDevice, st));
    }
    RELNN_CUDA(cudaStreamSynchronize(st));  // the job vectors are copied from, and the buffers are shared
    V.n_fix1 = (int64_t)j1.size();
    V.n_fix2 = (int64_t)j2.size();
    V.n_l2 = l2;
    return RELNN_OK;
}

// Builds (once) the virtual rows of an ordered tuple list: `sorted` = every key in 0..R-1 occupies
// one contiguous run of the list (the keys ascend, or each key's tuples are grouped) and the rows
// come in key order, every row with at least one virtual row (an empty row writes zeros);
// otherwise the rows are the runs of equal keys in list order. A sorted list takes one synchronisation (the
// totals; buffers are sized by bounds and allocated before it), plus one when rows were cut.
relnn_status ensure_vrows(VRows& V, const int32_t* key, int64_t m, int64_t R, bool sorted, cudaStream_t st) {
    if (V.nv >= 0) return RELNN_OK;
    DevBuf beg, end, rkey, flag;
    int64_t rows = R;
    if (!sorted) {
        RELNN_TRY(flag.alloc_tmp(sizeof(int32_t) * (m + 1), st));
        if (m > 0) { vr_run_flags_kernel<<<grid_for(m), 256, 0, st>>>(key, m, flag.as<int32_t>()); note_launch(); }
        RELNN_TRY(exclusive_scan<int32_t>(flag.as<int32_t>(), flag.as<int32_t>(), m, flag.as<int32_t>() + m, st));
        int32_t nr = 0;
        RELNN_CUDA(cudaMemcpyAsync(&nr, flag.as<int32_t>() + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        RELNN_CUDA(cudaStreamSynchronize(st));
        rows = nr;
    }
    const int64_t r1 = std::max<int64_t>(rows, 1);
    // every row gives ceil(cnt / kChunk) virtual rows (at least one), and a row is cut only when it
    // holds more than kChunk tuples
    const int64_t nv_max = rows + m / kChunk + 1;
    const int64_t ns_max = std::min<int64_t>(r1, m / (kChunk + 1) + 1);
    RELNN_TRY(beg.alloc_tmp(sizeof(int32_t) * r1, st));
    RELNN_TRY(end.alloc_tmp(sizeof(int32_t) * r1, st));
    if (sorted) {
        RELNN_CUDA(cudaMemsetAsync(beg.p, 0, sizeof(int32_t) * r1, st));
        RELNN_CUDA(cudaMemsetAsync(end.p, 0, sizeof(int32_t) * r1, st));
        if (m > 0) { vr_bounds_kernel<<<(unsigned)ceil_div(m, 1024), 256, 0, st>>>(key, m, beg.as<int32_t>(), end.as<int32_t>()); note_launch(); }
    } else {
        RELNN_TRY(rkey.alloc_tmp(sizeof(int32_t) * r1, st));
        if (m > 0) { vr_runs_kernel<<<grid_for(m), 256, 0, st>>>(key, m, flag.as<int32_t>(), beg.as<int32_t>(), end.as<int32_t>(),
                                                               rkey.as<int32_t>()); note_launch(); }
    }
    DevBuf cnts;  // nch | npart | split, each rows + 1 (exclusive scans in place), then the 3 totals
                  // and the long-row flag
    RELNN_TRY(cnts.alloc_tmp(sizeof(int32_t) * (3 * (rows + 1) + 4), st));
    int32_t* nch = cnts.as<int32_t>();
    int32_t* npart = nch + rows + 1;
    int32_t* split = npart + rows + 1;
    int32_t* tot_d = split + rows + 1;
    RELNN_CUDA(cudaMemsetAsync(tot_d + 3, 0, sizeof(int32_t), st));
    if (sorted) RELNN_TRY(V.cnt.alloc_nosync(sizeof(int32_t) * r1, st));
    RELNN_TRY(V.vr.alloc_nosync(sizeof(int4) * nv_max, st));
    // the split rows {row, first partial, chunks, -1}: with no row above kFixChunk chunks they are
    // the fix-up's jobs as they stand (no host pass), so they are written into V.fix1 directly
    RELNN_TRY(V.fix1.alloc_nosync(sizeof(int4) * ns_max, st));
    if (rows > 0) { vr_count_kernel<<<grid_for(rows), 256, 0, st>>>(beg.as<int32_t>(), end.as<int32_t>(), rows, nch, npart, split,
                                                                   sorted ? V.cnt.as<int32_t>() : nullptr, tot_d + 3); note_launch(); }
    RELNN_TRY(exclusive_scan<int32_t>(nch, nch, rows, tot_d, st));
    RELNN_TRY(exclusive_scan<int32_t>(npart, npart, rows, tot_d + 1, st));
    RELNN_TRY(exclusive_scan<int32_t>(split, split, rows, tot_d + 2, st));
    if (rows > 0) { vr_fill_kernel<<<grid_for(rows), 256, 0, st>>>(beg.as<int32_t>(), end.as<int32_t>(),
                                                                  sorted ? nullptr : rkey.as<int32_t>(), rows, nch, npart,
                                                                  split, V.vr.as<int4>(), V.fix1.as<int4>()); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    int32_t tot[4] = {0, 0, 0, 0};
    RELNN_CUDA(cudaMemcpyAsync(tot, tot_d, sizeof(tot), cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaStreamSynchronize(st));
    if (tot[3]) {
        // some row has more than kFixChunk chunks: two-level jobs built on the host from the splits
        DevBuf splits = std::move(V.fix1);
        RELNN_TRY(make_fix_jobs(V, splits.as<int4>(), tot[2], st));
    } else {
        V.n_fix1 = tot[2];
        V.n_fix2 = V.n_l2 = 0;
    }
    V.n_parts = tot[1];
    V.nv = tot[0];
    return RELNN_OK;
}

// Tile rows and pipeline depth: the largest N (128, 64, 32) that leaves two stages in shared
// memory and fits TMEM.
struct AggCfg {
    int N = 0, stages = 0;
    uint32_t tmem_cols = 0, dw_col = 0;
    size_t smem = 0;
};

AggCfg agg_config(int n_kb, int m_blocks, bool bwd, int z_blocks, int m_dw, int d_z) {
    AggCfg c;
    const uint32_t a_bytes = (uint32_t)n_kb * m_blocks * 16384u;
    // two stages at the largest N; a single stage of 32 rows as the last resort (wide A operands)
    const int tries[4][2] = {{128, 2}, {64, 2}, {32, 2}, {32, 1}};
    const int64_t want = tune_get(RELNN_TUNE_AGG_ROWS);  // 0: the largest that fits
    for (const auto& tr : tries) {
        const int N = tr[0];
        if (want != 0 && N > want) continue;
        const size_t stage = (size_t)(2 * n_kb + z_blocks) * N * 128;
        const size_t fixed = 1024 + a_bytes + 512;
        if (fixed + stage > (size_t)kSmemLimit) continue;
        const int stages = (int)std::min<size_t>(4, (kSmemLimit - fixed) / stage);
        const uint32_t cols = 2u * m_blocks * N + (bwd ? (uint32_t)(m_dw * d_z) : 0u);
        if (stages >= tr[1] && cols <= 512) {
            c.N = N;
            c.stages = stages;
            c.dw_col = 2u * m_blocks * N;
            uint32_t t = 32;
            while (t < cols) t <<= 1;
            c.tmem_cols = t;
            c.smem = fixed + (size_t)stages * stage;
            return c;
        }
    }
    return c;
}

template <bool BWD, bool KAHAN, int K1, int K0>
relnn_status launch_agg_t(const CUtensorMap& amap, const AggArgs& a, size_t smem, int grid, cudaStream_t st, int prof) {
    static bool attr_set = false;
    if (!attr_set) {
        RELNN_CUDA(cudaFuncSetAttribute(agg_tc_kernel<BWD, KAHAN, K1, K0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kSmemLimit));
        attr_set = true;
    }
    ProfToken pt = prof_begin(prof, st);
    { agg_tc_kernel<BWD, KAHAN, K1, K0><<<grid, kThreads, smem, st>>>(amap, a); note_launch(); }
    prof_end(pt, st);
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

// The instantiation for the launch's parts: forward (a single-row dst part, then a per-tuple src
// part, or the src part alone), backward src pass (per-tuple dOut rows), backward dst pass (a
// single dOut row per run).
template <bool BWD>
relnn_status launch_agg(const CUtensorMap& amap, const AggArgs& a, bool kahan, size_t smem, int grid, cudaStream_t st,
                        int prof) {
    const bool k1 = a.n_parts == 2 || a.kind[0] == 1;
    const bool k0 = a.n_parts == 2 || a.kind[0] == 0;
    if constexpr (!BWD) {
        if (k1 && k0) return kahan ? launch_agg_t<false, true, 1, 1>(amap, a, smem, grid, st, prof)
                                   : launch_agg_t<false, false, 1, 1>(amap, a, smem, grid, st, prof);
    }
    if (k1) return kahan ? launch_agg_t<BWD, true, 1, 0>(amap, a, smem, grid, st, prof)
                         : launch_agg_t<BWD, false, 1, 0>(amap, a, smem, grid, st, prof);
    return kahan ? launch_agg_t<BWD, true, 0, 1>(amap, a, smem, grid, st, prof)
                 : launch_agg_t<BWD, false, 0, 1>(amap, a, smem, grid, st, prof);
}

// Fix-up of the split rows of one launch: partial rows in p.vpart (level-2 sums after them).
relnn_status agg_fixup(const VRows& V, const float* vpart, float* vpart2, float* out, int F, bool accumulate, bool kahan,
                       int64_t out_rows, int* status, cudaStream_t st) {
    if (!out || V.n_fix1 == 0) return RELNN_OK;
    ProfToken pt = prof_begin(RELNN_PROF_FIXUP, st);
    { agg_fix_kernel<<<(int)std::min<int64_t>(V.n_fix1, 65535), 256, 0, st>>>(V.fix1.as<int4>(), V.n_fix1, vpart, vpart2, out, F,
                                                                            accumulate ? 1 : 0, kahan ? 1 : 0, out_rows, status); note_launch(); }
    if (V.n_fix2 > 0)
        { agg_fix_kernel<<<(int)std::min<int64_t>(V.n_fix2, 65535), 256, 0, st>>>(V.fix2.as<int4>(), V.n_fix2, vpart2, nullptr, out,
                                                                                F, accumulate ? 1 : 0, kahan ? 1 : 0, out_rows, status); note_launch(); }
    prof_end(pt, st);
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Epilogue warps of agg_gemm_kernel (RELNN_TUNE_AGG_EPI; 8 by default).
int gemm_epi() { return tune_get(RELNN_TUNE_AGG_EPI) == 4 ? 4 : 8; }

// Tile rows and stages of agg_gemm_kernel (two stages at the largest N). Backward: A holds only the
// S part's K blocks, and TMEM also holds dW (m_dw blocks of w_r columns).
AggCfg gemm_config(int n_kb_s, int n_kb_r, int m_blocks, bool bwd = false, int m_dw = 0, int w_r = 0) {
    AggCfg c;
    const uint32_t a_bytes = (uint32_t)(n_kb_s + (bwd ? 0 : n_kb_r)) * m_blocks * 16384u;
    const int64_t want = tune_get(RELNN_TUNE_AGG_ROWS);
    for (int N : {128, 64, 32}) {
        if (want != 0 && N > want) continue;
        const size_t stage = (size_t)(2 * n_kb_s + n_kb_r) * N * 128;
        const size_t fixed = 1024 + a_bytes + 512;
        if (fixed + 2 * stage > (size_t)kSmemLimit) continue;
        const uint32_t cols = bwd ? 2u * m_blocks * N + (uint32_t)(m_dw * w_r) : 4u * m_blocks * N;
        if (cols > 512) continue;
        c.N = N;
        c.dw_col = 2u * m_blocks * N;
        const int64_t want_st = tune_get(RELNN_TUNE_AGG_STAGES);
        c.stages = (int)std::min<size_t>(want_st ? (size_t)want_st : 4, (kSmemLimit - fixed) / stage);
        uint32_t t = 32;
        while (t < cols) t <<= 1;
        c.tmem_cols = t;
        c.smem = fixed + (size_t)c.stages * stage;
        return c;
    }
    return c;
}

bool two_kernel_forward(const Plan& p) {
    const int kpad = ((p.d + 63) / 64) * 64;
    return (!p.concat_dst || p.Ht().n_unique == p.n_h) && p.d % 8 == 0 && kpad <= 256 &&
           gemm_config(kpad / 64, p.concat_dst ? kpad / 64 : 0, (p.d_out + 127) / 128).N > 0;
}

// Forward: A = W with each Concat part padded to 64 columns; M = output features.
AggCfg fwd_cfg(const Plan& p) {
    const int n_parts = p.concat_dst ? 2 : 1;
    const int kpad = ((p.d + 63) / 64) * 64;
    return agg_config(n_parts * kpad / 64, (p.d_out + 127) / 128, false, 0, 0, 0);
}

template <int D, bool CDST>
relnn_status launch_fp32_agg_t(bool kahan, int grid, size_t smem, cudaStream_t st, const int4* vr, int64_t nv,
                               const int32_t* hs, const int32_t* d1, const float* z, int64_t z_rows, const float* W,
                               const float* b, int d_out, float* out, int64_t out_rows, float* vpart, int acc,
                               int* status) {
    // W above 48 KB (d_out x d_in floats) needs the larger dynamic shared-memory limit
    static size_t attr[2] = {0, 0};
    if (smem > 48 * 1024 && attr[kahan ? 1 : 0] < smem) {
        if (kahan) RELNN_CUDA(cudaFuncSetAttribute(fwd_fp32_agg_kernel<D, CDST, true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        else RELNN_CUDA(cudaFuncSetAttribute(fwd_fp32_agg_kernel<D, CDST, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr[kahan ? 1 : 0] = smem;
    }
    if (kahan) { fwd_fp32_agg_kernel<D, CDST, true><<<grid, 256, smem, st>>>(vr, nv, hs, d1, z, z_rows, W, b, d_out, out,
                                                                          out_rows, vpart, acc, status); note_launch(); }
    else { fwd_fp32_agg_kernel<D, CDST, false><<<grid, 256, smem, st>>>(vr, nv, hs, d1, z, z_rows, W, b, d_out, out,
                                                                     out_rows, vpart, acc, status); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

}  // namespace

namespace {
// The aggregate-first form's conditions other than the activation.
bool agg_shape_ok(const Plan& p, const CallIO& io, const float* out) {
    if (!aligned16(out)) return false;  // the fix-up adds partial rows as float4
    if (!p.bf16 || p.identity) return false;
    if (p.flags & (RELNN_FLAG_MAX | RELNN_FLAG_PUSHDOWN | RELNN_FLAG_PER_TUPLE | kPlanDense)) return false;
    if (p.Hx || p.dense_out || p.acc_out) return false;
    for (auto& b : p.br)
        if (b.d_r > 0) return false;
    if (!pow2_in(p.d, 8, 256) || p.d_out > 256 || p.d_out % 4 != 0) return false;
    // the gathered table is bf16 (given, or the plan's copy of an aligned f32 table)
    return aligned16(io.z) && fwd_cfg(p).N > 0;
}

// A ReLU rule's backward runs aggregate-first when every branch kept the forward's ReLU mask and
// the rule has the dst part (the dst pass also yields db).
bool relu_masked(const Plan& p) {
    if (p.act != RELNN_ACT_RELU || !p.concat_dst || (p.flags & RELNN_FLAG_MAX)) return false;
    for (auto& b : p.br)
        if (b.m > 0 && !b.relu_mask.p) return false;
    return true;
}
}  // namespace

bool agg_forward_ok(const Plan& p, const CallIO& io, const float* out) {
    return p.act == RELNN_ACT_NONE && agg_shape_ok(p, io, out);
}

bool agg_backward_ok(const Plan& p, const CallIO& io, const GradIO& g) {
    if (!(p.act == RELNN_ACT_NONE || relu_masked(p)) || !agg_shape_ok(p, io, g.dz)) return false;
    if (!pow2_in(p.d_out, 8, 256) || p.d % 32 != 0) return false;
    return g.dout != nullptr && aligned16(g.dout) &&
           gemm_config((p.d_out + 63) / 64, (p.d + 63) / 64, (p.d + 127) / 128, true, (p.d_out + 127) / 128, p.d).N > 0;
}

bool agg_forward_fp32_ok(const Plan& p, const CallIO& io, const float* out) {
    if (p.bf16 || p.identity || p.act != RELNN_ACT_NONE || !p.join_dst) return false;
    if (p.flags & (RELNN_FLAG_MAX | RELNN_FLAG_PUSHDOWN | RELNN_FLAG_PER_TUPLE | kPlanDense)) return false;
    if (p.Hx || p.dense_out || p.acc_out) return false;
    if (p.concat_dst && p.Ht().n_unique != p.n_h) return false;  // one dst H row per virtual row
    if (!(p.d == 4 || p.d == 8 || p.d == 16 || p.d == 32) || p.d_out % 4 != 0 || p.d_out > 256) return false;
    if (io.z_bf16 || io.w_bf16 || !aligned16(io.z) || !aligned16(out)) return false;
    for (size_t i = 0; i < p.br.size(); ++i)
        if (p.br[i].d_r > 0 || !aligned16(io.br[i].W)) return false;
    return true;
}

// Identity rules of the FP32 form (no Linear, no activation, Concat = z_src only: e.g. a SUM
// readout Out(g; SUM z) :- H(k; z), G(k, g)): out[row] = the f32 sum of z[hs_t] over the row's
// tuples. Lane groups of d / 4 lanes each own one virtual row at a time (a lane = one 16-byte column
// chunk), with kIdUnroll row loads in flight per lane; whole rows are written (or, for a later
// branch of a union, added), chunk partials of cut rows go to vpart for the fix-up. The per-tuple
// FP32 form computes the same sums in tuple order; the two differ by the order of f32 additions only.
constexpr int kIdUnroll = 4;

template <bool KAHAN>
__global__ void __launch_bounds__(256) fwd_identity_agg_kernel(const int4* __restrict__ vr, int64_t nv,
                                                            const int32_t* __restrict__ hs,
                                                            const float* __restrict__ z, int64_t z_rows, int d,
                                                            float* __restrict__ out, int64_t out_rows,
                                                            float* __restrict__ vpart, int accumulate, int* status) {
    const int lane = threadIdx.x & 31;
    const int L = d >> 2, lsh = 31 - __clz(L), G = 32 >> lsh;
    const int grp = lane >> lsh, ch = lane & (L - 1);
    const int64_t g0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * G + grp;
    const int64_t gs = (((int64_t)gridDim.x * blockDim.x) >> 5) * G;
    const float4* __restrict__ z4 = reinterpret_cast<const float4*>(z) + ch;
    for (int64_t v = g0; v < nv; v += gs) {
        const int4 m = __ldg(vr + v);  // {first tuple, tuples, output row, chunk slot or -1}
        const int n = m.y > 0 ? m.y : 0;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f), cmp = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int t0 = 0; t0 < n; t0 += kIdUnroll) {
            float4 u[kIdUnroll];
#pragma unroll
            for (int q = 0; q < kIdUnroll; ++q) {
                u[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (t0 + q < n) {
                    const int r = __ldg(hs + m.x + t0 + q);
                    if (in_bounds(r, z_rows, status)) u[q] = __ldg(z4 + (int64_t)r * L);
                }
            }
#pragma unroll
            for (int q = 0; q < kIdUnroll; ++q) {
                if (t0 + q >= n) break;
                if (KAHAN) {
                    kahan_add(acc.x, cmp.x, u[q].x);
                    kahan_add(acc.y, cmp.y, u[q].y);
                    kahan_add(acc.z, cmp.z, u[q].z);
                    kahan_add(acc.w, cmp.w, u[q].w);
                } else {
                    acc.x += u[q].x;
                    acc.y += u[q].y;
                    acc.z += u[q].z;
                    acc.w += u[q].w;
                }
            }
        }
        if (m.w >= 0) {
            reinterpret_cast<float4*>(vpart + (int64_t)m.w * d)[ch] = acc;
        } else if (m.z >= 0 && in_bounds(m.z, out_rows, status)) {
            float4* dst = reinterpret_cast<float4*>(out + (int64_t)m.z * d) + ch;
            if (accumulate) {
                const float4 o = *dst;
                acc = make_float4(o.x + acc.x, o.y + acc.y, o.z + acc.z, o.w + acc.w);
            }
            *dst = acc;
        }
    }
}

bool agg_forward_identity_ok(const Plan& p, const CallIO& io, const float* out) {
    if (p.bf16 || !p.identity || p.act != RELNN_ACT_NONE || p.concat_dst) return false;
    if (p.flags & (RELNN_FLAG_MAX | RELNN_FLAG_PUSHDOWN | RELNN_FLAG_PER_TUPLE | kPlanDense)) return false;
    if (p.Hx || p.dense_out || p.acc_out) return false;
    if (!(p.d == 4 || p.d == 8 || p.d == 16 || p.d == 32 || p.d == 64 || p.d == 128) || p.d_out != p.d) return false;
    if (io.z_bf16 || !aligned16(io.z) || !aligned16(out)) return false;
    for (size_t i = 0; i < p.br.size(); ++i)
        if (p.br[i].d_r > 0) return false;
    return true;
}

relnn_status forward_agg_identity(Plan& p, const CallIO& io, float* out, cudaStream_t st) {
    size_t vp_max = 0;
    for (auto& b : p.br) {
        RELNN_TRY(ensure_vrows(b.vr_out, b.seg.as<int32_t>(), b.m, p.n_out, true, st));
        vp_max = std::max(vp_max, (size_t)(b.vr_out.n_parts + b.vr_out.n_l2) * p.d);
    }
    if (vp_max) RELNN_TRY(p.vpart.alloc_nosync(sizeof(float) * vp_max, st));
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        const VRows& V = b.vr_out;
        if (V.nv == 0) continue;
        const int G = 32 / (p.d / 4);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(V.nv, 8 * (int64_t)G), (int64_t)num_sms() * 8));
        const float* z = reinterpret_cast<const float*>(io.z);
        const int acc = i > 0 ? 1 : 0;  // every branch covers every output row: the first one stores
        ProfToken pt = prof_begin(RELNN_PROF_FWD_FP32, st);
        if (p.kahan)
            fwd_identity_agg_kernel<true><<<grid, 256, 0, st>>>(V.vr.as<int4>(), V.nv, b.hs.as<int32_t>(), z, p.n_h, p.d,
                                                                out, p.n_out, p.vpart.as<float>(), acc, p.status.as<int>());
        else
            fwd_identity_agg_kernel<false><<<grid, 256, 0, st>>>(V.vr.as<int4>(), V.nv, b.hs.as<int32_t>(), z, p.n_h, p.d,
                                                                 out, p.n_out, p.vpart.as<float>(), acc, p.status.as<int>());
        note_launch();
        prof_end(pt, st);
        RELNN_CUDA(cudaGetLastError());
        RELNN_TRY(agg_fixup(V, p.vpart.as<float>(), p.vpart.as<float>() + (size_t)V.n_parts * p.d, out, p.d, i > 0,
                            p.kahan, p.n_out, p.status.as<int>(), st));
    }
    return RELNN_OK;
}

relnn_status forward_agg_fp32(Plan& p, const CallIO& io, float* out, cudaStream_t st) {
    size_t vp_max = 0;
    for (auto& b : p.br) {
        VRows& V = b.vr_out;
        RELNN_TRY(ensure_vrows(V, b.seg.as<int32_t>(), b.m, p.n_out, true, st));
        if (p.concat_dst && !V.has_d1) {
            RELNN_TRY(V.d1.alloc_nosync(sizeof(int32_t) * std::max<int64_t>(V.nv, 1), st));
            if (V.nv > 0) { vr_first_kernel<<<grid_for(V.nv), 256, 0, st>>>(V.vr.as<int4>(), V.nv, b.hd.as<int32_t>(), V.d1.as<int32_t>()); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
            V.has_d1 = true;
        }
        vp_max = std::max(vp_max, (size_t)(V.n_parts + V.n_l2) * p.d_out);
    }
    if (vp_max) RELNN_TRY(p.vpart.alloc_nosync(sizeof(float) * vp_max, st));
    const size_t smem = sizeof(float) * ((size_t)p.d_out * p.d_in + p.d_out);
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        const VRows& V = b.vr_out;
        if (V.nv == 0) continue;
        const int grid = grid_for(V.nv);
        const float* z = reinterpret_cast<const float*>(io.z);
        const float* W = reinterpret_cast<const float*>(io.br[i].W);
        const int32_t* d1 = p.concat_dst ? V.d1.as<int32_t>() : nullptr;
        const int acc = i > 0 ? 1 : 0;  // every branch covers every output row: the first one stores
        ProfToken pt = prof_begin(RELNN_PROF_FWD_FP32, st);
        relnn_status s = RELNN_OK;
#define RELNN_F32AGG(DD)                                                                                            \
        s = p.concat_dst ? launch_fp32_agg_t<DD, true>(p.kahan, grid, smem, st, V.vr.as<int4>(), V.nv, b.hs.as<int32_t>(), \
                                                       d1, z, p.n_h, W, io.br[i].b, p.d_out, out, p.n_out,             \
                                                       p.vpart.as<float>(), acc, p.status.as<int>())                   \
                         : launch_fp32_agg_t<DD, false>(p.kahan, grid, smem, st, V.vr.as<int4>(), V.nv,                \
                                                        b.hs.as<int32_t>(), d1, z, p.n_h, W, io.br[i].b, p.d_out, out, \
                                                        p.n_out, p.vpart.as<float>(), acc, p.status.as<int>())
        switch (p.d) {
            case 4: RELNN_F32AGG(4); break;
            case 8: RELNN_F32AGG(8); break;
            case 16: RELNN_F32AGG(16); break;
            default: RELNN_F32AGG(32); break;
        }
#undef RELNN_F32AGG
        prof_end(pt, st);
        RELNN_TRY(s);
        RELNN_TRY(agg_fixup(V, p.vpart.as<float>(), p.vpart.as<float>() + (size_t)V.n_parts * p.d_out, out, p.d_out, i > 0,
                            p.kahan, p.n_out, p.status.as<int>(), st));
    }
    return RELNN_OK;
}

// Two-kernel forward (unique H keys or no dst part): gather-sum into S, then the TMA-fed GEMM.
relnn_status forward_two_kernel(Plan& p, const CallIO& io, float* out, cudaStream_t st) {
    const int kpad = ((p.d + 63) / 64) * 64;
    const int n_kb_s = kpad / 64, n_kb_r = p.concat_dst ? kpad / 64 : 0;
    const int m_blocks = (p.d_out + 127) / 128;
    const AggCfg cfg = gemm_config(n_kb_s, n_kb_r, m_blocks);
    const int rows_pad = m_blocks * 128, cols = (n_kb_s + n_kb_r) * 64;
    RELNN_TRY(p.wpack.alloc_nosync(sizeof(uint16_t) * (size_t)rows_pad * cols, st));
    CUtensorMap amap;
    RELNN_TRY(encode_bf16_tile_map(&amap, p.wpack.p, cols, rows_pad));
    size_t vp_max = 0;
    int64_t nv_max = 0;
    for (auto& b : p.br) {
        VRows& V = b.vr_out;
        RELNN_TRY(ensure_vrows(V, b.seg.as<int32_t>(), b.m, p.n_out, true, st));
        if (p.concat_dst && !V.has_d1) {
            RELNN_TRY(V.d1.alloc_nosync(sizeof(int32_t) * std::max<int64_t>(V.nv, 1), st));
            if (V.nv > 0) { vr_first_kernel<<<grid_for(V.nv), 256, 0, st>>>(V.vr.as<int4>(), V.nv, b.hd.as<int32_t>(), V.d1.as<int32_t>()); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
            V.has_d1 = true;
        }
        vp_max = std::max(vp_max, (size_t)(V.n_parts + V.n_l2) * p.d_out);
        nv_max = std::max(nv_max, V.nv);
    }
    if (vp_max) RELNN_TRY(p.vpart.alloc_nosync(sizeof(float) * vp_max, st));
    static bool attr_set = false;
    if (!attr_set) {
        RELNN_CUDA(cudaFuncSetAttribute(agg_gemm_kernel<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        RELNN_CUDA(cudaFuncSetAttribute(agg_gemm_kernel<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        RELNN_CUDA(cudaFuncSetAttribute(agg_gemm_kernel<false, 4, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        RELNN_CUDA(cudaFuncSetAttribute(agg_gemm_kernel<false, 8, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        attr_set = true;
    }
    const int kmin = (int)tune_get(RELNN_TUNE_KAHAN_MIN);
    // compensation inside the 32-tuple chunks only when the threshold reaches them (the chunks of a
    // longer row are always added with compensation by the fix-up)
    const bool ksum = p.kahan && kmin <= kChunk;
    // fused (RELNN_TUNE_AGG_FUSE): the GEMM's own producer warps compute the pairs (plain f32 sums)
    const int fuse = ksum ? 0 : (int)tune_get(RELNN_TUNE_AGG_FUSE);
    if (!fuse) RELNN_TRY(p.sbuf.alloc_nosync(sizeof(uint16_t) * 2 * (size_t)kpad * std::max<int64_t>(nv_max, 1), st));
    const bool wide = !ksum && seg_sum_wide_ok(p.d, io.z);
    const int ss_blocks = ksum ? seg_sum_grid<true, false>(nv_max)
                               : wide ? seg_sum_wide_grid(nv_max) : seg_sum_grid<false, false>(nv_max);
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        const VRows& V = b.vr_out;
        if (V.nv == 0) continue;
        uint16_t* S = fuse ? p.wpack.as<uint16_t>() : p.sbuf.as<uint16_t>();  // (fused: the map is unused)
        if (!fuse) {
            ProfToken pt = prof_begin(RELNN_PROF_AGG_SUM, st);
            const uint16_t* zt = reinterpret_cast<const uint16_t*>(io.z);
            if (ksum) seg_sum_kernel<true, false><<<ss_blocks, 32 * kSegWarps, 0, st>>>(V.vr.as<int4>(), V.nv, b.hs.as<int32_t>(), zt,
                                                                                p.n_h, p.d, kpad, S, p.status.as<int>(), kmin);
            else if (wide) seg_sum_wide_kernel<kSegUnrollWide><<<ss_blocks, 32 * kSegWarps, 0, st>>>(
                V.vr.as<int4>(), V.nv, b.hs.as<int32_t>(), zt, p.n_h, p.d, kpad, S, p.status.as<int>());
            else seg_sum_kernel<false, false><<<ss_blocks, 32 * kSegWarps, 0, st>>>(V.vr.as<int4>(), V.nv, b.hs.as<int32_t>(), zt,
                                                                          p.n_h, p.d, kpad, S, p.status.as<int>(), kmin);
            note_launch();
            prof_end(pt, st);
        }
        RELNN_CUDA(cudaGetLastError());
        { pack_a_fwd_kernel<<<grid_for((int64_t)rows_pad * cols), 256, 0, st>>>(io.br[i].W, io.w_bf16, p.d_out, p.d_in, p.d,
                                                                               kpad, rows_pad, cols, p.wpack.as<uint16_t>()); note_launch(); }
        CUtensorMap smap;
        if (fuse) RELNN_TRY(encode_bf16_tile_map(&smap, S, cols, rows_pad, cfg.N));
        else RELNN_TRY(encode_bf16_tile_map(&smap, S, 2 * kpad, V.nv, cfg.N));
        GemmArgs a{};
        a.vr = V.vr.as<int4>();
        a.nv = V.nv;
        a.n_tiles = ceil_div(V.nv, cfg.N);
        a.gidx = b.hs.as<int32_t>();
        a.gtbl = reinterpret_cast<const uint16_t*>(io.z);
        a.gtbl_rows = p.n_h;
        a.w_s = p.d;
        a.ridx = p.concat_dst ? V.d1.as<int32_t>() : nullptr;
        a.ridx_stride = 1;
        a.rtbl = reinterpret_cast<const uint16_t*>(io.z);
        a.rtbl_rows = p.n_h;
        a.out_rows = p.n_out;
        a.w_r = p.concat_dst ? p.d : 0;
        a.n_kb_s = n_kb_s;
        a.n_kb_r = n_kb_r;
        a.kpad_s = kpad;
        a.m_blocks = m_blocks;
        a.n_feat = p.d_out;
        a.bias = io.br[i].b;
        a.out = out;
        a.vpart = p.vpart.as<float>();
        a.accumulate = i > 0 ? 1 : 0;  // every branch covers every output row: the first one stores
        a.tile_n = cfg.N;
        a.stages = cfg.stages;
        a.idesc = tc::idesc_bf16_f32(128, cfg.N);
        a.tmem_cols = cfg.tmem_cols;
        a.status = p.status.as<int>();
        const int grid = (int)std::min<int64_t>(a.n_tiles, num_sms());
        {
            ProfToken pt = prof_begin(RELNN_PROF_AGG_FWD, st);
            if (fuse == 1) agg_gemm_kernel<false, 4, 8><<<grid, gemm_threads(4, 8), cfg.smem, st>>>(amap, smap, a);
            else if (fuse == 2) agg_gemm_kernel<false, 8, 4><<<grid, gemm_threads(8, 4), cfg.smem, st>>>(amap, smap, a);
            else if (gemm_epi() == 4) agg_gemm_kernel<false, 4><<<grid, gemm_threads(4), cfg.smem, st>>>(amap, smap, a);
            else agg_gemm_kernel<false, 8><<<grid, gemm_threads(8), cfg.smem, st>>>(amap, smap, a);
            note_launch();
            prof_end(pt, st);
        }
        RELNN_CUDA(cudaGetLastError());
        RELNN_TRY(agg_fixup(V, p.vpart.as<float>(), p.vpart.as<float>() + (size_t)V.n_parts * p.d_out, out, p.d_out, i > 0,
                            p.kahan, p.n_out, p.status.as<int>(), st));
    }
    return RELNN_OK;
}

relnn_status forward_agg(Plan& p, const CallIO& io_in, float* out, cudaStream_t st) {
    CallIO io;
    RELNN_TRY(with_bf16_z(p, io_in, io, st));
    if (two_kernel_forward(p)) return forward_two_kernel(p, io, out, st);
    const int n_parts = p.concat_dst ? 2 : 1;
    const int kpad = ((p.d + 63) / 64) * 64;
    const int n_kb = n_parts * kpad / 64;
    const int m_blocks = (p.d_out + 127) / 128;
    const AggCfg cfg = fwd_cfg(p);
    if (cfg.N == 0) {
        set_error("aggregate-first forward: operands too large for shared memory");
        return RELNN_ENOTSUP;
    }
    const int rows_pad = m_blocks * 128, cols = n_kb * 64;
    RELNN_TRY(p.wpack.alloc_nosync(sizeof(uint16_t) * (size_t)rows_pad * cols, st));
    CUtensorMap amap;
    RELNN_TRY(encode_bf16_tile_map(&amap, p.wpack.p, cols, rows_pad));
    size_t vp_max = 0;
    for (auto& b : p.br) {
        RELNN_TRY(ensure_vrows(b.vr_out, b.seg.as<int32_t>(), b.m, p.n_out, true, st));
        vp_max = std::max(vp_max, (size_t)(b.vr_out.n_parts + b.vr_out.n_l2) * p.d_out);
    }
    if (vp_max) RELNN_TRY(p.vpart.alloc_nosync(sizeof(float) * vp_max, st));
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        const VRows& V = b.vr_out;
        if (V.nv == 0) continue;
        { pack_a_fwd_kernel<<<grid_for((int64_t)rows_pad * cols), 256, 0, st>>>(io.br[i].W, io.w_bf16, p.d_out, p.d_in, p.d,
                                                                               kpad, rows_pad, cols, p.wpack.as<uint16_t>()); note_launch(); }
        AggArgs a{};
        a.vr = V.vr.as<int4>();
        a.nv = V.nv;
        a.n_tiles = ceil_div(V.nv, cfg.N);
        // the dst part first (one or a few rows per virtual row: its load overlaps the src part's)
        int pi = 0;
        if (p.concat_dst) {
            a.gidx[pi] = b.hd.as<int32_t>();
            a.tbl[pi] = reinterpret_cast<const uint16_t*>(io.z);
            a.tbl_rows[pi] = p.n_h;
            a.width[pi] = p.d;
            a.kind[pi] = 1;
            a.kofs[pi] = kpad;
            ++pi;
        }
        a.gidx[pi] = b.hs.as<int32_t>();
        a.tbl[pi] = reinterpret_cast<const uint16_t*>(io.z);
        a.tbl_rows[pi] = p.n_h;
        a.width[pi] = p.d;
        a.kind[pi] = 0;
        a.kofs[pi] = 0;
        a.n_parts = pi + 1;
        a.n_kb = n_kb;
        a.m_blocks = m_blocks;
        a.n_feat = p.d_out;
        a.bias = io.br[i].b;
        a.out = out;
        a.vpart = p.vpart.as<float>();
        a.accumulate = i > 0 ? 1 : 0;  // every branch covers every output row: the first one stores
        a.tile_n = cfg.N;
        a.stages = cfg.stages;
        a.idesc = tc::idesc_bf16_f32(128, cfg.N);
        a.tmem_cols = cfg.tmem_cols;
        a.status = p.status.as<int>();
        const int grid = (int)std::min<int64_t>(a.n_tiles, num_sms());
        RELNN_TRY(launch_agg<false>(amap, a, p.kahan, cfg.smem, grid, st, RELNN_PROF_AGG_FWD));
        RELNN_TRY(agg_fixup(V, p.vpart.as<float>(), p.vpart.as<float>() + (size_t)V.n_parts * p.d_out, out, p.d_out, i > 0,
                            p.kahan, p.n_out, p.status.as<int>(), st));
    }
    return RELNN_OK;
}

relnn_status backward_agg(Plan& p, const CallIO& io_in, const GradIO& g, cudaStream_t st) {
    CallIO io;
    RELNN_TRY(with_bf16_z(p, io_in, io, st));
    const int n_kb = (p.d_out + 63) / 64;       // K of the dz GEMM: the G features
    const int m_blocks = (p.d + 127) / 128;     // dz features
    const int z_blocks = (p.d + 63) / 64;
    const int m_dw = (p.d_out + 127) / 128;     // dW rows (G features)
    const int kpad_g = ((p.d_out + 63) / 64) * 64;  // S row: the bf16 pair of a G row
    const AggCfg cfg = gemm_config(n_kb, z_blocks, m_blocks, true, m_dw, p.d);
    if (cfg.N == 0) {
        set_error("aggregate-first backward: operands too large for shared memory");
        return RELNN_ENOTSUP;
    }
    const int rows_pad = m_blocks * 128, cols = n_kb * 64;
    const int grid_max = num_sms();
    const int pblocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(p.n_out, 64), 4 * (int64_t)num_sms()));
    // scratch: A (bf16), the CTAs' dW partials, the blocks' db partials
    const size_t a_elems = (size_t)rows_pad * cols;
    const size_t a_bytes = (a_elems * 2 + 255) & ~(size_t)255;
    // ReLU rule: dY_t = dOut[seg_t] masked by the forward's ReLU mask; db then comes from the masked
    // dst pass (its blocks' partials), not from the tuple counts
    const bool masked = p.act == RELNN_ACT_RELU;
    const int mask_words = ((p.d_out + 127) / 128) * 4;
    const int64_t ss_max = (int64_t)num_sms() * 8;  // blocks of a gather-sum launch, at most
    const size_t dwp = (size_t)grid_max * p.d_out * p.d,
                 dbp = (size_t)std::max<int64_t>(pblocks * kDbBranches, masked ? ss_max : 0) * p.d_out;
    RELNN_TRY(p.scratch.alloc_nosync(a_bytes + sizeof(float) * (dwp + dbp), st));
    uint16_t* abuf = p.scratch.as<uint16_t>();
    float* dw_part = reinterpret_cast<float*>(p.scratch.as<uint8_t>() + a_bytes);
    float* db_part = dw_part + dwp;
    // dOut rows are gathered as bf16 (the rounding the tensor cores give dY in the per-tuple form);
    // the sums G are split into a bf16 pair like S in the forward. db comes from the f32 dOut, in
    // the pass that makes the bf16 copy (tuples per output row from the forward's virtual rows).
    for (auto& b : p.br) RELNN_TRY(ensure_vrows(b.vr_out, b.seg.as<int32_t>(), b.m, p.n_out, true, st));
    if (p.n_out > 0) {
        RELNN_TRY(p.doutbf.alloc_nosync(sizeof(uint16_t) * (size_t)p.n_out * p.d_out, st));
        const int64_t rpb = ceil_div(p.n_out, pblocks);
        for (size_t b0 = 0; b0 < p.br.size(); b0 += kDbBranches) {
            CntSet cs{};
            cs.n = (int)std::min<size_t>(kDbBranches, p.br.size() - b0);
            for (int k = 0; k < cs.n; ++k) cs.c[k] = p.br[b0 + k].vr_out.cnt.as<int32_t>();
            { dout_prep_kernel<<<pblocks, 256, 0, st>>>(g.dout, p.n_out, p.d_out, cs, rpb, p.doutbf.as<uint16_t>(),
                                                       db_part); note_launch(); }
            for (int k = 0; k < cs.n && !masked; ++k) {
                float* db = g.db.size() > b0 + k ? g.db[b0 + k] : nullptr;
                if (db) { db_reduce_kernel<<<(unsigned)ceil_div(p.d_out, 32), 256, 0, st>>>(db_part, pblocks, p.d_out, k, db); note_launch(); }
            }
        }
        RELNN_CUDA(cudaGetLastError());
    } else {
        for (size_t i = 0; i < p.br.size(); ++i)
            if (g.db.size() > i && g.db[i]) RELNN_CUDA(cudaMemsetAsync(g.db[i], 0, sizeof(float) * p.d_out, st));
    }
    CUtensorMap amap;
    RELNN_TRY(encode_bf16_tile_map(&amap, abuf, cols, rows_pad));
    // virtual rows of both passes of every branch first, so the partial rows and sums are allocated once
    const int n_pass = p.concat_dst ? 2 : 1;
    size_t vp_max = 0;
    int64_t nv_max = 0;
    for (auto& b : p.br) {
        RELNN_TRY(ensure_src_order(p, b, st));
        RELNN_TRY(ensure_vrows(b.vr_src, b.hs_src.as<int32_t>(), b.m, p.n_h, true, st));
        // dst pass: one virtual row per H row in H-row order (the tuples of one dst H row are one
        // contiguous run of the plan's order), so the GEMM adds into consecutive dz rows; only when
        // that adds at most as many empty rows as there are runs, else the runs in plan order
        const bool h_order = 2 * p.n_out >= p.n_h;
        if (n_pass > 1) RELNN_TRY(ensure_vrows(b.vr_dst, b.hd.as<int32_t>(), b.m, h_order ? p.n_h : 0, h_order, st));
        vp_max = std::max(vp_max, (size_t)(b.vr_src.n_parts + b.vr_src.n_l2) * p.d);
        nv_max = std::max(nv_max, b.vr_src.nv);
        if (n_pass > 1) {
            vp_max = std::max(vp_max, (size_t)(b.vr_dst.n_parts + b.vr_dst.n_l2) * p.d);
            nv_max = std::max(nv_max, b.vr_dst.nv);
        }
    }
    if (vp_max) RELNN_TRY(p.vpart.alloc_nosync(sizeof(float) * vp_max, st));
    RELNN_TRY(p.sbuf.alloc_nosync(sizeof(uint16_t) * 2 * (size_t)kpad_g * std::max<int64_t>(nv_max, 1), st));
    static bool attr_set = false;
    if (!attr_set) {
        RELNN_CUDA(cudaFuncSetAttribute(agg_gemm_kernel<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        RELNN_CUDA(cudaFuncSetAttribute(agg_gemm_kernel<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        attr_set = true;
    }
    DevBuf mask_src;  // ReLU rule: the mask in the src pass's tuple order
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        float* dW = g.dW.size() > i ? g.dW[i] : nullptr;
        for (int pass = 0; pass < n_pass; ++pass) {
            VRows& V = pass == 0 ? b.vr_src : b.vr_dst;
            const int col0 = pass == 0 ? 0 : p.d;
            if (V.nv == 0) {
                if (dW) {
                    // no tuples: this slice of dW is zero
                    RELNN_CUDA(cudaMemset2DAsync(dW + col0, sizeof(float) * p.d_in, 0, sizeof(float) * p.d, p.d_out, st));
                }
                continue;
            }
            // G rows: sums of dOut rows per virtual row (src order: a row per tuple; dst order: one
            // row times the run's length), as bf16 pairs
            uint16_t* S = p.sbuf.as<uint16_t>();
            const int kmin = (int)tune_get(RELNN_TUNE_KAHAN_MIN);
            const bool ksum = p.kahan && kmin <= kChunk;  // as in the forward
            const bool wide = !masked && pass == 0 && !ksum && seg_sum_wide_ok(p.d_out, p.doutbf.p);
            const int ss_blocks =
                (int)std::min<int64_t>(ss_max, masked ? (pass == 1 ? seg_sum_grid<false, true, true>(V.nv)
                                                        : ksum ? seg_sum_grid<true, false, true>(V.nv)
                                                               : seg_sum_grid<false, false, true>(V.nv))
                                                      : (pass == 1 ? seg_sum_grid<false, true>(V.nv)
                                                         : ksum ? seg_sum_grid<true, false>(V.nv)
                                                         : wide ? seg_sum_wide_grid(V.nv)
                                                                : seg_sum_grid<false, false>(V.nv)));
            const int32_t* gi = pass == 0 ? b.seg_src.as<int32_t>() : b.seg.as<int32_t>();
            {
                ProfToken pt = prof_begin(RELNN_PROF_AGG_SUM, st);
                const uint16_t* tb = p.doutbf.as<uint16_t>();
                int* stw = p.status.as<int>();
                const uint32_t* mk = masked ? b.relu_mask.as<uint32_t>() : nullptr;
                if (masked && pass == 0) {
                    // the mask in src order first (one gather of 4 x mask_words bytes per tuple)
                    const int src_words = (p.d_out + 31) / 32;
                    RELNN_TRY(mask_src.alloc_tmp(sizeof(uint32_t) * (size_t)b.m * src_words, st));
                    { permute_mask_kernel<<<grid_for(b.m), 256, 0, st>>>(mk, b.src_perm.as<int32_t>(), b.m, mask_words,
                                                                         src_words, mask_src.as<uint32_t>()); note_launch(); }
                    if (ksum) seg_sum_kernel<true, false, true><<<ss_blocks, 32 * kSegWarps, 0, st>>>(
                        V.vr.as<int4>(), V.nv, gi, tb, p.n_out, p.d_out, kpad_g, S, stw, kmin, mask_src.as<uint32_t>(),
                        src_words);
                    else seg_sum_kernel<false, false, true><<<ss_blocks, 32 * kSegWarps, 0, st>>>(
                        V.vr.as<int4>(), V.nv, gi, tb, p.n_out, p.d_out, kpad_g, S, stw, kmin, mask_src.as<uint32_t>(),
                        src_words);
                } else if (masked) {
                    seg_sum_kernel<false, true, true><<<ss_blocks, 32 * kSegWarps, 0, st>>>(
                        V.vr.as<int4>(), V.nv, gi, tb, p.n_out, p.d_out, kpad_g, S, stw, 0, mk, mask_words, db_part,
                        g.dout);
                } else if (pass == 0) {
                    if (ksum) seg_sum_kernel<true, false><<<ss_blocks, 32 * kSegWarps, 0, st>>>(V.vr.as<int4>(), V.nv, gi, tb, p.n_out,
                                                                                        p.d_out, kpad_g, S, stw, kmin);
                    else if (wide) seg_sum_wide_kernel<kSegUnrollWide><<<ss_blocks, 32 * kSegWarps, 0, st>>>(
                        V.vr.as<int4>(), V.nv, gi, tb, p.n_out, p.d_out, kpad_g, S, stw);
                    else seg_sum_kernel<false, false><<<ss_blocks, 32 * kSegWarps, 0, st>>>(V.vr.as<int4>(), V.nv, gi, tb, p.n_out,
                                                                                  p.d_out, kpad_g, S, stw, kmin);
                } else {
                    seg_sum_kernel<false, true><<<ss_blocks, 32 * kSegWarps, 0, st>>>(V.vr.as<int4>(), V.nv, gi, tb, p.n_out, p.d_out,
                                                                            kpad_g, S, stw, 0);
                }
                note_launch();
                prof_end(pt, st);
            }
            RELNN_CUDA(cudaGetLastError());
            if (masked && pass == 1) {
                // db of this branch: the masked dst pass's block partials, added in block order
                float* db = g.db.size() > i ? g.db[i] : nullptr;
                if (db) { db_reduce_kernel<<<(unsigned)ceil_div(p.d_out, 32), 256, 0, st>>>(db_part, ss_blocks, p.d_out, -1, db); note_launch(); }
            }
            { pack_a_bwd_kernel<<<grid_for((int64_t)a_elems), 256, 0, st>>>(io.br[i].W, io.w_bf16, p.d_out, p.d_in, col0, p.d,
                                                                           rows_pad, cols, abuf); note_launch(); }
            CUtensorMap smap;
            RELNN_TRY(encode_bf16_tile_map(&smap, S, 2 * kpad_g, V.nv, cfg.N));
            const bool accumulate = pass > 0 || i > 0 || g.accumulate_dz;
            GemmArgs a{};
            a.vr = V.vr.as<int4>();
            a.nv = V.nv;
            a.n_tiles = ceil_div(V.nv, cfg.N);
            a.ridx = reinterpret_cast<const int32_t*>(V.vr.as<int4>()) + 2;  // the row id field (an H row)
            a.ridx_stride = 4;
            a.rtbl = reinterpret_cast<const uint16_t*>(io.z);
            a.rtbl_rows = p.n_h;
            a.out_rows = p.n_h;
            a.w_r = p.d;
            a.n_kb_s = n_kb;
            a.n_kb_r = z_blocks;
            a.kpad_s = kpad_g;
            a.m_blocks = m_blocks;
            a.n_feat = p.d;
            a.bias = nullptr;
            a.out = g.dz;
            a.vpart = p.vpart.as<float>();
            a.accumulate = accumulate ? 1 : 0;
            a.tile_n = cfg.N;
            a.stages = cfg.stages;
            a.idesc = tc::idesc_bf16_f32(128, cfg.N);
            a.tmem_cols = cfg.tmem_cols;
            a.status = p.status.as<int>();
            a.dw_part = dw_part;
            a.n_g = p.d_out;
            a.m_dw = m_dw;
            a.idesc_dw = tc::idesc_bf16_f32(128, p.d, true, true);
            a.dw_col = cfg.dw_col;
            const int grid = (int)std::min<int64_t>(a.n_tiles, grid_max);
            {
                ProfToken pt = prof_begin(RELNN_PROF_AGG_BWD, st);
                if (gemm_epi() == 4) agg_gemm_kernel<true, 4><<<grid, gemm_threads(4), cfg.smem, st>>>(amap, smap, a);
                else agg_gemm_kernel<true, 8><<<grid, gemm_threads(8), cfg.smem, st>>>(amap, smap, a);
                note_launch();
                prof_end(pt, st);
            }
            RELNN_CUDA(cudaGetLastError());
            RELNN_TRY(agg_fixup(V, p.vpart.as<float>(), p.vpart.as<float>() + (size_t)V.n_parts * p.d, g.dz, p.d, accumulate,
                                p.kahan, p.n_h, p.status.as<int>(), st));
            if (dW) {
                const int64_t nw = (int64_t)p.d_out * p.d;
                { agg_reduce_dw_kernel<<<(unsigned)ceil_div(nw, 32), 256, 0, st>>>(dw_part, grid, p.d_out, p.d, dW, p.d_in, col0); note_launch(); }
            }
            RELNN_CUDA(cudaGetLastError());
        }
    }
    return RELNN_OK;
}

}  // namespace relnn
