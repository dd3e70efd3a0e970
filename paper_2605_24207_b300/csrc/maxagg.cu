// MAX aggregator of the projected union (paper Sec. 2.2: alpha over the multiset B_t of contributing
// tuples; Sec. 4.2 compiles the union to a scatter whose reduction is selected by alpha, MAX among
// them). For a single-branch rule, per output row k and feature o,
//   Out[k][o] = max_{t -> k} Y_t[o],   arg[k][o] = the first such t in plan order,
// plan order within a row being (dst H row, E row, src H row). The backward sends dOut[k][o] to
// arg[k][o] alone, times ReLU' there (arg = -1 when ReLU'd to zero: no gradient).
//
// The forward kernels compute each tile's pieces; a segment cut by tile boundaries leaves one
// (value, position) partial per tile, combined here in tile order with a strict comparison, so the
// earliest maximum wins as in a sequential walk. The backward reuses the ReLU-mask path: the winner
// mask has bit o of tuple t set iff t = arg[seg_t][o].
#include "maxagg.cuh"
#include "segfix.cuh"

#include <algorithm>

namespace relnn {

namespace {

constexpr int kLongPieces = 64;  // segments with more pieces go to the block-per-segment pass

__device__ __forceinline__ void max_take(float& v, int& p, float x, int xp) {
    const bool t = x > v;
    v = t ? x : v;
    p = t ? xp : p;
}

__global__ void fixup_max_kernel(const int32_t* __restrict__ seg, int64_t m, int tile, int64_t n_tiles,
                                 const float* __restrict__ carry, const int32_t* __restrict__ cpos,
                                 float* __restrict__ out, int32_t* __restrict__ arg, int d_out, int relu, int vec4,
                                 int* __restrict__ jobs, int max_jobs) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) + 1; b < n_tiles; b += nwarps) {
        int s, fs;
        int64_t e;
        if (!first_cut(seg, m, tile, b, lane, s, fs, e)) continue;
        const int64_t P = e - b + 2;
        if (jobs && P > kLongPieces) {
            if (lane == 0) {
                const int k = atomicAdd(jobs, 1);
                if (k < max_jobs) reinterpret_cast<int4*>(jobs + 4)[k] = make_int4((int)b, (int)e, fs, s);
            }
            continue;
        }
        if (vec4) {
            // four features per lane: 16-byte loads of the values and positions of every piece
            for (int o = lane * 4; o < d_out; o += 128) {
                const int64_t c0 = piece_slot(b, fs, 0) * d_out + o;
                float4 v = *reinterpret_cast<const float4*>(carry + c0);
                int4 p = *reinterpret_cast<const int4*>(cpos + c0);
                for (int64_t i = 1; i < P; ++i) {
                    const int64_t c = piece_slot(b, fs, i) * d_out + o;
                    const float4 x = *reinterpret_cast<const float4*>(carry + c);
                    const int4 xp = *reinterpret_cast<const int4*>(cpos + c);
                    max_take(v.x, p.x, x.x, xp.x);
                    max_take(v.y, p.y, x.y, xp.y);
                    max_take(v.z, p.z, x.z, xp.z);
                    max_take(v.w, p.w, x.w, xp.w);
                }
                if (relu) {
                    p.x = v.x > 0.f ? p.x : -1;
                    p.y = v.y > 0.f ? p.y : -1;
                    p.z = v.z > 0.f ? p.z : -1;
                    p.w = v.w > 0.f ? p.w : -1;
                }
                *reinterpret_cast<float4*>(out + (int64_t)s * d_out + o) = v;
                *reinterpret_cast<int4*>(arg + (int64_t)s * d_out + o) = p;
            }
            continue;
        }
        for (int o = lane; o < d_out; o += 32) {
            float v = carry[piece_slot(b, fs, 0) * d_out + o];
            int p = cpos[piece_slot(b, fs, 0) * d_out + o];
            int64_t i = 1;
            for (; i + 3 < P; i += 4) {
                float x[4];
                int xp[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t c = piece_slot(b, fs, i + u) * d_out + o;
                    x[u] = carry[c];
                    xp[u] = cpos[c];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) max_take(v, p, x[u], xp[u]);
            }
            for (; i < P; ++i) {
                const int64_t c = piece_slot(b, fs, i) * d_out + o;
                max_take(v, p, carry[c], cpos[c]);
            }
            out[(int64_t)s * d_out + o] = v;
            arg[(int64_t)s * d_out + o] = (relu && !(v > 0.f)) ? -1 : p;
        }
    }
}

// One block of 8 warps per recorded long segment: warp w reduces the w-th eighth of the pieces, the
// eight partials are then combined in warp order (strict comparison: the earliest maximum wins).
__global__ void __launch_bounds__(256) long_fixup_max_kernel(const int* __restrict__ jobs, int max_jobs,
                                                             const float* __restrict__ carry,
                                                             const int32_t* __restrict__ cpos, float* __restrict__ out,
                                                             int32_t* __restrict__ arg, int d_out, int relu) {
    __shared__ float pv[8][256];
    __shared__ int pp[8][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int njobs = min(jobs[0], max_jobs);
    for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
        const int4 J = reinterpret_cast<const int4*>(jobs + 4)[jb];
        const int64_t b = J.x, e = J.y;
        const int fs = J.z, s = J.w;
        const int64_t P = e - b + 2;
        const int64_t p0 = P * warp / 8, p1 = P * (warp + 1) / 8;  // p1 > p0: P > 8
        for (int o = lane; o < d_out; o += 32) {
            float v = carry[piece_slot(b, fs, p0) * d_out + o];
            int p = cpos[piece_slot(b, fs, p0) * d_out + o];
            for (int64_t i = p0 + 1; i < p1; ++i) {
                const int64_t c = piece_slot(b, fs, i) * d_out + o;
                max_take(v, p, carry[c], cpos[c]);
            }
            pv[warp][o] = v;
            pp[warp][o] = p;
        }
        __syncthreads();
        if (warp == 0) {
            for (int o = lane; o < d_out; o += 32) {
                float v = pv[0][o];
                int p = pp[0][o];
                for (int w = 1; w < 8; ++w) max_take(v, p, pv[w][o], pp[w][o]);
                out[(int64_t)s * d_out + o] = v;
                arg[(int64_t)s * d_out + o] = (relu && !(v > 0.f)) ? -1 : p;
            }
        }
        __syncthreads();
    }
}

// Winner mask: for output row k and 32-feature word w, the lanes of a warp hold arg[k][32 w + lane];
// lanes naming the same tuple form one word (bit = lane) written once. Only row k's item names a
// tuple of row k, so every word is written by at most one warp (no atomics).
__global__ void win_mask_kernel(const int32_t* __restrict__ arg, int64_t n_out, int d_out, int words,
                                int64_t m, uint32_t* __restrict__ win, int mask_words, int* status) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t items = n_out * words;
    for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nwarps) {
        const int64_t k = it / words;
        const int w = (int)(it - k * words);
        const int o = 32 * w + lane;
        int p = o < d_out ? __ldg(arg + k * d_out + o) : -1;
        if (p >= m) {  // a position outside the plan: record, skip
            raise_status(status, RELNN_DEV_BOUNDS);
            p = -1;
        }
        const unsigned grp = __match_any_sync(0xffffffffu, p);
        if (p >= 0 && lane == __ffs(grp) - 1) win[(int64_t)p * mask_words + w] = grp;
    }
}

int grid_of(int64_t warps) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps, 8), (int64_t)num_sms() * 8));
}

}  // namespace

relnn_status launch_fixup_max(const int32_t* seg, int64_t m, int tile, int64_t n_tiles, const float* carry,
                              const int32_t* carry_pos, float* out, int32_t* arg, int d_out, bool relu,
                              DevBuf& jobs_buf, cudaStream_t st) {
    if (n_tiles <= 1) return RELNN_OK;
    RELNN_CHECK_ARG(d_out <= 256, "MAX fix-up: d_out <= 256");
    const bool split = n_tiles > kLongPieces;
    const int max_jobs = split ? (int)(n_tiles / kLongPieces + 1) : 0;
    int* jobs = nullptr;
    if (split) {
        RELNN_TRY(jobs_buf.alloc(sizeof(int) * (4 + 4 * (size_t)max_jobs)));
        jobs = jobs_buf.as<int>();
        RELNN_CUDA(cudaMemsetAsync(jobs, 0, sizeof(int), st));
    }
    const bool vec4 = d_out % 4 == 0 && ((reinterpret_cast<uintptr_t>(carry) | reinterpret_cast<uintptr_t>(carry_pos) |
                                          reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(arg)) & 15u) == 0;
    ProfToken pt = prof_begin(RELNN_PROF_FIXUP, st);
    { fixup_max_kernel<<<grid_of(n_tiles - 1), 256, 0, st>>>(seg, m, tile, n_tiles, carry, carry_pos, out, arg, d_out,
                                                             relu ? 1 : 0, vec4 ? 1 : 0, jobs, max_jobs); note_launch(); }
    if (split) {
        { long_fixup_max_kernel<<<num_sms(), 256, 0, st>>>(jobs, max_jobs, carry, carry_pos, out, arg, d_out,
                                                          relu ? 1 : 0); note_launch(); }
    }
    prof_end(pt, st);
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

int max_mask_words(int d_out) { return ((d_out + 127) / 128) * 4; }

relnn_status build_win_mask(Plan& p, cudaStream_t st) {
    if (!p.max_ready) {
        set_error("MAX backward: run the plan's forward first (the argmax is recorded there)");
        return RELNN_ENOTSUP;
    }
    BranchPlan& b = p.br[0];
    if (b.m == 0 || p.n_out == 0) return RELNN_OK;
    const int mw = max_mask_words(p.d_out);
    const size_t bytes = sizeof(uint32_t) * (size_t)b.m * mw;
    RELNN_TRY(p.win_mask.alloc(bytes));
    RELNN_CUDA(cudaMemsetAsync(p.win_mask.p, 0, bytes, st));
    const int words = (p.d_out + 31) / 32;
    { win_mask_kernel<<<grid_of(p.n_out * words), 256, 0, st>>>(p.max_arg.as<int32_t>(), p.n_out, p.d_out, words, b.m,
                                                               p.win_mask.as<uint32_t>(), mw, p.status.as<int>()); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

}  // namespace relnn
