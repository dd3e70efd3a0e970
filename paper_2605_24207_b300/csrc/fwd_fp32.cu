// FP32 form of the rule forward: f32 FMA on CUDA cores (no TF32), used where the output must match
// the FP64 definition to ~1e-5 relative. One block owns 32-tuple tiles in turn; one thread owns one
// output feature o and keeps y[t][o] for the tile's 32 tuples in registers, so the SUM over a run of
// equal output rows is a sequential walk in registers (Sec. 2.2 projected union with SUM).
#include "agg.cuh"
#include "fwd.cuh"
#include "maxagg.cuh"

#include <algorithm>

namespace relnn {

namespace {

constexpr int kTT = 32;  // tuples per tile

struct Fp32Args {
    const void* z;
    int z_bf16, d;
    const void* r;
    int r_bf16, d_r;
    const float* Wt;     // [d_in][d_out] (transposed Linear weight), nullptr = identity
    const float* bias;   // [d_out] or nullptr
    const int32_t *hs, *hd, *er, *seg;
    int64_t m, n_tiles;
    int64_t n_ranges;    // lane kernel: ranges of range_tiles 32-tuple tiles, one warp each
    int range_tiles;
    int vec_in;          // widths multiples of 4 and rows aligned: 4-element loads
    int concat_dst, d_in, d_out, act, kahan, accumulate, w_in_smem;
    int maxagg;          // MAX aggregator (fwd_fp32_kernel only)
    float* out;
    float* carry;
    int32_t* arg;        // MAX: [n_out][d_out] plan position of each maximum (-1: ReLU'd zero)
    int32_t* carry_pos;  // MAX: positions of the boundary partials
};

__device__ __forceinline__ float load_elem(const void* base, int bf16, int64_t idx) {
    return bf16 ? bf16_to_f32(reinterpret_cast<const uint16_t*>(base)[idx])
                : reinterpret_cast<const float*>(base)[idx];
}

// Elements idx..idx+3 (idx a multiple of 4, the row base aligned to 4 elements).
__device__ __forceinline__ float4 load_elem4(const void* base, int bf16, int64_t idx) {
    if (bf16) {
        const uint2 u = *reinterpret_cast<const uint2*>(reinterpret_cast<const uint16_t*>(base) + idx);
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    }
    return *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(base) + idx);
}

__global__ void __launch_bounds__(256) fwd_fp32_kernel(Fp32Args a) {
    extern __shared__ float sm[];
    float* Ws = sm;                                            // [d_in][d_out] if w_in_smem
    float* X = sm + (a.w_in_smem ? (size_t)a.d_in * a.d_out : 0);  // [kTT][d_in]
    __shared__ int seg_s[kTT];
    const int tid = threadIdx.x;
    if (a.w_in_smem && a.Wt) {
        for (int i = tid; i < a.d_in * a.d_out; i += blockDim.x) Ws[i] = a.Wt[i];
    }
    const float* W = a.w_in_smem ? Ws : a.Wt;
    const int o = tid;
    const float bo = (a.bias && o < a.d_out) ? a.bias[o] : 0.f;
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const int64_t t0 = tile * kTT;
        const int nt = (int)imin64(kTT, a.m - t0);
        __syncthreads();  // previous tile's X fully consumed
        if (tid < kTT) seg_s[tid] = tid < nt ? a.seg[t0 + tid] : -1;
        for (int idx = tid; idx < nt * a.d_in; idx += blockDim.x) {
            const int t = idx / a.d_in, k = idx - t * a.d_in;
            float v;
            if (k < a.d) {
                v = load_elem(a.z, a.z_bf16, (int64_t)a.hs[t0 + t] * a.d + k);
            } else if (a.concat_dst && k < 2 * a.d) {
                v = load_elem(a.z, a.z_bf16, (int64_t)a.hd[t0 + t] * a.d + (k - a.d));
            } else {
                const int kr = k - (a.concat_dst ? 2 : 1) * a.d;
                v = load_elem(a.r, a.r_bf16, (int64_t)a.er[t0 + t] * a.d_r + kr);
            }
            X[t * a.d_in + k] = v;
        }
        __syncthreads();
        if (o >= a.d_out) continue;
        float y[kTT];
#pragma unroll
        for (int t = 0; t < kTT; ++t) y[t] = bo;
        if (W) {
            for (int k = 0; k < a.d_in; ++k) {
                const float w = W[k * a.d_out + o];
#pragma unroll
                for (int t = 0; t < kTT; ++t) y[t] = fmaf(X[t * a.d_in + k], w, y[t]);
            }
        } else {
#pragma unroll
            for (int t = 0; t < kTT; ++t) y[t] = t < nt ? X[t * a.d_in + o] : 0.f;
        }
        if (a.act == RELNN_ACT_RELU) {
#pragma unroll
            for (int t = 0; t < kTT; ++t) y[t] = fmaxf(y[t], 0.f);
        }
        const int prev_seg = t0 > 0 ? a.seg[t0 - 1] : -1;
        const int next_seg = t0 + nt < a.m ? a.seg[t0 + nt] : -1;
        float acc = 0.f, comp = 0.f;
        int rpos = 0;       // MAX: position of the piece's running maximum (first occurrence)
        bool fresh = true;  // the next tuple starts a piece
        bool first = true;
#pragma unroll
        for (int t = 0; t < kTT; ++t) {
            if (t < nt) {
                if (a.maxagg) {
                    if (fresh || y[t] > acc) {
                        acc = y[t];
                        rpos = (int)(t0 + t);
                    }
                } else if (a.kahan) {
                    kahan_add(acc, comp, y[t]);
                } else {
                    acc += y[t];
                }
                fresh = false;
                const int s = seg_s[t];
                const bool last = (t == nt - 1);
                const int sn = last ? next_seg : seg_s[t + 1 < kTT ? t + 1 : t];
                if (sn != s || last) {
                    const bool split = (first && prev_seg == s) || (last && sn == s);
                    if (split) {
                        const int64_t ci = (tile * 2 + (first ? 0 : 1)) * a.d_out + o;
                        a.carry[ci] = acc;
                        if (a.maxagg) a.carry_pos[ci] = rpos;
                    } else if (a.maxagg) {
                        a.out[(int64_t)s * a.d_out + o] = acc;
                        a.arg[(int64_t)s * a.d_out + o] = (a.act == RELNN_ACT_RELU && !(acc > 0.f)) ? -1 : rpos;
                    } else {
                        float* dst = a.out + (int64_t)s * a.d_out + o;
                        emit_out(dst, acc, a.accumulate);
                    }
                    acc = 0.f;
                    comp = 0.f;
                    fresh = true;
                    first = false;
                }
            }
        }
    }
}

// Narrow widths (d_in <= DIN, d_out <= DOUT): lane = tuple. A warp owns a range of range_tiles
// consecutive 32-tuple tiles; each lane loads its tuple's Concat row into registers, computes its
// d_out outputs with W^T broadcast from shared memory (4 outputs per shared load), and the SUM over
// each run of equal output rows is a segmented scan across the lanes (5 shuffle steps, the segment
// pattern computed once per tile). The lane holding a run's last tuple writes the row; a run that
// goes on into the next tile of the range leaves its partial in the warp's shared slot, where the
// next tile's first lane picks it up, so only the range's two boundary runs become fix-up partials.
template <int DIN, int DOUT>
__global__ void __launch_bounds__(256) fwd_fp32_lane_kernel(Fp32Args a) {
    extern __shared__ float sm[];
    float* Ws = sm;                                 // [d_in][DOUT] (zero beyond d_out), when there is a W
    float* bs = sm + (a.Wt ? DIN * DOUT : 0);       // [DOUT]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* cb = bs + DOUT + warp * 2 * DOUT;        // [DOUT] this warp's open-run partial
    float* cc = cb + DOUT;                          // [DOUT] and its compensation
    if (a.Wt) {
        for (int i = threadIdx.x; i < DIN * DOUT; i += blockDim.x) {
            const int k = i / DOUT, o = i - k * DOUT;
            Ws[i] = (k < a.d_in && o < a.d_out) ? a.Wt[k * a.d_out + o] : 0.f;
        }
    }
    for (int o = threadIdx.x; o < DOUT; o += blockDim.x) bs[o] = (a.bias && o < a.d_out) ? a.bias[o] : 0.f;
    __syncthreads();
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int64_t span = (int64_t)a.range_tiles * 32;
    for (int64_t rg = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; rg < a.n_ranges; rg += warps_total) {
        const int64_t r0 = rg * span, r1 = imin64(a.m, r0 + span);
        const int prev_seg = r0 > 0 ? a.seg[r0 - 1] : -1;
        bool first_run = true;  // no run of this range has ended yet
        bool open = false;      // the previous tile's last run goes on into this tile
        for (int64_t t0 = r0; t0 < r1; t0 += 32) {
            const int64_t t = t0 + lane;
            const bool tv = t < r1;
            const int nt = (int)imin64(32, r1 - t0);
            // this lane's Concat row (z[hs] | z[hd] | r[er])
            float x[DIN];
            const int64_t rs = tv ? (int64_t)a.hs[t] * a.d : 0;
            const int64_t rd = (tv && a.concat_dst) ? (int64_t)a.hd[t] * a.d : 0;
            const int64_t rr = (tv && a.d_r > 0) ? (int64_t)a.er[t] * a.d_r : 0;
            const int kr0 = a.concat_dst ? 2 * a.d : a.d;
            if (a.vec_in) {
#pragma unroll
                for (int k = 0; k < DIN; k += 4) {
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (tv && k < a.d_in) {
                        if (k < a.d) v = load_elem4(a.z, a.z_bf16, rs + k);
                        else if (k < kr0) v = load_elem4(a.z, a.z_bf16, rd + (k - a.d));
                        else v = load_elem4(a.r, a.r_bf16, rr + (k - kr0));
                    }
                    x[k] = v.x;
                    x[k + 1] = v.y;
                    x[k + 2] = v.z;
                    x[k + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int k = 0; k < DIN; ++k) {
                    float v = 0.f;
                    if (tv && k < a.d_in) {
                        if (k < a.d) v = load_elem(a.z, a.z_bf16, rs + k);
                        else if (k < kr0) v = load_elem(a.z, a.z_bf16, rd + (k - a.d));
                        else v = load_elem(a.r, a.r_bf16, rr + (k - kr0));
                    }
                    x[k] = v;
                }
            }
            float y[DOUT];
            if (a.Wt) {
#pragma unroll
                for (int o = 0; o < DOUT; ++o) y[o] = bs[o];
#pragma unroll
                for (int k = 0; k < DIN; ++k) {
                    const float4* wr = reinterpret_cast<const float4*>(Ws + k * DOUT);
#pragma unroll
                    for (int o4 = 0; o4 < DOUT / 4; ++o4) {
                        const float4 w = wr[o4];
                        y[4 * o4 + 0] = fmaf(x[k], w.x, y[4 * o4 + 0]);
                        y[4 * o4 + 1] = fmaf(x[k], w.y, y[4 * o4 + 1]);
                        y[4 * o4 + 2] = fmaf(x[k], w.z, y[4 * o4 + 2]);
                        y[4 * o4 + 3] = fmaf(x[k], w.w, y[4 * o4 + 3]);
                    }
                }
            } else {
#pragma unroll
                for (int o = 0; o < DOUT; ++o) y[o] = o < DIN ? x[o < DIN ? o : 0] : 0.f;
            }
            if (a.act == RELNN_ACT_RELU) {
#pragma unroll
                for (int o = 0; o < DOUT; ++o) y[o] = fmaxf(y[o], 0.f);
            }
            if (!tv) {
#pragma unroll
                for (int o = 0; o < DOUT; ++o) y[o] = 0.f;
            }
            // segment pattern of the tile: lane adds the value d lanes up at step d unless a run
            // start lies in between
            const int sg = tv ? a.seg[t] : -1;
            const int sg_prev = __shfl_up_sync(0xffffffffu, sg, 1);
            bool head = lane == 0 || sg_prev != sg;
            unsigned add_mask[5];
#pragma unroll
            for (int st = 0; st < 5; ++st) {
                const int dd = 1 << st;
                const bool up_head = __shfl_up_sync(0xffffffffu, head ? 1 : 0, dd) != 0;
                const bool add = lane >= dd && !head;
                add_mask[st] = add ? 1u : 0u;
                head = head || (add && up_head);
            }
#pragma unroll
            for (int o = 0; o < DOUT; ++o) {
#pragma unroll
                for (int st = 0; st < 5; ++st) {
                    const float u = __shfl_up_sync(0xffffffffu, y[o], 1 << st);
                    if (add_mask[st]) y[o] += u;
                }
            }
            // run ends: the next tuple has another output row, or the tile's last tuple unless its
            // run goes on into the next tile of the range
            const int sg_next = __shfl_down_sync(0xffffffffu, sg, 1);
            const int sg_last = __shfl_sync(0xffffffffu, sg, nt - 1);
            const int next_seg = (t0 + nt < a.m) ? a.seg[t0 + nt] : -1;
            const bool cont = next_seg == sg_last;
            const bool carry_on = cont && t0 + nt < r1;
            const bool last = lane == nt - 1;
            // the partial carried from the previous tile joins the tile's first run at that run's
            // last lane (compensated for compensated plans)
            const unsigned runends = __ballot_sync(0xffffffffu, tv && (last || sg_next != sg));
            const bool merge = open && lane == __ffs(runends) - 1;
            if (merge) {
#pragma unroll
                for (int o4 = 0; o4 < DOUT / 4; ++o4) {
                    float4 sv = reinterpret_cast<const float4*>(cb)[o4];
                    if (a.kahan) {
                        float4 cv = reinterpret_cast<const float4*>(cc)[o4];
                        kahan_add(sv.x, cv.x, y[4 * o4 + 0]);
                        kahan_add(sv.y, cv.y, y[4 * o4 + 1]);
                        kahan_add(sv.z, cv.z, y[4 * o4 + 2]);
                        kahan_add(sv.w, cv.w, y[4 * o4 + 3]);
                        reinterpret_cast<float4*>(cc)[o4] = cv;
                        y[4 * o4 + 0] = sv.x;
                        y[4 * o4 + 1] = sv.y;
                        y[4 * o4 + 2] = sv.z;
                        y[4 * o4 + 3] = sv.w;
                    } else {
                        y[4 * o4 + 0] += sv.x;
                        y[4 * o4 + 1] += sv.y;
                        y[4 * o4 + 2] += sv.z;
                        y[4 * o4 + 3] += sv.w;
                    }
                }
            }
            const bool end = tv && (last ? !carry_on : sg_next != sg);
            const unsigned endmask = __ballot_sync(0xffffffffu, end);
            if (last && carry_on) {  // a fresh carry starts without compensation
#pragma unroll
                for (int o4 = 0; o4 < DOUT / 4; ++o4) {
                    reinterpret_cast<float4*>(cb)[o4] =
                        make_float4(y[4 * o4 + 0], y[4 * o4 + 1], y[4 * o4 + 2], y[4 * o4 + 3]);
                    if (a.kahan && !merge) reinterpret_cast<float4*>(cc)[o4] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            if (end) {
                const bool first_piece = first_run && (endmask & ((1u << lane) - 1u)) == 0;
                const bool split = (first_piece && prev_seg == sg) || (last && cont);
                float* dst = split ? a.carry + (rg * 2 + (first_piece ? 0 : 1)) * a.d_out
                                   : a.out + (int64_t)sg * a.d_out;
#pragma unroll
                for (int o = 0; o < DOUT; ++o)
                    if (o < a.d_out) {
                        if (split) __stcg(dst + o, y[o]);
                        else emit_out(dst + o, y[o], a.accumulate);
                    }
            }
            first_run = first_run && endmask == 0;
            open = carry_on;
            __syncwarp();
        }
    }
}

// One warp per tile boundary b (1..n_tiles-1). The warp that sees the FIRST boundary crossed by a
// segment adds that segment's pieces in tile order and writes the output row. The five seg values
// the decision needs are fetched by five lanes at once; the last tile whose first row lies in the
// segment is the next tile unless the segment reaches past it (then one lane binary-searches).
// A segment cut into more than kLongPieces pieces is not summed by its first boundary's warp:
// that warp records it (first boundary, last tile, first slot, output row) for long_fixup_kernel.
constexpr int kLongPieces = 64;

__global__ void fixup_kernel(const int32_t* __restrict__ seg, int64_t m, int tile, int64_t n_tiles,
                             const float* __restrict__ carry, float* __restrict__ out, int d_out,
                             int accumulate, int kahan, int vec4, int* __restrict__ jobs, int max_jobs) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) + 1; b < n_tiles; b += nwarps) {
        const int64_t row = b * tile;  // < m because b < n_tiles = ceil(m / tile)
        int v = -1;
        if (lane == 0) v = seg[row];
        else if (lane == 1) v = seg[row - 1];
        else if (lane == 2) v = seg[(b - 1) * tile];
        else if (lane == 3 && b >= 2) v = seg[(b - 1) * tile - 1];
        else if (lane == 4 && row + tile < m) v = seg[row + tile];
        const int s = __shfl_sync(0xffffffffu, v, 0);
        const int s_before = __shfl_sync(0xffffffffu, v, 1);
        const int s_prev_first = __shfl_sync(0xffffffffu, v, 2);
        const int s_prev_before = __shfl_sync(0xffffffffu, v, 3);
        const int s_next_first = __shfl_sync(0xffffffffu, v, 4);
        if (s_before != s) continue;              // boundary b cuts no segment
        if (b >= 2 && s_prev_before == s) continue;  // not the first boundary of s
        const int first_slot = (s_prev_first == s) ? 0 : 1;
        int64_t e = b;  // last tile whose first row is in s (seg is non-decreasing)
        if (s_next_first == s) {
            int64_t last = 0;
            if (lane == 0) {
                int64_t lo = row + tile, hi = m;  // seg[lo] == s; the first row past s lies in (lo, m]
                while (lo + 1 < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (seg[mid] == s) lo = mid;
                    else hi = mid;
                }
                last = lo;
            }
            e = __shfl_sync(0xffffffffu, last, 0) / tile;
        }
        if (vec4 && jobs && e - b + 2 > kLongPieces) {
            if (lane == 0) {
                const int k = atomicAdd(jobs, 1);
                if (k < max_jobs) {
                    int4* jb = reinterpret_cast<int4*>(jobs + 4) + k;
                    *jb = make_int4((int)b, (int)e, first_slot, s);
                }
            }
            continue;
        }
        const float* c0 = carry + ((b - 1) * 2 + first_slot) * (int64_t)d_out;
        float* dst = out + (int64_t)s * d_out;
        if (vec4) {
            for (int o = lane * 4; o < d_out; o += 128) {
                // tiles b..e all start inside s (their slot 0 piece): added in tile order, with the
                // loads of 8 tiles in flight at a time
                float4 acc = *reinterpret_cast<const float4*>(c0 + o);
                float4 comp = make_float4(0.f, 0.f, 0.f, 0.f);
                auto add4 = [&](const float4& x) {
                    if (kahan) {
                        kahan_add(acc.x, comp.x, x.x); kahan_add(acc.y, comp.y, x.y);
                        kahan_add(acc.z, comp.z, x.z); kahan_add(acc.w, comp.w, x.w);
                    } else {
                        acc.x += x.x; acc.y += x.y; acc.z += x.z; acc.w += x.w;
                    }
                };
                int64_t j = b;
                for (; j + 7 <= e; j += 8) {
                    float4 x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) x[u] = *reinterpret_cast<const float4*>(carry + ((j + u) * 2) * (int64_t)d_out + o);
#pragma unroll
                    for (int u = 0; u < 8; ++u) add4(x[u]);
                }
                for (; j <= e; ++j) add4(*reinterpret_cast<const float4*>(carry + (j * 2) * (int64_t)d_out + o));
                if (accumulate) {
                    const float4 old = *reinterpret_cast<const float4*>(dst + o);
                    acc.x += old.x; acc.y += old.y; acc.z += old.z; acc.w += old.w;
                }
                __stcg(reinterpret_cast<float4*>(dst + o), acc);
            }
        } else {
            for (int o = lane; o < d_out; o += 32) {
                float acc = c0[o], comp = 0.f;
                for (int64_t j = b; j <= e; ++j) {
                    const float x = carry[(j * 2) * (int64_t)d_out + o];
                    if (kahan) kahan_add(acc, comp, x);
                    else acc += x;
                }
                emit_out(dst + o, acc, accumulate);
            }
        }
    }
}

// One block of 8 warps per recorded long segment: warp w adds the w-th eighth of the segment's
// pieces in order (8 loads in flight), the 8 partials are then added in warp order (compensated
// when kahan): a fixed order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) long_fixup_kernel(const int* __restrict__ jobs, int max_jobs,
                                                         const float* __restrict__ carry, float* __restrict__ out,
                                                         int d_out, int accumulate, int kahan) {
    __shared__ float4 part[8][64];  // d_out <= 256
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int njobs = min(jobs[0], max_jobs);
    for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
        const int4 J = reinterpret_cast<const int4*>(jobs + 4)[jb];
        const int64_t b = J.x, e = J.y;
        const int first_slot = J.z, s = J.w;
        // piece 0 = the first tile's cut piece, piece i >= 1 = slot 0 of tile b + i - 1
        const int64_t P = e - b + 2;
        const int64_t p0 = P * warp / 8, p1 = P * (warp + 1) / 8;
        auto piece = [&](int64_t i) -> const float* {
            return i == 0 ? carry + ((b - 1) * 2 + first_slot) * (int64_t)d_out
                          : carry + ((b + i - 1) * 2) * (int64_t)d_out;
        };
        for (int q = lane; q * 4 < d_out; q += 32) {
            const int o = q * 4;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f), comp = make_float4(0.f, 0.f, 0.f, 0.f);
            auto add4 = [&](const float4& x) {
                if (kahan) {
                    kahan_add(acc.x, comp.x, x.x); kahan_add(acc.y, comp.y, x.y);
                    kahan_add(acc.z, comp.z, x.z); kahan_add(acc.w, comp.w, x.w);
                } else {
                    acc.x += x.x; acc.y += x.y; acc.z += x.z; acc.w += x.w;
                }
            };
            int64_t i = p0;
            for (; i + 7 < p1; i += 8) {
                float4 x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u] = *reinterpret_cast<const float4*>(piece(i + u) + o);
#pragma unroll
                for (int u = 0; u < 8; ++u) add4(x[u]);
            }
            for (; i < p1; ++i) add4(*reinterpret_cast<const float4*>(piece(i) + o));
            part[warp][q] = acc;
        }
        __syncthreads();
        if (warp == 0) {
            float* dst = out + (int64_t)s * d_out;
            for (int q = lane; q * 4 < d_out; q += 32) {
                float4 acc = part[0][q], comp = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int w = 1; w < 8; ++w) {
                    const float4 x = part[w][q];
                    if (kahan) {
                        kahan_add(acc.x, comp.x, x.x); kahan_add(acc.y, comp.y, x.y);
                        kahan_add(acc.z, comp.z, x.z); kahan_add(acc.w, comp.w, x.w);
                    } else {
                        acc.x += x.x; acc.y += x.y; acc.z += x.z; acc.w += x.w;
                    }
                }
                if (accumulate) {
                    const float4 old = *reinterpret_cast<const float4*>(dst + q * 4);
                    acc.x += old.x; acc.y += old.y; acc.z += old.z; acc.w += old.w;
                }
                __stcg(reinterpret_cast<float4*>(dst + q * 4), acc);
            }
        }
        __syncthreads();
    }
}

// Wt[k][o] = W[o][k] in f32.
__global__ void transpose_w_kernel(const void* W, int w_bf16, int d_out, int d_in, float* Wt) {
    const int n = d_out * d_in;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = i / d_in, k = i - o * d_in;
        Wt[k * d_out + o] = w_bf16 ? bf16_to_f32(reinterpret_cast<const uint16_t*>(W)[i])
                                   : reinterpret_cast<const float*>(W)[i];
    }
}

}  // namespace

relnn_status launch_fixup(const int32_t* seg, int64_t m, int tile, int64_t n_tiles, const float* carry,
                          float* out, int d_out, bool accumulate, bool kahan, DevBuf& jobs_buf, cudaStream_t st) {
    if (n_tiles <= 1) return RELNN_OK;
    // one warp per boundary, 8 warps per block
    const int blocks = (int)std::min<int64_t>(ceil_div(n_tiles - 1, 8), (int64_t)num_sms() * 8);
    const bool vec4 = d_out % 4 == 0 && d_out <= 256 && (reinterpret_cast<uintptr_t>(out) & 15u) == 0 &&
                      (reinterpret_cast<uintptr_t>(carry) & 15u) == 0;
    // segments longer than kLongPieces pieces go to long_fixup_kernel (at most one per kLongPieces tiles)
    const bool split = vec4 && n_tiles > kLongPieces;
    const int max_jobs = split ? (int)(n_tiles / kLongPieces + 1) : 0;
    int* jobs = nullptr;
    if (split) {
        RELNN_TRY(jobs_buf.alloc(sizeof(int) * (4 + 4 * (size_t)max_jobs)));
        jobs = jobs_buf.as<int>();
        RELNN_CUDA(cudaMemsetAsync(jobs, 0, sizeof(int), st));
    }
    ProfToken pt = prof_begin(RELNN_PROF_FIXUP, st);
    { fixup_kernel<<<blocks, 256, 0, st>>>(seg, m, tile, n_tiles, carry, out, d_out, accumulate ? 1 : 0,
                                         kahan ? 1 : 0, vec4 ? 1 : 0, jobs, max_jobs); note_launch(); }
    if (split) {
        { long_fixup_kernel<<<num_sms(), 256, 0, st>>>(jobs, max_jobs, carry, out, d_out, accumulate ? 1 : 0,
                                                      kahan ? 1 : 0); note_launch(); }
    }
    prof_end(pt, st);
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

relnn_status forward_fp32(Plan& p, const CallIO& io, float* out, cudaStream_t st) {
    RELNN_CHECK_ARG(p.d_in <= 1024 && p.d_out <= 256, "FP32 form: d_in <= 1024 and d_out <= 256 required");
    // linear rules with narrow rows: the SUM first, then the Linear once per output row (agg.cu)
    if (agg_forward_fp32_ok(p, io, out)) return forward_agg_fp32(p, io, out, st);
    // identity rules (e.g. a SUM readout): the gather-sum alone
    if (agg_forward_identity_ok(p, io, out)) return forward_agg_identity(p, io, out, st);
    // several branches add into one output; a stream chunk adds into the stream's accumulator
    const bool multi = p.br.size() > 1 || p.acc_out;
    if (p.br.size() > 1 && !p.acc_out) RELNN_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * p.n_out * p.d_out, st));
    const int threads = std::max(32, ((p.d_out + 31) / 32) * 32);
    int64_t max_tiles = 1;
    for (auto& b : p.br) max_tiles = std::max<int64_t>(max_tiles, ceil_div(b.m, kTT));
    RELNN_TRY(p.carry.alloc(sizeof(float) * 2 * p.d_out * max_tiles));
    const bool maxagg = (p.flags & RELNN_FLAG_MAX) != 0;
    if (maxagg) {
        RELNN_CHECK_ARG(!multi, "MAX aggregator: single-branch rules only");
        RELNN_TRY(p.carry_pos.alloc(sizeof(int32_t) * 2 * p.d_out * max_tiles));
        RELNN_TRY(p.max_arg.alloc(sizeof(int32_t) * (size_t)p.n_out * p.d_out));
    }
    const size_t wt_bytes = sizeof(float) * p.d_in * p.d_out;
    RELNN_TRY(p.scratch.alloc(wt_bytes));
    const bool w_in_smem = !p.identity && wt_bytes <= 160 * 1024;
    const size_t smem = (w_in_smem ? wt_bytes : 0) + sizeof(float) * kTT * p.d_in;
    RELNN_CHECK_ARG(smem <= 220 * 1024, "FP32 form: tile does not fit in shared memory");
    RELNN_CUDA(cudaFuncSetAttribute(fwd_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        if (b.m == 0) continue;
        Fp32Args a{};
        a.z = io.z;
        a.z_bf16 = io.z_bf16;
        a.d = p.d;
        a.r = io.br[i].r;
        a.r_bf16 = io.r_bf16;
        a.d_r = b.d_r;
        if (!p.identity) {
            { transpose_w_kernel<<<64, 256, 0, st>>>(io.br[i].W, io.w_bf16, p.d_out, p.d_in, p.scratch.as<float>()); note_launch(); }
            a.Wt = p.scratch.as<float>();
            a.bias = io.br[i].b;
        }
        a.hs = b.hs.as<int32_t>();
        a.hd = b.hd.as<int32_t>();
        a.er = b.er.as<int32_t>();
        a.seg = b.seg.as<int32_t>();
        a.m = b.m;
        a.n_tiles = ceil_div(b.m, kTT);
        a.concat_dst = p.concat_dst;
        a.d_in = p.d_in;
        a.d_out = p.d_out;
        a.act = p.act;
        a.kahan = p.kahan;
        a.accumulate = multi;
        a.w_in_smem = w_in_smem;
        a.out = out;
        {
            const uintptr_t za = reinterpret_cast<uintptr_t>(io.z), ra = reinterpret_cast<uintptr_t>(a.r);
            const uintptr_t zmask = io.z_bf16 ? 7u : 15u, rmask = io.r_bf16 ? 7u : 15u;
            a.vec_in = p.d % 4 == 0 && (za & zmask) == 0 &&
                       (b.d_r == 0 || (b.d_r % 4 == 0 && (ra & rmask) == 0));
        }
        a.carry = p.carry.as<float>();
        if (maxagg) {
            a.maxagg = 1;
            a.arg = p.max_arg.as<int32_t>();
            a.carry_pos = p.carry_pos.as<int32_t>();
        }
        // narrow widths: the lane-per-tuple kernel (its in-tile sums are 5-level trees, whose error
        // bound is below that of a compensated 32-term walk; the fix-up compensates across tiles)
        // one wave of warps, each over an equal range of tiles
        int64_t fix_tile = kTT, fix_n = a.n_tiles;
        auto lane_launch = [&](auto kern, int din, int dout, int* bps_cache) -> bool {
            if (p.d_in > din || p.d_out > dout) return false;
            const size_t lsmem = sizeof(float) * ((a.Wt ? din * dout : 0) + dout + 16 * dout);
            int& bps = bps_cache[a.Wt ? 1 : 0];
            if (bps <= 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, lsmem) != cudaSuccess) {
                (void)cudaGetLastError();  // the query only sizes the ranges: assume one block per SM
                bps = 1;
            }
            bps = std::max(1, bps);
            const int64_t n32 = ceil_div(b.m, 32);
            const int64_t resident = (int64_t)bps * num_sms() * 8;
            a.range_tiles = (int)std::min<int64_t>(ceil_div(n32, resident), 1 << 20);
            a.n_ranges = ceil_div(n32, a.range_tiles);
            fix_tile = (int64_t)a.range_tiles * 32;
            fix_n = a.n_ranges;
            const int lgrid = (int)std::min<int64_t>(ceil_div(a.n_ranges, 8), (int64_t)bps * num_sms());
            { ProfToken pt = prof_begin(RELNN_PROF_FWD_FP32, st); kern<<<lgrid, 256, lsmem, st>>>(a); note_launch(); prof_end(pt, st); }
            return true;
        };
        static int bps64x64[2], bps32x16[2], bps32x32[2], bps64x16[2];
        // (MAX runs in the feature-per-thread kernel: a sequential walk keeps the first maximum)
        const bool lane_done = maxagg ? false : p.identity ? lane_launch(fwd_fp32_lane_kernel<64, 64>, 64, 64, bps64x64)
                                          : (lane_launch(fwd_fp32_lane_kernel<32, 16>, 32, 16, bps32x16) ||
                                             lane_launch(fwd_fp32_lane_kernel<32, 32>, 32, 32, bps32x32) ||
                                             lane_launch(fwd_fp32_lane_kernel<64, 16>, 64, 16, bps64x16));
        if (!lane_done) {
            const int grid = (int)std::min<int64_t>(a.n_tiles, (int64_t)num_sms() * (smem > 100 * 1024 ? 1 : 4));
            { ProfToken pt = prof_begin(RELNN_PROF_FWD_FP32, st); fwd_fp32_kernel<<<grid, threads, smem, st>>>(a); note_launch(); prof_end(pt, st); }
        }
        RELNN_CUDA(cudaGetLastError());
        if (maxagg)
            RELNN_TRY(launch_fixup_max(a.seg, a.m, (int)fix_tile, fix_n, a.carry, a.carry_pos, out, a.arg, p.d_out,
                                       p.act == RELNN_ACT_RELU, p.fixjobs, st));
        else
            RELNN_TRY(launch_fixup(a.seg, a.m, (int)fix_tile, fix_n, a.carry, out, p.d_out, multi, p.kahan, p.fixjobs, st));
        RELNN_CUDA(cudaGetLastError());
    }
    return RELNN_OK;
}

}  // namespace relnn
