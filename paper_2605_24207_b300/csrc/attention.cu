// Attention over a join (paper Sec. 1: Score(p, t; q*k) :- Treat(p, t), Queries(p; q), Keys(t; k)
// and Attention(p; sum(a*v)) :- Score(p, t; a), Values(t; v); Sec. 5: the HGT attention head, a
// per-head softmax over t of the scaled dot product). On a plan's content track the rule's E(src =
// t, dst = p) tuples are already grouped by output key p, with hd = p's H row (q) and hs = t's H
// row (k, v), so one pass over the dst-sorted tuples evaluates
//   product: Out[p] = sum_t q_t * k_t * v_t                                  (element-wise)
//   softmax: Out[p][h] = sum_t a_t v_t[h],  a_t = softmax_t(scale * q_t . k_t over head h)
// with the softmax computed online (running maximum m, normaliser l, unnormalised sum) so every
// k and v row is read once. Each warp owns a range of consecutive tuples; lane j holds features
// [F j, F j + F) (F = d / 32), so a head's dot product is a partial sum over the lane's F features
// and log2(lanes per head) butterfly shuffles. A run cut by a range edge leaves its (m, l, sum)
// state as a boundary partial; the fix-up merges a row's partials in range order (rescaling by the
// running maxima) and writes the row and its log-sum-exp, which the backward uses to rebuild a_t.
//
// Backward: dv_t += a_t dOut_p, da_t = dOut_p . v_t, D_p = dOut_p . Out_p (per head), ds_t =
// scale a_t (da_t - D_p), dk_t += ds_t q_p, dq_p += ds_t k_t; the product head's gradients are the
// three two-factor products. Two walks: in output order dq is summed over runs of equal q rows; in
// src order (the plan's cached permutation) dk and dv are summed over runs of equal k / v rows, so
// each run, not each tuple, adds into the gradients.
#include "fwd.cuh"
#include "segfix.cuh"

#include <algorithm>
#include <cmath>

namespace relnn {

namespace {

constexpr int kSoftmax = RELNN_ATTN_SOFTMAX;
constexpr int kProduct = RELNN_ATTN_PRODUCT;

struct AttnArgs {
    const void* q;
    const void* k;
    const void* v;
    const int32_t *hs, *hd, *seg;
    int64_t m;
    int d, n_heads, lph;   // lanes per head (32 / n_heads)
    float scale;
    float* out;            // [n_out][d]
    float* lse;            // [n_out][n_heads] (softmax; may be null)
    float* carry;          // [n_ranges][2][cs]
    int cs;                // carry stride: hdr + d floats (a multiple of 4: every slot 16-byte aligned)
    int hdr;               // softmax: the slot's m[n_heads], l[n_heads] padded to a multiple of 4; product: 0
    int64_t n_ranges;
    int range_tiles;
    // backward
    const float* fout;     // forward output (softmax)
    const float* flse;     // forward log-sum-exp (softmax)
    const float* dout;
    float *dq, *dk, *dv;
    // src pass: the same tuples in src order (k and v rows non-decreasing), their q rows and
    // output rows, and D[p][h] = dOut_p . Out_p per head
    const int32_t *k_src, *q_src, *seg_src;
    const float* Dh;
};

// F consecutive elements of row `row` starting at column c (bf16 or f32), as f32.
template <int F, bool BF16>
__device__ __forceinline__ void load_f(const void* base, int64_t row, int d, int c, float (&x)[F]) {
    if (BF16) {
        const uint16_t* p = reinterpret_cast<const uint16_t*>(base) + row * d + c;
        if (F == 8) {
            const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                x[2 * i] = __uint_as_float(w[i] << 16);
                x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
            }
        } else if (F == 4) {
            const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
            x[0] = __uint_as_float(u.x << 16);
            x[1] = __uint_as_float(u.x & 0xffff0000u);
            x[2] = __uint_as_float(u.y << 16);
            x[3] = __uint_as_float(u.y & 0xffff0000u);
        } else if (F == 2) {
            const uint32_t u = __ldg(reinterpret_cast<const uint32_t*>(p));
            x[0] = __uint_as_float(u << 16);
            x[1] = __uint_as_float(u & 0xffff0000u);
        } else {
            x[0] = __uint_as_float((uint32_t)__ldg(p) << 16);
        }
    } else {
        const float* p = reinterpret_cast<const float*>(base) + row * d + c;
        if (F >= 4) {
#pragma unroll
            for (int i = 0; i < F; i += 4) {
                const float4 u = __ldg(reinterpret_cast<const float4*>(p + i));
                x[i] = u.x; x[i + 1] = u.y; x[i + 2] = u.z; x[i + 3] = u.w;
            }
        } else if (F == 2) {
            const float2 u = __ldg(reinterpret_cast<const float2*>(p));
            x[0] = u.x; x[1] = u.y;
        } else {
            x[0] = __ldg(p);
        }
    }
}

template <int F>
__device__ __forceinline__ void store_f(float* p, const float (&x)[F]) {
    if (F >= 4) {
#pragma unroll
        for (int i = 0; i < F; i += 4) __stcg(reinterpret_cast<float4*>(p + i), make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]));
    } else {
#pragma unroll
        for (int i = 0; i < F; ++i) __stcg(p + i, x[i]);
    }
}

template <int F>
__device__ __forceinline__ void atomic_add_f(float* p, const float (&x)[F]) {
    if (F >= 4) {
#pragma unroll
        for (int i = 0; i < F; i += 4) atomicAdd(reinterpret_cast<float4*>(p + i), make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]));
    } else if (F == 2) {
        atomicAdd(reinterpret_cast<float2*>(p), make_float2(x[0], x[1]));
    } else {
        atomicAdd(p, x[0]);
    }
}

// Sum over the lph lanes of a head (aligned groups of lph lanes; lph a power of two).
__device__ __forceinline__ float head_sum(float x, int lph) {
    for (int o = lph >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sum over the lph lanes of a head within the lanes of `mask` (aligned groups of lph lanes).
__device__ __forceinline__ float head_sum_m(float x, int lph, unsigned mask) {
    for (int o = lph >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
}

// Each group of G lanes (a warp, or a half-warp for narrow rows) owns one range of tuples; lane j of
// a group holds features [F j, F j + F) (F = d / G), and KIN tuples' k and v rows are loaded before
// any is used.
template <int F, bool BF16, int MODE, int G>
__global__ void __launch_bounds__(256) attn_fwd_kernel(AttnArgs a) {
    constexpr int KIN = G == 32 ? 4 : 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, grp = lane / G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (0xffffu << (16 * grp));
    const int64_t groups_total = (int64_t)gridDim.x * (blockDim.x >> 5) * (32 / G);
    const int64_t span = (int64_t)a.range_tiles * 32;
    const int lph = G / a.n_heads;          // lanes per head within the group
    const int c0 = gl * F;                  // this lane's first feature
    const int head = gl / lph;              // its head
    const bool head_lead = (gl % lph) == 0;
    for (int64_t rg = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * (32 / G) + grp; rg < a.n_ranges;
         rg += groups_total) {
        const int64_t r0 = rg * span, r1 = imin64(a.m, r0 + span);
        const int prev_seg = r0 > 0 ? a.seg[r0 - 1] : -1;
        const int next_seg = r1 < a.m ? a.seg[r1] : -1;
        int cur = -1, curq = -1;
        bool first = true;
        float qf[F], acc[F];
        float mx = -INFINITY, l = 0.f;
#pragma unroll
        for (int i = 0; i < F; ++i) qf[i] = acc[i] = 0.f;
        auto flush = [&](int s, bool last) {
            const bool split = (first && prev_seg == s) || (last && next_seg == s);
            if (split) {
                float* base = a.carry + (rg * 2 + (first ? 0 : 1)) * a.cs;
                if (MODE == kSoftmax) {
                    if (head_lead) {
                        __stcg(base + head, mx);
                        __stcg(base + a.n_heads + head, l);
                    }
                    store_f<F>(base + a.hdr + c0, acc);
                } else {
                    store_f<F>(base + c0, acc);
                }
            } else {
                if (MODE == kSoftmax) {
                    const float inv = 1.f / l;
                    float o[F];
#pragma unroll
                    for (int i = 0; i < F; ++i) o[i] = acc[i] * inv;
                    store_f<F>(a.out + (int64_t)s * a.d + c0, o);
                    if (a.lse && head_lead) a.lse[(int64_t)s * a.n_heads + head] = mx + logf(l);
                } else {
                    store_f<F>(a.out + (int64_t)s * a.d + c0, acc);
                }
            }
#pragma unroll
            for (int i = 0; i < F; ++i) acc[i] = 0.f;
            mx = -INFINITY;
            l = 0.f;
            first = false;
        };
        for (int64_t b0 = r0; b0 < r1; b0 += G) {
            const int nb = (int)imin64(G, r1 - b0);
            const bool tv = gl < nb;
            const int sv = tv ? a.seg[b0 + gl] : -1;
            const int kv = tv ? a.hs[b0 + gl] : 0;
            const int qv = tv ? a.hd[b0 + gl] : 0;
            for (int j0 = 0; j0 < nb; j0 += KIN) {
                float kf[KIN][F], vf[KIN][F];
                int sj[KIN], qj[KIN];
#pragma unroll
                for (int u = 0; u < KIN; ++u) {
                    const int j = j0 + u < nb ? j0 + u : nb - 1;
                    sj[u] = __shfl_sync(gmask, sv, j, G);
                    qj[u] = __shfl_sync(gmask, qv, j, G);
                    const int kr = __shfl_sync(gmask, kv, j, G);
                    load_f<F, BF16>(a.k, kr, a.d, c0, kf[u]);
                    load_f<F, BF16>(a.v, kr, a.d, c0, vf[u]);
                }
#pragma unroll
                for (int u = 0; u < KIN; ++u) {
                    if (j0 + u >= nb) break;
                    if (sj[u] != cur) {
                        if (cur >= 0) flush(cur, false);
                        cur = sj[u];
                    }
                    if (qj[u] != curq) {
                        load_f<F, BF16>(a.q, qj[u], a.d, c0, qf);
                        curq = qj[u];
                    }
                    if (MODE == kProduct) {
#pragma unroll
                        for (int i = 0; i < F; ++i) acc[i] = fmaf(qf[i] * kf[u][i], vf[u][i], acc[i]);
                    } else {
                        float p = 0.f;
#pragma unroll
                        for (int i = 0; i < F; ++i) p = fmaf(qf[i], kf[u][i], p);
                        const float sc = head_sum_m(p, lph, gmask) * a.scale;
                        const float mn = fmaxf(mx, sc);
                        const float corr = __expf(mx - mn);
                        const float e = __expf(sc - mn);
                        l = fmaf(l, corr, e);
#pragma unroll
                        for (int i = 0; i < F; ++i) acc[i] = fmaf(acc[i], corr, e * vf[u][i]);
                        mx = mn;
                    }
                }
            }
        }
        if (cur >= 0) flush(cur, true);
    }
}

// Softmax fix-up: a row cut by range edges has one (m, l, sum) partial per range piece (slot layout:
// m[n_heads], l[n_heads], padding to hdr floats, then the d unnormalised sums); merged in
// range order: M = max m_i, L = sum l_i e^(m_i - M), S = sum s_i e^(m_i - M); Out = S / L.
template <int F>
__global__ void attn_fixup_kernel(AttnArgs a, int tile, int64_t n_tiles) {
    const int lane = threadIdx.x & 31;
    const int c0 = lane * F, head = lane / a.lph;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) + 1; b < n_tiles; b += nwarps) {
        int s, fs;
        int64_t e;
        if (!first_cut(a.seg, a.m, tile, b, lane, s, fs, e)) continue;
        const int64_t P = e - b + 2;
        float M = -INFINITY, L = 0.f, S[F];
#pragma unroll
        for (int i = 0; i < F; ++i) S[i] = 0.f;
        for (int64_t i = 0; i < P; ++i) {
            const float* base = a.carry + piece_slot(b, fs, i) * a.cs;
            const float mi = base[head], li = base[a.n_heads + head];
            const float mn = fmaxf(M, mi);
            const float c1 = __expf(M - mn), c2 = __expf(mi - mn);
            L = L * c1 + li * c2;
#pragma unroll
            for (int j = 0; j < F; ++j) S[j] = S[j] * c1 + base[a.hdr + c0 + j] * c2;
            M = mn;
        }
        const float inv = 1.f / L;
#pragma unroll
        for (int j = 0; j < F; ++j) S[j] *= inv;
        store_f<F>(a.out + (int64_t)s * a.d + c0, S);
        if (a.lse && lane % a.lph == 0) a.lse[(int64_t)s * a.n_heads + head] = M + logf(L);
    }
}

template <int F, bool BF16, int MODE>
__global__ void __launch_bounds__(256) attn_bwd_kernel(AttnArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int64_t span = (int64_t)a.range_tiles * 32;
    const int c0 = lane * F, head = lane / a.lph;
    for (int64_t rg = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; rg < a.n_ranges; rg += warps_total) {
        const int64_t r0 = rg * span, r1 = imin64(a.m, r0 + span);
        int cur = -1, curq = -1;
        float go[F], qf[F], dqa[F];
        float L = 0.f, D = 0.f;
#pragma unroll
        for (int i = 0; i < F; ++i) go[i] = qf[i] = dqa[i] = 0.f;
        auto flush_q = [&]() {
            if (curq >= 0 && a.dq) atomic_add_f<F>(a.dq + (int64_t)curq * a.d + c0, dqa);
#pragma unroll
            for (int i = 0; i < F; ++i) dqa[i] = 0.f;
        };
        for (int64_t b0 = r0; b0 < r1; b0 += 32) {
            const int nb = (int)imin64(32, r1 - b0);
            const bool tv = lane < nb;
            const int sv = tv ? a.seg[b0 + lane] : -1;
            const int kv = tv ? a.hs[b0 + lane] : 0;
            const int qv = tv ? a.hd[b0 + lane] : 0;
            for (int j0 = 0; j0 < nb; j0 += 4) {
                float kf[4][F], vf[4][F];
                int sj[4], qj[4], kj[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u < nb ? j0 + u : nb - 1;
                    sj[u] = __shfl_sync(0xffffffffu, sv, j);
                    qj[u] = __shfl_sync(0xffffffffu, qv, j);
                    kj[u] = __shfl_sync(0xffffffffu, kv, j);
                    load_f<F, BF16>(a.k, kj[u], a.d, c0, kf[u]);
                    load_f<F, BF16>(a.v, kj[u], a.d, c0, vf[u]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (j0 + u >= nb) break;
                    if (sj[u] != cur) {
                        cur = sj[u];
                        load_f<F, false>(a.dout, cur, a.d, c0, go);
                        if (MODE == kSoftmax) {
                            float fo[F];
                            load_f<F, false>(a.fout, cur, a.d, c0, fo);
                            float p = 0.f;
#pragma unroll
                            for (int i = 0; i < F; ++i) p = fmaf(go[i], fo[i], p);
                            D = head_sum(p, a.lph);
                            L = a.flse[(int64_t)cur * a.n_heads + head];
                        }
                    }
                    if (qj[u] != curq) {
                        flush_q();
                        curq = qj[u];
                        load_f<F, BF16>(a.q, curq, a.d, c0, qf);
                    }
                    float gk[F], gv[F];
                    if (MODE == kProduct) {
#pragma unroll
                        for (int i = 0; i < F; ++i) {
                            gv[i] = go[i] * qf[i] * kf[u][i];
                            gk[i] = go[i] * qf[i] * vf[u][i];
                            dqa[i] = fmaf(go[i] * kf[u][i], vf[u][i], dqa[i]);
                        }
                    } else {
                        float p = 0.f, pv = 0.f;
#pragma unroll
                        for (int i = 0; i < F; ++i) {
                            p = fmaf(qf[i], kf[u][i], p);
                            pv = fmaf(go[i], vf[u][i], pv);
                        }
                        const float sc = head_sum(p, a.lph) * a.scale;
                        const float da = head_sum(pv, a.lph);
                        const float at = __expf(sc - L);
                        const float ds = at * (da - D) * a.scale;
#pragma unroll
                        for (int i = 0; i < F; ++i) {
                            gv[i] = at * go[i];
                            gk[i] = ds * qf[i];
                            dqa[i] = fmaf(ds, kf[u][i], dqa[i]);
                        }
                    }
                    if (a.dv) atomic_add_f<F>(a.dv + (int64_t)kj[u] * a.d + c0, gv);
                    if (a.dk) atomic_add_f<F>(a.dk + (int64_t)kj[u] * a.d + c0, gk);
                }
            }
        }
        flush_q();
    }
}

// D[p][h] = dOut_p . Out_p over head h's features (one warp per output row).
template <int F>
__global__ void attn_dterm_kernel(AttnArgs a, int64_t n_out, float* D) {
    const int lane = threadIdx.x & 31;
    const int c0 = lane * F, head = lane / a.lph;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_out; p += nw) {
        float g[F], o[F];
        load_f<F, false>(a.dout, p, a.d, c0, g);
        load_f<F, false>(a.fout, p, a.d, c0, o);
        float x = 0.f;
#pragma unroll
        for (int i = 0; i < F; ++i) x = fmaf(g[i], o[i], x);
        x = head_sum(x, a.lph);
        if (lane % a.lph == 0) D[p * a.n_heads + head] = x;
    }
}

__global__ void gather_rows_kernel(const int32_t* idx, const int32_t* perm, int64_t m, int32_t* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = idx[perm[i]];
}

// Backward, src pass: the tuples in src order, so a k / v row stays in registers over its run and
// dk, dv receive one atomic add per run; per tuple the q row, the dOut row and (softmax) the row's
// log-sum-exp and D are gathered.
template <int F, bool BF16, int MODE>
__global__ void __launch_bounds__(256) attn_bwd_src_kernel(AttnArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int64_t span = (int64_t)a.range_tiles * 32;
    const int c0 = lane * F, head = lane / a.lph;
    for (int64_t rg = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; rg < a.n_ranges; rg += warps_total) {
        const int64_t r0 = rg * span, r1 = imin64(a.m, r0 + span);
        int curk = -1;
        float kf[F], vf[F], dka[F], dva[F];
#pragma unroll
        for (int i = 0; i < F; ++i) kf[i] = vf[i] = dka[i] = dva[i] = 0.f;
        auto flush = [&]() {
            if (curk >= 0) {
                if (a.dk) atomic_add_f<F>(a.dk + (int64_t)curk * a.d + c0, dka);
                if (a.dv) atomic_add_f<F>(a.dv + (int64_t)curk * a.d + c0, dva);
            }
#pragma unroll
            for (int i = 0; i < F; ++i) dka[i] = dva[i] = 0.f;
        };
        for (int64_t b0 = r0; b0 < r1; b0 += 32) {
            const int nb = (int)imin64(32, r1 - b0);
            const bool tv = lane < nb;
            const int sv = tv ? a.seg_src[b0 + lane] : 0;
            const int kv = tv ? a.k_src[b0 + lane] : 0;
            const int qv = tv ? a.q_src[b0 + lane] : 0;
            for (int j0 = 0; j0 < nb; j0 += 4) {
                float qf[4][F], gf[4][F], Lj[4], Dj[4];
                int kj[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u < nb ? j0 + u : nb - 1;
                    const int sj = __shfl_sync(0xffffffffu, sv, j);
                    kj[u] = __shfl_sync(0xffffffffu, kv, j);
                    load_f<F, BF16>(a.q, __shfl_sync(0xffffffffu, qv, j), a.d, c0, qf[u]);
                    load_f<F, false>(a.dout, sj, a.d, c0, gf[u]);
                    if (MODE == kSoftmax) {
                        Lj[u] = __ldg(a.flse + (int64_t)sj * a.n_heads + head);
                        Dj[u] = __ldg(a.Dh + (int64_t)sj * a.n_heads + head);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (j0 + u >= nb) break;
                    if (kj[u] != curk) {
                        flush();
                        curk = kj[u];
                        load_f<F, BF16>(a.k, curk, a.d, c0, kf);
                        load_f<F, BF16>(a.v, curk, a.d, c0, vf);
                    }
                    if (MODE == kProduct) {
#pragma unroll
                        for (int i = 0; i < F; ++i) {
                            const float gq = gf[u][i] * qf[u][i];
                            dva[i] = fmaf(gq, kf[i], dva[i]);
                            dka[i] = fmaf(gq, vf[i], dka[i]);
                        }
                    } else {
                        float p = 0.f, pv = 0.f;
#pragma unroll
                        for (int i = 0; i < F; ++i) {
                            p = fmaf(qf[u][i], kf[i], p);
                            pv = fmaf(gf[u][i], vf[i], pv);
                        }
                        const float sc = head_sum(p, a.lph) * a.scale;
                        const float da = head_sum(pv, a.lph);
                        const float at = __expf(sc - Lj[u]);
                        const float ds = at * (da - Dj[u]) * a.scale;
#pragma unroll
                        for (int i = 0; i < F; ++i) {
                            dva[i] = fmaf(at, gf[u][i], dva[i]);
                            dka[i] = fmaf(ds, qf[u][i], dka[i]);
                        }
                    }
                }
            }
        }
        flush();
    }
}

template <class K>
void range_launch(K kern, AttnArgs& a, cudaStream_t st, int& bps_cache, int groups_per_warp = 1) {
    if (bps_cache <= 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_cache, kern, 256, 0) != cudaSuccess) {
        (void)cudaGetLastError();  // sizes the ranges only: assume one block per SM
        bps_cache = 1;
    }
    const int bps = std::max(1, bps_cache);
    const int64_t n32 = ceil_div(a.m, 32);
    const int64_t resident = (int64_t)bps * num_sms() * 8 * groups_per_warp;
    a.range_tiles = (int)std::min<int64_t>(ceil_div(n32, resident), 1 << 20);
    a.n_ranges = ceil_div(n32, a.range_tiles);
}

// F = d / 32 (the fix-up's warp layout); the walk runs half-warp groups (2F features per lane) for
// rows of up to 128 features with at most 16 heads, whole warps otherwise.
template <int F, bool BF16>
relnn_status attn_forward_t(Plan& p, AttnArgs& a, int mode, cudaStream_t st) {
    static int bps[4] = {0, 0, 0, 0};
    const int grid_cap = num_sms() * 8;
    constexpr int FH = F <= 4 ? 2 * F : F;  // features per lane in a half-warp group
    const bool half = F <= 4 && (mode == kProduct || a.n_heads <= 16);
    if (mode == kSoftmax) {
        if (half) range_launch(attn_fwd_kernel<FH, BF16, kSoftmax, 16>, a, st, bps[0], 2);
        else range_launch(attn_fwd_kernel<F, BF16, kSoftmax, 32>, a, st, bps[1]);
        a.hdr = (2 * a.n_heads + 3) & ~3;
    } else {
        if (half) range_launch(attn_fwd_kernel<FH, BF16, kProduct, 16>, a, st, bps[2], 2);
        else range_launch(attn_fwd_kernel<F, BF16, kProduct, 32>, a, st, bps[3]);
        a.hdr = 0;
    }
    a.cs = a.hdr + a.d;  // d is a multiple of 32, so cs is a multiple of 4 floats
    RELNN_TRY(p.carry.alloc(sizeof(float) * 2 * (size_t)a.cs * a.n_ranges));
    a.carry = p.carry.as<float>();
    const int grid = (int)std::min<int64_t>(ceil_div(a.n_ranges, half ? 16 : 8), grid_cap);
    ProfToken pt = prof_begin(RELNN_PROF_FWD_FP32, st);
    if (mode == kSoftmax) {
        if (half) attn_fwd_kernel<FH, BF16, kSoftmax, 16><<<grid, 256, 0, st>>>(a);
        else attn_fwd_kernel<F, BF16, kSoftmax, 32><<<grid, 256, 0, st>>>(a);
    } else {
        if (half) attn_fwd_kernel<FH, BF16, kProduct, 16><<<grid, 256, 0, st>>>(a);
        else attn_fwd_kernel<F, BF16, kProduct, 32><<<grid, 256, 0, st>>>(a);
    }
    note_launch();
    prof_end(pt, st);
    RELNN_CUDA(cudaGetLastError());
    const int tile = a.range_tiles * 32;
    if (a.n_ranges > 1) {
        if (mode == kSoftmax) {
            ProfToken pf = prof_begin(RELNN_PROF_FIXUP, st);
            { attn_fixup_kernel<F><<<(int)std::min<int64_t>(ceil_div(a.n_ranges - 1, 8), grid_cap), 256, 0, st>>>(
                  a, tile, a.n_ranges); note_launch(); }
            prof_end(pf, st);
        } else {
            RELNN_TRY(launch_fixup(a.seg, a.m, tile, a.n_ranges, a.carry, a.out, a.d, false, false, p.fixjobs, st));
        }
        RELNN_CUDA(cudaGetLastError());
    }
    return RELNN_OK;
}

// Two walks: the dst pass (output order) sums dq over runs of equal q rows; the src pass (src order)
// sums dk and dv over runs of equal k / v rows, so no per-tuple atomics remain.
template <int F, bool BF16>
relnn_status attn_backward_t(Plan& p, AttnArgs& a, int mode, cudaStream_t st) {
    static int bps[4] = {0, 0, 0, 0};
    const int cap = num_sms() * 8;
    BranchPlan& b = p.br[0];
    const bool need_kv = a.dk || a.dv;
    float* dk = a.dk;
    float* dv = a.dv;
    if (need_kv) {
        RELNN_TRY(ensure_src_order(p, b, st));
        const size_t dbytes = mode == kSoftmax ? sizeof(float) * (size_t)p.n_out * a.n_heads : 0;
        RELNN_TRY(p.scratch.alloc(sizeof(int32_t) * (size_t)b.m + dbytes + 256));
        int32_t* q_src = p.scratch.as<int32_t>();
        { gather_rows_kernel<<<(int)std::min<int64_t>(ceil_div(b.m, 256), cap), 256, 0, st>>>(
              b.hd.as<int32_t>(), b.src_perm.as<int32_t>(), b.m, q_src); note_launch(); }
        a.q_src = q_src;
        a.k_src = b.hs_src.as<int32_t>();
        a.seg_src = b.seg_src.as<int32_t>();
        if (mode == kSoftmax) {
            float* D = reinterpret_cast<float*>(p.scratch.as<uint8_t>() + ((sizeof(int32_t) * (size_t)b.m + 255) & ~(size_t)255));
            { attn_dterm_kernel<F><<<(int)std::min<int64_t>(ceil_div(p.n_out, 8), cap), 256, 0, st>>>(a, p.n_out, D); note_launch(); }
            a.Dh = D;
        }
    }
    ProfToken pt = prof_begin(RELNN_PROF_BWD_FP32, st);
    // dst pass: dq only
    a.dk = a.dv = nullptr;
    if (a.dq) {
        if (mode == kSoftmax) {
            range_launch(attn_bwd_kernel<F, BF16, kSoftmax>, a, st, bps[0]);
            attn_bwd_kernel<F, BF16, kSoftmax><<<(int)std::min<int64_t>(ceil_div(a.n_ranges, 8), cap), 256, 0, st>>>(a);
        } else {
            range_launch(attn_bwd_kernel<F, BF16, kProduct>, a, st, bps[1]);
            attn_bwd_kernel<F, BF16, kProduct><<<(int)std::min<int64_t>(ceil_div(a.n_ranges, 8), cap), 256, 0, st>>>(a);
        }
        note_launch();
    }
    // src pass: dk, dv
    a.dk = dk;
    a.dv = dv;
    if (need_kv) {
        if (mode == kSoftmax) {
            range_launch(attn_bwd_src_kernel<F, BF16, kSoftmax>, a, st, bps[2]);
            attn_bwd_src_kernel<F, BF16, kSoftmax><<<(int)std::min<int64_t>(ceil_div(a.n_ranges, 8), cap), 256, 0, st>>>(a);
        } else {
            range_launch(attn_bwd_src_kernel<F, BF16, kProduct>, a, st, bps[3]);
            attn_bwd_src_kernel<F, BF16, kProduct><<<(int)std::min<int64_t>(ceil_div(a.n_ranges, 8), cap), 256, 0, st>>>(a);
        }
        note_launch();
    }
    prof_end(pt, st);
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

relnn_status check_attn(const Plan& p, const relnn_attn_params* prm) {
    RELNN_CHECK_ARG(prm && prm->d_q && prm->d_k && prm->d_v, "attention: null rows");
    RELNN_CHECK_ARG(p.br.size() == 1 && p.join_dst && p.br[0].d_r == 0 && !(p.flags & kPlanDense),
                    "attention: single-branch plan with a dst join and no per-tuple embedding");
    RELNN_CHECK_ARG(prm->mode == kSoftmax || prm->mode == kProduct, "attention: bad mode");
    RELNN_CHECK_ARG(prm->d == 32 || prm->d == 64 || prm->d == 128 || prm->d == 256, "attention: d in {32, 64, 128, 256}");
    RELNN_CHECK_ARG(prm->d_val == prm->d, "attention: the width of v must equal d");
    const int h = prm->n_heads;
    RELNN_CHECK_ARG(h >= 1 && h <= 32 && (h & (h - 1)) == 0, "attention: n_heads a power of two <= 32");
    RELNN_CHECK_ARG(prm->dtype == RELNN_F32 || prm->dtype == RELNN_BF16, "attention: bad dtype");
    const uintptr_t al = reinterpret_cast<uintptr_t>(prm->d_q) | reinterpret_cast<uintptr_t>(prm->d_k) |
                         reinterpret_cast<uintptr_t>(prm->d_v);
    RELNN_CHECK_ARG((al & 15u) == 0, "attention: q, k, v must be 16-byte aligned");
    return RELNN_OK;
}

AttnArgs make_args(const Plan& p, const relnn_attn_params* prm) {
    const BranchPlan& b = p.br[0];
    AttnArgs a{};
    a.q = prm->d_q;
    a.k = prm->d_k;
    a.v = prm->d_v;
    a.hs = b.hs.as<int32_t>();
    a.hd = b.hd.as<int32_t>();
    a.seg = b.seg.as<int32_t>();
    a.m = b.m;
    a.d = prm->d;
    a.n_heads = prm->mode == kSoftmax ? prm->n_heads : 1;
    a.lph = 32 / a.n_heads;
    a.scale = prm->scale;
    return a;
}

template <bool BF16>
relnn_status dispatch_fwd(Plan& p, AttnArgs& a, int mode, cudaStream_t st) {
    switch (a.d / 32) {
        case 1: return attn_forward_t<1, BF16>(p, a, mode, st);
        case 2: return attn_forward_t<2, BF16>(p, a, mode, st);
        case 4: return attn_forward_t<4, BF16>(p, a, mode, st);
        default: return attn_forward_t<8, BF16>(p, a, mode, st);
    }
}

template <bool BF16>
relnn_status dispatch_bwd(Plan& p, AttnArgs& a, int mode, cudaStream_t st) {
    switch (a.d / 32) {
        case 1: return attn_backward_t<1, BF16>(p, a, mode, st);
        case 2: return attn_backward_t<2, BF16>(p, a, mode, st);
        case 4: return attn_backward_t<4, BF16>(p, a, mode, st);
        default: return attn_backward_t<8, BF16>(p, a, mode, st);
    }
}

}  // namespace

relnn_status attention_forward(Plan& p, const relnn_attn_params* prm, float* out, float* lse, cudaStream_t st) {
    RELNN_TRY(check_attn(p, prm));
    if (p.n_out == 0 || p.br[0].m == 0) return RELNN_OK;
    RELNN_CHECK_ARG(out && (reinterpret_cast<uintptr_t>(out) & 15u) == 0, "attention: null or unaligned output");
    AttnArgs a = make_args(p, prm);
    a.out = out;
    a.lse = prm->mode == kSoftmax ? lse : nullptr;
    return prm->dtype == RELNN_BF16 ? dispatch_fwd<true>(p, a, prm->mode, st) : dispatch_fwd<false>(p, a, prm->mode, st);
}

relnn_status attention_backward(Plan& p, const relnn_attn_params* prm, const float* fout, const float* flse,
                                const float* dout, float* dq, float* dk, float* dv, cudaStream_t st) {
    RELNN_TRY(check_attn(p, prm));
    const size_t rows = sizeof(float) * (size_t)p.n_h * prm->d;
    if (dq) RELNN_CUDA(cudaMemsetAsync(dq, 0, rows, st));
    if (dk) RELNN_CUDA(cudaMemsetAsync(dk, 0, rows, st));
    if (dv) RELNN_CUDA(cudaMemsetAsync(dv, 0, rows, st));
    if (p.n_out == 0 || p.br[0].m == 0) return RELNN_OK;
    RELNN_CHECK_ARG(dout, "attention backward: null output gradient");
    RELNN_CHECK_ARG(prm->mode != kSoftmax || (fout && flse), "attention backward: softmax needs the forward's output and log-sum-exp");
    const uintptr_t al = reinterpret_cast<uintptr_t>(fout) | reinterpret_cast<uintptr_t>(dout) |
                         reinterpret_cast<uintptr_t>(dq) | reinterpret_cast<uintptr_t>(dk) | reinterpret_cast<uintptr_t>(dv);
    RELNN_CHECK_ARG((al & 15u) == 0, "attention backward: buffers must be 16-byte aligned");
    AttnArgs a = make_args(p, prm);
    a.fout = fout;
    a.flse = flse;
    a.dout = dout;
    a.dq = dq;
    a.dk = dk;
    a.dv = dv;
    return prm->dtype == RELNN_BF16 ? dispatch_bwd<true>(p, a, prm->mode, st) : dispatch_bwd<false>(p, a, prm->mode, st);
}

}  // namespace relnn
