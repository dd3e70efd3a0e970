// Transformation push-down below the join (the paper's future work, Sec. 6: apply the
// transformation to the embeddings once per node instead of once per edge).
//
// For a rule whose tau is a Linear (+ReLU) over Concat(z_src, z_dst) with no per-tuple embedding,
//   Y_t = act(W_src z[hs_t] + W_dst z[hd_t] + b) = act(P[hs_t] + Q[hd_t]),
//   P = Z W_src^T and Q = Z W_dst^T + b, one row per H row (Q = b when z_dst is not in the Concat),
// so the Linear runs once per H row instead of once per matched tuple. P and Q are dense products
// computed by the fused tensor-core forward on an identity plan (every H row its own tuple and
// output row); the per-tuple work is two f32 row gathers, an add, the activation and the SUM walk
// over runs of equal output rows (pd_sum_kernel). The result equals the per-tuple form up to the
// order of the f32 additions: the products see the same bf16 operands and accumulate in f32.
#include "fwd.cuh"

#include <algorithm>
#include <memory>

namespace relnn {

namespace {

__global__ void iota_kernel(int32_t* a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

// Ws[o][k] = W[o][col0 + k], k < d: one Concat part's column block of W, in W's dtype.
__global__ void w_cols_kernel(const void* W, int w_bf16, int d_out, int d_in, int col0, int d, void* Ws) {
    const int n = d_out * d;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = i / d, k = i - o * d;
        if (w_bf16) reinterpret_cast<uint16_t*>(Ws)[i] = reinterpret_cast<const uint16_t*>(W)[o * d_in + col0 + k];
        else reinterpret_cast<float*>(Ws)[i] = reinterpret_cast<const float*>(W)[o * d_in + col0 + k];
    }
}

struct PdArgs {
    const float* P;      // [n_h][d_out]
    const float* Q;      // [n_h][d_out], or nullptr (then bias per tuple)
    const float* bias;   // [d_out] when Q is nullptr (may be nullptr)
    const int32_t *hs, *hd, *seg;
    int64_t m;
    int d_out, act, kahan, accumulate, mask_words;
    uint32_t* relu_mask;  // [m][mask_words] or nullptr
    float* out;
    float* carry;         // [n_ranges][2][d_out]
    int64_t n_ranges;
    int range_tiles;
};

// One warp per range of range_tiles x 32 consecutive tuples (output order); lane l holds outputs
// l, l + 32, ..., so every row gather and every row store is a coalesced 128-byte access. A run of
// equal output rows is summed in registers and stored when it ends; the range's first run (if it
// began before the range) and last run (if it goes on after it) become boundary partials that the
// fix-up adds in range order. The indices of 32 tuples are loaded at once and handed out by
// shuffles; the rows of 4 tuples are loaded before any is added.
template <int F>
__global__ void __launch_bounds__(256) pd_sum_kernel(PdArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int64_t span = (int64_t)a.range_tiles * 32;
    const bool relu = a.act == RELNN_ACT_RELU;
    float qb[F];
#pragma unroll
    for (int f = 0; f < F; ++f) qb[f] = (!a.Q && a.bias) ? a.bias[32 * f + lane] : 0.f;
    for (int64_t rg = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; rg < a.n_ranges; rg += warps_total) {
        const int64_t r0 = rg * span, r1 = imin64(a.m, r0 + span);
        const int prev_seg = r0 > 0 ? a.seg[r0 - 1] : -1;
        const int next_seg = r1 < a.m ? a.seg[r1] : -1;
        int cur = -1;
        bool first = true;
        float acc[F], comp[F];
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f] = comp[f] = 0.f;
        // a run of output row s ends inside the range (last = false) or at the range's end
        auto flush = [&](int s, bool last) {
            const bool split = (first && prev_seg == s) || (last && next_seg == s);
            float* dst = split ? a.carry + (rg * 2 + (first ? 0 : 1)) * a.d_out : a.out + (int64_t)s * a.d_out;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (split) __stcg(dst + 32 * f + lane, acc[f]);
                else emit_out(dst + 32 * f + lane, acc[f], a.accumulate);
                acc[f] = comp[f] = 0.f;
            }
            first = false;
        };
        for (int64_t b0 = r0; b0 < r1; b0 += 32) {
            const int nb = (int)imin64(32, r1 - b0);
            const bool tv = lane < nb;
            const int sv = tv ? a.seg[b0 + lane] : -1;
            const int hv = tv ? a.hs[b0 + lane] : 0;
            const int dv = (tv && a.Q) ? a.hd[b0 + lane] : 0;
            uint32_t mw[F];  // this lane's tuple's mask words (tuple b0 + lane)
#pragma unroll
            for (int f = 0; f < F; ++f) mw[f] = 0u;
            for (int j0 = 0; j0 < nb; j0 += 4) {
                float y[4][F];
                int sj[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u < nb ? j0 + u : nb - 1;
                    sj[u] = __shfl_sync(0xffffffffu, sv, j);
                    const int64_t ph = (int64_t)__shfl_sync(0xffffffffu, hv, j) * a.d_out;
                    const int64_t qh = (int64_t)__shfl_sync(0xffffffffu, dv, j) * a.d_out;
#pragma unroll
                    for (int f = 0; f < F; ++f)
                        y[u][f] = __ldg(a.P + ph + 32 * f + lane) + (a.Q ? __ldg(a.Q + qh + 32 * f + lane) : qb[f]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (j0 + u >= nb) break;
                    if (sj[u] != cur) {
                        if (cur >= 0) flush(cur, false);
                        cur = sj[u];
                    }
#pragma unroll
                    for (int f = 0; f < F; ++f) {
                        float v = y[u][f];
                        if (relu) {
                            if (a.relu_mask) {
                                const unsigned w = __ballot_sync(0xffffffffu, v > 0.f);
                                if (lane == j0 + u) mw[f] = w;
                            }
                            v = fmaxf(v, 0.f);
                        }
                        if (a.kahan) kahan_add(acc[f], comp[f], v);
                        else acc[f] += v;
                    }
                }
            }
            if (a.relu_mask && tv) {
#pragma unroll
                for (int f = 0; f < F; ++f) a.relu_mask[(b0 + lane) * a.mask_words + f] = mw[f];
            }
        }
        if (cur >= 0) flush(cur, true);
    }
}

// The same walk in half-warp groups when no ReLU mask is kept and d_out is 64 or 128: each group of
// 16 lanes owns a range, lane j holds outputs [F j, F j + F) (16-byte loads of the P and Q rows),
// so every warp instruction serves two tuples.
template <int F>
__global__ void __launch_bounds__(256) pd_sum_half_kernel(PdArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane & 15, grp = lane >> 4;
    const unsigned gmask = 0xffffu << (16 * grp);
    const int64_t groups_total = (int64_t)gridDim.x * (blockDim.x >> 5) * 2;
    const int64_t span = (int64_t)a.range_tiles * 32;
    const bool relu = a.act == RELNN_ACT_RELU;
    const int c0 = gl * F;
    float qb[F];
#pragma unroll
    for (int i = 0; i < F; ++i) qb[i] = (!a.Q && a.bias) ? a.bias[c0 + i] : 0.f;
    for (int64_t rg = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 2 + grp; rg < a.n_ranges;
         rg += groups_total) {
        const int64_t r0 = rg * span, r1 = imin64(a.m, r0 + span);
        const int prev_seg = r0 > 0 ? a.seg[r0 - 1] : -1;
        const int next_seg = r1 < a.m ? a.seg[r1] : -1;
        int cur = -1;
        bool first = true;
        float acc[F], comp[F];
#pragma unroll
        for (int i = 0; i < F; ++i) acc[i] = comp[i] = 0.f;
        auto flush = [&](int s, bool last) {
            const bool split = (first && prev_seg == s) || (last && next_seg == s);
            float* dst = (split ? a.carry + (rg * 2 + (first ? 0 : 1)) * a.d_out : a.out + (int64_t)s * a.d_out) + c0;
            if (split || !a.accumulate) {
#pragma unroll
                for (int i = 0; i < F; i += 4)
                    __stcg(reinterpret_cast<float4*>(dst + i), make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]));
            } else {
#pragma unroll
                for (int i = 0; i < F; ++i) atomicAdd(dst + i, acc[i]);
            }
#pragma unroll
            for (int i = 0; i < F; ++i) acc[i] = comp[i] = 0.f;
            first = false;
        };
        for (int64_t b0 = r0; b0 < r1; b0 += 16) {
            const int nb = (int)imin64(16, r1 - b0);
            const bool tv = gl < nb;
            const int sv = tv ? a.seg[b0 + gl] : -1;
            const int hv = tv ? a.hs[b0 + gl] : 0;
            const int dv = (tv && a.Q) ? a.hd[b0 + gl] : 0;
            for (int j0 = 0; j0 < nb; j0 += 4) {
                float y[4][F];
                int sj[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u < nb ? j0 + u : nb - 1;
                    sj[u] = __shfl_sync(gmask, sv, j, 16);
                    const int64_t ph = (int64_t)__shfl_sync(gmask, hv, j, 16) * a.d_out + c0;
                    const int64_t qh = (int64_t)__shfl_sync(gmask, dv, j, 16) * a.d_out + c0;
#pragma unroll
                    for (int i = 0; i < F; i += 4) {
                        const float4 pv = __ldg(reinterpret_cast<const float4*>(a.P + ph + i));
                        const float4 qv = a.Q ? __ldg(reinterpret_cast<const float4*>(a.Q + qh + i))
                                              : make_float4(qb[i], qb[i + 1], qb[i + 2], qb[i + 3]);
                        y[u][i] = pv.x + qv.x;
                        y[u][i + 1] = pv.y + qv.y;
                        y[u][i + 2] = pv.z + qv.z;
                        y[u][i + 3] = pv.w + qv.w;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (j0 + u >= nb) break;
                    if (sj[u] != cur) {
                        if (cur >= 0) flush(cur, false);
                        cur = sj[u];
                    }
#pragma unroll
                    for (int i = 0; i < F; ++i) {
                        const float v = relu ? fmaxf(y[u][i], 0.f) : y[u][i];
                        if (a.kahan) kahan_add(acc[i], comp[i], v);
                        else acc[i] += v;
                    }
                }
            }
        }
        if (cur >= 0) flush(cur, true);
    }
}

}  // namespace

relnn_status forward_pushdown(Plan& p, const CallIO& io_in, float* out, cudaStream_t st) {
    RELNN_CHECK_ARG(!p.identity, "push-down: the rule needs a Linear");
    RELNN_CHECK_ARG(p.d_out % 32 == 0 && p.d_out <= 128, "push-down: d_out must be a multiple of 32, at most 128");
    for (auto& b : p.br) RELNN_CHECK_ARG(b.d_r == 0, "push-down: rules with a per-tuple embedding are not pushed down");
    // the identity plan of the per-H-row products (built once)
    if (!p.pd) {
        p.pd.reset(new Plan());
        Plan& g = *p.pd;
        g.flags = RELNN_FLAG_BF16 | kPlanDense;
        g.act = RELNN_ACT_NONE;
        g.d = p.d;
        g.d_in = p.d;
        g.d_out = p.d_out;
        g.join_dst = false;
        g.concat_dst = false;
        g.bf16 = true;
        g.n_h = p.n_h;
        g.n_out = p.n_h;
        g.br.resize(1);
        BranchPlan& b = g.br[0];
        b.n_tuples = b.m = p.n_h;
        RELNN_TRY(b.hs.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(p.n_h, 1)));
        RELNN_TRY(b.seg.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(p.n_h, 1)));
        RELNN_TRY(g.status.alloc(sizeof(int) * kStatusInts));
        RELNN_CUDA(cudaMemsetAsync(g.status.p, 0, sizeof(int) * kStatusInts, st));
        const int blocks = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(p.n_h, 1), 256), (int64_t)num_sms() * 8);
        { iota_kernel<<<blocks, 256, 0, st>>>(b.hs.as<int32_t>(), p.n_h); note_launch(); }
        { iota_kernel<<<blocks, 256, 0, st>>>(b.seg.as<int32_t>(), p.n_h); note_launch(); }
        RELNN_CUDA(cudaGetLastError());
    }
    Plan& g = *p.pd;
    CallIO io;  // an f32 H table is rounded to bf16 once for both products
    RELNN_TRY(with_bf16_z(p, io_in, io, st));
    const size_t rows_bytes = sizeof(float) * (size_t)p.n_h * p.d_out;
    RELNN_TRY(p.pdP.alloc(rows_bytes));
    if (p.concat_dst) RELNN_TRY(p.pdQ.alloc(rows_bytes));
    RELNN_TRY(p.pdW.alloc((io.w_bf16 ? 2 : 4) * (size_t)p.d_out * p.d));
    const bool multi = p.br.size() > 1;
    if (multi) RELNN_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * p.n_out * p.d_out, st));
    const bool want_mask = p.act == RELNN_ACT_RELU && (p.flags & RELNN_FLAG_RELU_MASK);
    const int mask_words = ((p.d_out + 127) / 128) * 4;
    const int F = p.d_out / 32;
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        if (b.m == 0) continue;
        // P = Z W_src^T, then Q = Z W_dst^T + b: dense products on the identity plan
        auto product = [&](int col0, const float* bias, float* dst) -> relnn_status {
            { w_cols_kernel<<<64, 256, 0, st>>>(io.br[i].W, io.w_bf16, p.d_out, p.d_in, col0, p.d, p.pdW.p); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
            CallIO gio;
            gio.z = io.z;
            gio.z_bf16 = io.z_bf16;
            gio.w_bf16 = io.w_bf16;
            gio.br.resize(1);
            gio.br[0].W = p.pdW.p;
            gio.br[0].b = bias;
            return forward_tc(g, gio, dst, st);
        };
        RELNN_TRY(product(0, nullptr, p.pdP.as<float>()));
        if (p.concat_dst) RELNN_TRY(product(p.d, io.br[i].b, p.pdQ.as<float>()));
        // per-tuple gathers + activation + SUM walk
        PdArgs a{};
        a.P = p.pdP.as<float>();
        a.Q = p.concat_dst ? p.pdQ.as<float>() : nullptr;
        a.bias = io.br[i].b;
        a.hs = b.hs.as<int32_t>();
        a.hd = b.hd.as<int32_t>();
        a.seg = b.seg.as<int32_t>();
        a.m = b.m;
        a.d_out = p.d_out;
        a.act = p.act;
        a.kahan = p.kahan;
        a.accumulate = multi;
        a.mask_words = mask_words;
        if (want_mask) {
            RELNN_TRY(b.relu_mask.alloc(sizeof(uint32_t) * (size_t)b.m * mask_words));
            a.relu_mask = b.relu_mask.as<uint32_t>();
        }
        a.out = out;
        // one wave of warps, each over an equal range of tuples
        static int bps = 0;
        if (bps <= 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, pd_sum_kernel<4>, 256, 0) != cudaSuccess) {
                (void)cudaGetLastError();
                bps = 1;
            }
            bps = std::max(1, bps);
        }
        // half-warp groups (two ranges per warp, 16-byte row accesses) when no mask is kept, d_out is 64
        // or 128 and out is 16-byte aligned; otherwise one range per warp
        const bool half = !want_mask && (p.d_out == 64 || p.d_out == 128) &&
                          (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
        const int64_t n32 = ceil_div(b.m, 32);
        const int64_t resident = (int64_t)bps * num_sms() * 8 * (half ? 2 : 1);
        a.range_tiles = (int)std::min<int64_t>(ceil_div(n32, resident), 1 << 20);
        a.n_ranges = ceil_div(n32, a.range_tiles);
        RELNN_TRY(p.carry.alloc(sizeof(float) * 2 * p.d_out * (size_t)a.n_ranges));
        a.carry = p.carry.as<float>();
        const int grid = (int)std::min<int64_t>(ceil_div(a.n_ranges, half ? 16 : 8), (int64_t)bps * num_sms());
        {
            ProfToken pt = prof_begin(RELNN_PROF_FWD_FP32, st);
            if (half && p.d_out == 128) pd_sum_half_kernel<8><<<grid, 256, 0, st>>>(a);
            else if (half) pd_sum_half_kernel<4><<<grid, 256, 0, st>>>(a);
            else switch (F) {
                case 1: pd_sum_kernel<1><<<grid, 256, 0, st>>>(a); break;
                case 2: pd_sum_kernel<2><<<grid, 256, 0, st>>>(a); break;
                case 3: pd_sum_kernel<3><<<grid, 256, 0, st>>>(a); break;
                default: pd_sum_kernel<4><<<grid, 256, 0, st>>>(a); break;
            }
            note_launch();
            prof_end(pt, st);
        }
        RELNN_CUDA(cudaGetLastError());
        RELNN_TRY(launch_fixup(a.seg, a.m, a.range_tiles * 32, a.n_ranges, a.carry, out, p.d_out, multi, p.kahan,
                               p.fixjobs, st));
    }
    return RELNN_OK;
}

}  // namespace relnn
