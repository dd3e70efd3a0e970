// FP32 form of the rule backward on CUDA cores (f32 FMA, no TF32).
//   bw_dy_kernel : per 32-tuple tile, dY[t] = dOut[seg_t] (masked by ReLU'(pre_t), pre recomputed
//                  from the regathered Concat), stored to scratch; dX = dY W scattered into dz / dr
//                  with f32 atomics.
//   bw_dw_kernel : dW = dY^T X as a split-K SIMT GEMM over tuple chunks (X regathered), plus the
//                  db = sum_t dY[t] partials (2048-tuple chunks); bw_reduce_kernel adds the chunk partials in order, compensated.
#include "bwd.cuh"

#include <algorithm>

namespace relnn {

namespace {

constexpr int kTT = 32;

__device__ __forceinline__ float ld_elem(const void* base, int bf16, int64_t idx) {
    return bf16 ? bf16_to_f32(reinterpret_cast<const uint16_t*>(base)[idx])
                : reinterpret_cast<const float*>(base)[idx];
}

struct BwArgs {
    const void* z;
    const void* r;
    const void* W;      // [d_out][d_in] (nullptr = identity)
    const float* bias;
    const float* dout;
    const int32_t *hs, *hd, *er, *seg;
    float* dY;          // [m][d_out] scratch
    float* dz;
    float* dr;
    const uint32_t* mask;  // ReLU mask stored by a BF16-form forward ([m][mask_words]) or nullptr
    int64_t m, n_tiles;
    int z_bf16, r_bf16, w_bf16, d, d_r, d_in, d_out, concat_dst, act, mask_words;
};

// X value k of matched tuple t.
__device__ __forceinline__ float gather_x(const BwArgs& a, int64_t t, int k) {
    if (k < a.d) return ld_elem(a.z, a.z_bf16, (int64_t)a.hs[t] * a.d + k);
    if (a.concat_dst && k < 2 * a.d) return ld_elem(a.z, a.z_bf16, (int64_t)a.hd[t] * a.d + (k - a.d));
    const int kr = k - (a.concat_dst ? 2 : 1) * a.d;
    return ld_elem(a.r, a.r_bf16, (int64_t)a.er[t] * a.d_r + kr);
}

__global__ void bw_dy_kernel(BwArgs a) {
    extern __shared__ float sm[];
    float* X = sm;                       // [kTT][d_in]
    float* Yg = sm + kTT * a.d_in;       // [kTT][d_out]
    const int tid = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const int64_t t0 = tile * kTT;
        const int nt = (int)imin64(kTT, a.m - t0);
        __syncthreads();
        if (a.act == RELNN_ACT_RELU && a.W) {
            for (int idx = tid; idx < nt * a.d_in; idx += blockDim.x) {
                const int t = idx / a.d_in, k = idx - t * a.d_in;
                X[idx] = gather_x(a, t0 + t, k);
            }
        }
        for (int idx = tid; idx < nt * a.d_out; idx += blockDim.x) {
            const int t = idx / a.d_out, o = idx - t * a.d_out;
            Yg[idx] = a.dout[(int64_t)a.seg[t0 + t] * a.d_out + o];
        }
        __syncthreads();
        if (a.mask) {
            // the ReLU mask the forward used (keeps a BF16-form forward and this backward
            // consistent), or the MAX aggregator's winner mask
            for (int idx = tid; idx < nt * a.d_out; idx += blockDim.x) {
                const int t = idx / a.d_out, o = idx - t * a.d_out;
                if (!((a.mask[(t0 + t) * a.mask_words + (o >> 5)] >> (o & 31)) & 1u)) Yg[idx] = 0.f;
            }
            __syncthreads();
        } else if (a.act == RELNN_ACT_RELU && a.W) {
            for (int idx = tid; idx < nt * a.d_out; idx += blockDim.x) {
                const int t = idx / a.d_out, o = idx - t * a.d_out;
                float pre = a.bias ? a.bias[o] : 0.f;
                for (int k = 0; k < a.d_in; ++k)
                    pre = fmaf(ld_elem(a.W, a.w_bf16, (int64_t)o * a.d_in + k), X[t * a.d_in + k], pre);
                if (!(pre > 0.f)) Yg[idx] = 0.f;
            }
            __syncthreads();
        } else if (a.act == RELNN_ACT_RELU) {
            // identity + ReLU: pre = x itself
            for (int idx = tid; idx < nt * a.d_out; idx += blockDim.x) {
                const int t = idx / a.d_out, o = idx - t * a.d_out;
                if (!(gather_x(a, t0 + t, o) > 0.f)) Yg[idx] = 0.f;
            }
            __syncthreads();
        }
        for (int idx = tid; idx < nt * a.d_out; idx += blockDim.x) a.dY[t0 * a.d_out + idx] = Yg[idx];
        // dX[t][k] = sum_o dY[t][o] W[o][k]; scatter by the Concat slice k falls in
        for (int idx = tid; idx < nt * a.d_in; idx += blockDim.x) {
            const int t = idx / a.d_in, k = idx - t * a.d_in;
            float v;
            if (a.W) {
                v = 0.f;
                for (int o = 0; o < a.d_out; ++o) v = fmaf(Yg[t * a.d_out + o], ld_elem(a.W, a.w_bf16, (int64_t)o * a.d_in + k), v);
            } else {
                v = Yg[t * a.d_out + k];
            }
            const int64_t tt = t0 + t;
            if (k < a.d) {
                if (a.dz) atomicAdd(&a.dz[(int64_t)a.hs[tt] * a.d + k], v);
            } else if (a.concat_dst && k < 2 * a.d) {
                if (a.dz) atomicAdd(&a.dz[(int64_t)a.hd[tt] * a.d + (k - a.d)], v);
            } else if (a.dr) {
                const int kr = k - (a.concat_dst ? 2 : 1) * a.d;
                atomicAdd(&a.dr[(int64_t)a.er[tt] * a.d_r + kr], v);
            }
        }
    }
}

// Identity rule without ReLU (e.g. a SUM readout): dX[t] = dOut[seg_t], added straight into the
// slice's gradient, 4 features per thread (16-byte loads and 16-byte atomic adds).
__global__ void bw_identity_kernel(BwArgs a) {
    const int q = a.d_in / 4;
    const int64_t n = a.m * q;
    // a row of q 4-feature chunks: the tuple by a shift when q is a power of two (no 64-bit division)
    const int lq = (q & (q - 1)) == 0 ? __ffs(q) - 1 : -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = lq >= 0 ? i >> lq : i / q;
        const int k = (int)(i - t * q) * 4;
        const float4 v = *reinterpret_cast<const float4*>(a.dout + (int64_t)a.seg[t] * a.d_out + k);
        if (k < a.d) {
            if (a.dz) atomicAdd(reinterpret_cast<float4*>(a.dz + (int64_t)a.hs[t] * a.d + k), v);
        } else if (a.concat_dst && k < 2 * a.d) {
            if (a.dz) atomicAdd(reinterpret_cast<float4*>(a.dz + (int64_t)a.hd[t] * a.d + (k - a.d)), v);
        } else if (a.dr) {
            const int kr = k - (a.concat_dst ? 2 : 1) * a.d;
            atomicAdd(reinterpret_cast<float4*>(a.dr + (int64_t)a.er[t] * a.d_r + kr), v);
        }
    }
}

// Split-K SIMT GEMM: block (ob, kb, chunk) computes a 32x32 tile of dW over one tuple chunk.
constexpr int kDwTile = 32;
constexpr int kDwChunk = 2048;  // short f32 chains per partial; partials added compensated

__global__ void bw_dw_kernel(BwArgs a, float* part, float* dbpart) {
    __shared__ float Ys[16][kDwTile + 1];
    __shared__ float Xs[16][kDwTile + 1];
    const int ob = blockIdx.x, kb = blockIdx.y;
    const int64_t c0 = (int64_t)blockIdx.z * kDwChunk;
    const int64_t c1 = imin64(c0 + kDwChunk, a.m);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float dbacc = 0.f;
    for (int64_t t = c0; t < c1; t += 16) {
        for (int i = threadIdx.x; i < 16 * kDwTile; i += blockDim.x) {
            const int tt = i / kDwTile, j = i - tt * kDwTile;
            const int64_t row = t + tt;
            const int o = ob * kDwTile + j, k = kb * kDwTile + j;
            Ys[tt][j] = (row < c1 && o < a.d_out) ? a.dY[row * a.d_out + o] : 0.f;
            Xs[tt][j] = (row < c1 && k < a.d_in) ? gather_x(a, row, k) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) {
            const float x = Xs[tt][tx];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(Ys[tt][ty * 4 + u], x, acc[u]);
            if (kb == 0 && ty == 0) dbacc += Ys[tt][tx];
        }
        __syncthreads();
    }
    const int k = kb * kDwTile + tx;
    for (int u = 0; u < 4; ++u) {
        const int o = ob * kDwTile + ty * 4 + u;
        if (o < a.d_out && k < a.d_in) part[((int64_t)blockIdx.z * a.d_out + o) * a.d_in + k] = acc[u];
    }
    if (kb == 0 && ty == 0) {
        const int o = ob * kDwTile + tx;
        if (o < a.d_out) dbpart[(int64_t)blockIdx.z * a.d_out + o] = dbacc;
    }
}

__global__ void bw_reduce_kernel(const float* part, int nchunks, int64_t n, float* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f, c = 0.f;
        for (int k = 0; k < nchunks; ++k) kahan_add(s, c, part[(int64_t)k * n + i]);
        out[i] = s;
    }
}

}  // namespace

relnn_status backward_fp32(Plan& p, const CallIO& io, const GradIO& g, cudaStream_t st) {
    RELNN_CHECK_ARG(g.dout, "backward: null output gradient");
    RELNN_CHECK_ARG(p.d_in <= 1024 && p.d_out <= 1024, "backward: widths too large");
    if (g.dz && !g.accumulate_dz) RELNN_CUDA(cudaMemsetAsync(g.dz, 0, sizeof(float) * p.n_h * p.d, st));
    for (size_t i = 0; i < p.br.size(); ++i) {
        BranchPlan& b = p.br[i];
        const bool need_w = !p.identity && (g.dW.size() > i && (g.dW[i] || g.db[i]));
        if (g.dr.size() > i && g.dr[i] && b.d_r > 0)
            RELNN_CUDA(cudaMemsetAsync(g.dr[i], 0, sizeof(float) * b.n_tuples * b.d_r, st));
        if (b.m == 0) {
            if (need_w && g.dW[i]) RELNN_CUDA(cudaMemsetAsync(g.dW[i], 0, sizeof(float) * p.d_out * p.d_in, st));
            if (need_w && g.db[i]) RELNN_CUDA(cudaMemsetAsync(g.db[i], 0, sizeof(float) * p.d_out, st));
            continue;
        }
        const int64_t nchunks = ceil_div(b.m, kDwChunk);
        const size_t dy_bytes = sizeof(float) * (size_t)b.m * p.d_out;
        const size_t part_bytes = need_w ? sizeof(float) * (size_t)nchunks * p.d_out * (p.d_in + 1) : 0;
        BwArgs a{};
        a.z = io.z;
        a.r = io.br[i].r;
        a.W = p.identity ? nullptr : io.br[i].W;
        a.bias = io.br[i].b;
        a.dout = g.dout;
        a.hs = b.hs.as<int32_t>();
        a.hd = b.hd.as<int32_t>();
        a.er = b.er.as<int32_t>();
        a.seg = b.seg.as<int32_t>();
        a.dz = g.dz;
        a.dr = (g.dr.size() > i && b.d_r > 0) ? g.dr[i] : nullptr;
        a.m = b.m;
        a.n_tiles = ceil_div(b.m, kTT);
        a.z_bf16 = io.z_bf16;
        a.r_bf16 = io.r_bf16;
        a.w_bf16 = io.w_bf16;
        a.d = p.d;
        a.d_r = b.d_r;
        a.d_in = p.d_in;
        a.d_out = p.d_out;
        a.concat_dst = p.concat_dst;
        a.act = p.act;
        const bool maxagg = (p.flags & RELNN_FLAG_MAX) != 0;
        a.mask = maxagg ? p.win_mask.as<uint32_t>()
                        : ((p.act == RELNN_ACT_RELU && b.relu_mask.p) ? b.relu_mask.as<uint32_t>() : nullptr);
        a.mask_words = ((p.d_out + 127) / 128) * 4;
        // identity without ReLU: a straight gather of dOut rows into the gradients
        const bool aligned16 = ((reinterpret_cast<uintptr_t>(g.dout) | reinterpret_cast<uintptr_t>(g.dz) |
                                 reinterpret_cast<uintptr_t>(a.dr)) & 15u) == 0;
        if (p.identity && p.act != RELNN_ACT_RELU && !maxagg && p.d % 4 == 0 && b.d_r % 4 == 0 && aligned16) {
            const int blocks = (int)std::min<int64_t>(ceil_div(b.m * (p.d_in / 4), 256), (int64_t)num_sms() * 16);
            { ProfToken pt = prof_begin(RELNN_PROF_BWD_FP32, st); bw_identity_kernel<<<blocks, 256, 0, st>>>(a); note_launch(); prof_end(pt, st); }
            RELNN_CUDA(cudaGetLastError());
            continue;
        }
        RELNN_TRY(p.scratch.alloc(dy_bytes + part_bytes + 256));
        a.dY = p.scratch.as<float>();
        const int threads = std::min(1024, std::max(32, ((std::max(p.d_in, p.d_out) + 31) / 32) * 32));
        const size_t smem = sizeof(float) * kTT * (p.d_in + p.d_out);
        RELNN_CHECK_ARG(smem <= 200 * 1024, "backward: tile too large");
        RELNN_CUDA(cudaFuncSetAttribute(bw_dy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int grid = (int)std::min<int64_t>(a.n_tiles, (int64_t)num_sms() * 4);
        { ProfToken pt = prof_begin(RELNN_PROF_BWD_FP32, st); bw_dy_kernel<<<grid, threads, smem, st>>>(a); note_launch(); prof_end(pt, st); }
        RELNN_CUDA(cudaGetLastError());
        if (need_w) {
            float* part = reinterpret_cast<float*>(p.scratch.as<uint8_t>() + dy_bytes);
            float* dbpart = part + (size_t)nchunks * p.d_out * p.d_in;
            dim3 grid3((unsigned)ceil_div(p.d_out, kDwTile), (unsigned)ceil_div(p.d_in, kDwTile), (unsigned)nchunks);
            { ProfToken pt = prof_begin(RELNN_PROF_BWD_FP32, st); bw_dw_kernel<<<grid3, 256, 0, st>>>(a, part, dbpart); note_launch(); prof_end(pt, st); }
            RELNN_CUDA(cudaGetLastError());
            const int64_t nw = (int64_t)p.d_out * p.d_in;
            if (g.dW[i]) { bw_reduce_kernel<<<(int)std::min<int64_t>(ceil_div(nw, 256), 1024), 256, 0, st>>>(part, (int)nchunks, nw, g.dW[i]); note_launch(); }
            if (g.db[i]) { bw_reduce_kernel<<<1, 256, 0, st>>>(dbpart, (int)nchunks, p.d_out, g.db[i]); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
        }
    }
    return RELNN_OK;
}

}  // namespace relnn
