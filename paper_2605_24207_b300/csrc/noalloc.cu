// relnn_rule_forward_noalloc: the FP32-form rule forward for callers that must not allocate device
// memory (see include/relnn.h). Its scratch -- the transposed Linear weight and the partial sums of
// output rows cut by tile boundaries -- lives in one file-scope device array instead of a cudaMalloc.
#include <algorithm>
#include <mutex>
#include <string>

#include "common.cuh"

namespace relnn {
namespace {

constexpr int kNaTile = 32;                           // tuples per tile
constexpr size_t kNaScratchFloats = (size_t)1 << 20;  // 4 MiB of f32 scratch per device

// The scratch itself. In host code this name is only a stand-in for the device array: kernels get
// its device address from cudaGetSymbolAddress (see scratch_ptr).
__device__ __align__(256) float g_noalloc_scratch[kNaScratchFloats];

constexpr int kMaxDevices = 64;
float* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on the current device, looked up once per device.
relnn_status scratch_ptr(float** out) {
    int dev = 0;
    RELNN_CUDA(cudaGetDevice(&dev));
    RELNN_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "noalloc forward: device index out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("noalloc forward: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return RELNN_ECUDA;
        }
        g_scratch_addr[dev] = reinterpret_cast<float*>(p);
    }
    *out = g_scratch_addr[dev];
    return RELNN_OK;
}

__global__ void na_transpose_kernel(const float* __restrict__ W, int d_out, int d_in, float* __restrict__ Wt) {
    const int n = d_out * d_in;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = i / d_in, k = i - o * d_in;
        Wt[k * d_out + o] = W[i];
    }
}

// One block per 32-tuple tile; thread o keeps y[t][o] for the tile's tuples and walks them in order,
// writing complete output rows and leaving the two pieces cut by the tile's edges in `carry`.
__global__ void __launch_bounds__(256) na_forward_kernel(const float* __restrict__ z, int d,
                                                         const int32_t* __restrict__ hs,
                                                         const int32_t* __restrict__ hd,
                                                         const int32_t* __restrict__ seg, int64_t m,
                                                         const float* __restrict__ Wt,
                                                         const float* __restrict__ b, int d_out, int relu,
                                                         float* __restrict__ out, float* __restrict__ carry) {
    extern __shared__ float X[];  // [kNaTile][2d]
    __shared__ int seg_s[kNaTile];
    const int d_in = 2 * d;
    const int64_t tile = blockIdx.x;
    const int64_t t0 = tile * kNaTile;
    const int nt = (int)imin64(kNaTile, m - t0);
    const int tid = threadIdx.x;
    if (tid < kNaTile) seg_s[tid] = tid < nt ? seg[t0 + tid] : -1;
    for (int idx = tid; idx < nt * d_in; idx += blockDim.x) {
        const int t = idx / d_in, k = idx - t * d_in;
        X[idx] = k < d ? z[(int64_t)hs[t0 + t] * d + k] : z[(int64_t)hd[t0 + t] * d + (k - d)];
    }
    __syncthreads();
    const int o = tid;
    if (o >= d_out) return;
    float y[kNaTile];
    const float bo = b ? b[o] : 0.f;
#pragma unroll
    for (int t = 0; t < kNaTile; ++t) y[t] = bo;
    for (int k = 0; k < d_in; ++k) {
        const float w = Wt[k * d_out + o];
#pragma unroll
        for (int t = 0; t < kNaTile; ++t) y[t] = fmaf(X[t * d_in + k], w, y[t]);
    }
    const int prev_seg = t0 > 0 ? seg[t0 - 1] : -1;
    const int next_seg = t0 + nt < m ? seg[t0 + nt] : -1;
    float acc = 0.f;
    bool first = true;
#pragma unroll
    for (int t = 0; t < kNaTile; ++t) {
        if (t < nt) {
            acc += relu ? fmaxf(y[t], 0.f) : y[t];
            const int s = seg_s[t];
            const bool last = (t == nt - 1);
            const int sn = last ? next_seg : seg_s[t + 1 < kNaTile ? t + 1 : t];
            if (sn != s || last) {
                if ((first && prev_seg == s) || (last && sn == s))
                    carry[(tile * 2 + (first ? 0 : 1)) * d_out + o] = acc;
                else
                    out[(int64_t)s * d_out + o] = acc;
                acc = 0.f;
                first = false;
            }
        }
    }
}

// Adds the pieces of every output row cut by tile boundaries, in tile order (one block per boundary;
// the block at a row's first boundary does the work).
__global__ void na_fixup_kernel(const int32_t* __restrict__ seg, int64_t m, int64_t n_tiles,
                                const float* __restrict__ carry, float* __restrict__ out, int d_out) {
    for (int64_t bnd = blockIdx.x + 1; bnd < n_tiles; bnd += gridDim.x) {
        const int64_t row = bnd * kNaTile;
        if (row >= m) continue;
        const int s = seg[row];
        if (seg[row - 1] != s) continue;
        if (bnd >= 2 && seg[(bnd - 1) * kNaTile - 1] == s) continue;
        const int first_slot = (seg[(bnd - 1) * kNaTile] == s) ? 0 : 1;
        for (int o = threadIdx.x; o < d_out; o += blockDim.x) {
            float acc = carry[((bnd - 1) * 2 + first_slot) * d_out + o];
            int64_t j = bnd;
            while (true) {
                acc += carry[(j * 2) * d_out + o];
                const int64_t nb = (j + 1) * kNaTile;
                if (j + 1 < n_tiles && nb < m && seg[nb - 1] == s && seg[nb] == s) ++j;
                else break;
            }
            out[(int64_t)s * d_out + o] = acc;
        }
    }
}

}  // namespace
}  // namespace relnn

using namespace relnn;

extern "C" relnn_status relnn_rule_forward_noalloc(const float* d_z, int32_t d, const int32_t* d_hs,
                                                   const int32_t* d_hd, const int32_t* d_seg, int64_t m,
                                                   const float* d_W, const float* d_b, int32_t d_out,
                                                   relnn_act_t act, float* d_out_z, void* stream) {
    RELNN_CHECK_ARG(m >= 0 && m < (1ll << 31) - 1, "noalloc forward: m out of range");
    RELNN_CHECK_ARG(d > 0 && d_out > 0 && d_out <= 256 && 2 * d <= 1024, "noalloc forward: need 0 < d_out <= 256, 2d <= 1024");
    RELNN_CHECK_ARG(act == RELNN_ACT_NONE || act == RELNN_ACT_RELU, "noalloc forward: bad act");
    if (m == 0) return RELNN_OK;
    RELNN_CHECK_ARG(d_z && d_hs && d_hd && d_seg && d_W && d_out_z, "noalloc forward: null pointer");
    const int d_in = 2 * d;
    const int64_t n_tiles = ceil_div(m, kNaTile);
    const size_t need = (size_t)d_in * d_out + (size_t)n_tiles * 2 * d_out;
    if (need > kNaScratchFloats) {
        set_error("noalloc forward: needs " + std::to_string(need * 4) + " bytes of scratch, the fixed array holds " +
                  std::to_string(kNaScratchFloats * 4) + " (split the call or use relnn_rule_forward)");
        return RELNN_ENOSPC;
    }
    // 32 x 2d floats of the gathered Concat rows: up to 128 KB (2d = 1024), above the 48 KB a launch
    // gets without asking, so the kernel's dynamic shared-memory limit is raised (an attribute of
    // the function, not an allocation)
    const size_t smem = sizeof(float) * kNaTile * d_in;
    if (smem > 48 * 1024) {
        static std::once_flag once;
        static cudaError_t attr_err = cudaSuccess;
        std::call_once(once, [] {
            attr_err = cudaFuncSetAttribute(na_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(sizeof(float) * kNaTile * 1024));
        });
        RELNN_CUDA(attr_err);
    }
    float* scratch = nullptr;
    RELNN_TRY(scratch_ptr(&scratch));
    float* Wt = scratch;
    float* carry = scratch + (size_t)d_in * d_out;
    cudaStream_t st = (cudaStream_t)stream;
    { na_transpose_kernel<<<64, 256, 0, st>>>(d_W, d_out, d_in, Wt); note_launch(); }
    const int threads = std::max(32, ((d_out + 31) / 32) * 32);
    { na_forward_kernel<<<(unsigned)n_tiles, threads, smem, st>>>(d_z, d, d_hs, d_hd, d_seg, m, Wt, d_b, d_out,
                                                               act == RELNN_ACT_RELU ? 1 : 0, d_out_z, carry); note_launch(); }
    if (n_tiles > 1) {
        const int blocks = (int)std::min<int64_t>(n_tiles - 1, 4096);
        { na_fixup_kernel<<<blocks, std::min(threads, 256), 0, st>>>(d_seg, m, n_tiles, carry, d_out_z, d_out); note_launch(); }
    }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}
