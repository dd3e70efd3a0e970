// Loss relation of arity 0 (paper Sec. 3.2): L(; mean((z_p - z_t)^2)) :- Pred(g; z_p), Target(g; z_t).
// The join on g pairs every prediction row with the target rows of the same key (both key columns
// sorted ascending, keys unique within each); the mean runs over every cell of the joined pairs.
#include <algorithm>

#include "common.cuh"

namespace relnn {
namespace {

// Index of `key` in the ascending array keys[0..n), or -1.
__device__ __forceinline__ int64_t find_key(const void* keys, int kt, int64_t n, int64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (load_key(keys, kt, mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && load_key(keys, kt, lo) == key) ? lo : -1;
}

// One block. Pass 1 counts joined rows; pass 2 accumulates the squared error and writes the gradient
// d mean / d pred = 2 (p - t) / (rows * width) (zero for prediction rows that join nothing).
__global__ void mse_kernel(const float* pred, const void* pkeys, int64_t n_pred, const float* target, const void* tkeys,
                           int64_t n_target, int width, int kt, float* loss, float* grad) {
    __shared__ double red[32];
    __shared__ unsigned long long cnt_s;
    if (threadIdx.x == 0) cnt_s = 0;
    __syncthreads();
    unsigned long long c = 0;
    for (int64_t i = threadIdx.x; i < n_pred; i += blockDim.x)
        c += find_key(tkeys, kt, n_target, load_key(pkeys, kt, i)) >= 0 ? 1 : 0;
    atomicAdd(&cnt_s, c);
    __syncthreads();
    const double n_cells = (double)cnt_s * width;
    double s = 0.0;
    for (int64_t i = 0; i < n_pred; ++i) {
        const int64_t j = find_key(tkeys, kt, n_target, load_key(pkeys, kt, i));
        for (int k = threadIdx.x; k < width; k += blockDim.x) {
            const float p = pred[i * width + k];
            float g = 0.f;
            if (j >= 0) {
                const double e = (double)p - (double)target[j * width + k];
                s += e * e;
                g = (float)(2.0 * e / n_cells);
            }
            if (grad) grad[i * width + k] = g;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *loss = n_cells > 0 ? (float)(t / n_cells) : 0.f;
    }
}

}  // namespace
}  // namespace relnn

using namespace relnn;

extern "C" relnn_status relnn_mse_loss(const float* d_pred, const void* d_pred_keys, int64_t n_pred, const float* d_target,
                                       const void* d_target_keys, int64_t n_target, int32_t width, relnn_key_t kt,
                                       float* d_loss, float* d_grad, void* stream) {
    RELNN_CHECK_ARG(n_pred >= 0 && n_target >= 0 && width > 0, "mse: bad sizes");
    RELNN_CHECK_ARG(d_loss, "mse: null loss");
    RELNN_CHECK_ARG(kt == RELNN_I32 || kt == RELNN_I64, "mse: bad key type");
    RELNN_CHECK_ARG((n_pred == 0 || (d_pred && d_pred_keys)) && (n_target == 0 || (d_target && d_target_keys)),
                    "mse: null input");
    cudaStream_t st = (cudaStream_t)stream;
    { mse_kernel<<<1, 256, 0, st>>>(d_pred, d_pred_keys, n_pred, d_target, d_target_keys, n_target, width, kt, d_loss,
                                    d_grad); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}
