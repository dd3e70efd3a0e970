// MEAN aggregator of the projected union (paper Sec. 2.2: alpha over the multiset B_t of the
// contributing tuples; MEAN is named beside SUM in Sec. 4.2 and Sec. 5). For a single-branch rule,
//   Out[k] = (1 / n_k) * SUM_{t -> k} Y_t,   n_k = number of matched tuples of output row k,
// so the forward is the SUM forward followed by a per-row scale, and the backward is the SUM
// backward of dOut[k] / n_k. The counts are integers taken from the plan once (exact).
#include "mean.cuh"

#include <algorithm>

namespace relnn {

namespace {

__global__ void count_rows_kernel(const int32_t* __restrict__ seg, int64_t m, int32_t* __restrict__ cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + seg[i], 1);
}

__global__ void inv_count_kernel(const int32_t* __restrict__ cnt, int64_t n, float* __restrict__ inv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        inv[i] = cnt[i] > 0 ? 1.f / (float)cnt[i] : 0.f;
}

// dst[k][o] = src[k][o] * inv[k] (dst may equal src)
__global__ void scale_rows_kernel(const float* src, const float* __restrict__ inv, int64_t n, int d, float* dst) {
    const int64_t total = n * d;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] * inv[i / d];
}

int grid_for(int64_t n) { return (int)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), 256), (int64_t)num_sms() * 8); }

}  // namespace

relnn_status ensure_inv_count(Plan& p, cudaStream_t st) {
    RELNN_CHECK_ARG(p.br.size() == 1, "MEAN aggregator: single-branch rules only");
    if (p.inv_cnt.p || p.n_out == 0) return RELNN_OK;
    BranchPlan& b = p.br[0];
    DevBuf cnt;
    RELNN_TRY(cnt.alloc_tmp(sizeof(int32_t) * (size_t)p.n_out, st));
    RELNN_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (size_t)p.n_out, st));
    if (b.m > 0) {
        count_rows_kernel<<<grid_for(b.m), 256, 0, st>>>(b.seg.as<int32_t>(), b.m, cnt.as<int32_t>());
        note_launch();
    }
    RELNN_TRY(p.inv_cnt.alloc(sizeof(float) * (size_t)p.n_out));
    { inv_count_kernel<<<grid_for(p.n_out), 256, 0, st>>>(cnt.as<int32_t>(), p.n_out, p.inv_cnt.as<float>()); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

relnn_status count_rows_into(const int32_t* seg, int64_t m, int32_t* cnt, cudaStream_t st) {
    if (m == 0) return RELNN_OK;
    { count_rows_kernel<<<grid_for(m), 256, 0, st>>>(seg, m, cnt); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

relnn_status scale_rows(const float* src, const float* inv, int64_t n, int d, float* dst, cudaStream_t st) {
    if (n == 0) return RELNN_OK;
    { scale_rows_kernel<<<grid_for(n * d), 256, 0, st>>>(src, inv, n, d, dst); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    return RELNN_OK;
}

}  // namespace relnn
