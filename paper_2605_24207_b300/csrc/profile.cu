// Launch counter and optional per-kernel CUDA-event timing (relnn_launch_count, relnn_profile_*).
// Events are recorded on the stream the kernel is launched on, so the elapsed time is that of the
// launch as the device ran it inside the caller's stream order.
#include <atomic>
#include <string>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace relnn {

namespace {

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_mu;

struct EvPair {
    cudaEvent_t a = nullptr, b = nullptr;
    int id = -1;
};
std::vector<EvPair*> g_free, g_pending;
constexpr int kIds = 16;
double g_total_ms[kIds];
int64_t g_count[kIds];

EvPair* take() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_free.empty()) {
        EvPair* e = g_free.back();
        g_free.pop_back();
        return e;
    }
    EvPair* e = new EvPair();
    if (cudaEventCreate(&e->a) != cudaSuccess || cudaEventCreate(&e->b) != cudaSuccess) {
        delete e;
        return nullptr;
    }
    return e;
}

}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
constexpr int kKnobs = 7;
std::atomic<int64_t> g_knobs[kKnobs] = {{8}, {0}, {0}, {0}, {33}, {0}, {0}};
bool knob_ok(int knob, int64_t v) {
    switch (knob) {
        case RELNN_TUNE_SORT_BITS: return v >= 4 && v <= 11;
        case RELNN_TUNE_AGG_ROWS: return v == 0 || v == 32 || v == 64 || v == 128;
        case RELNN_TUNE_AGG_STAGES: return v == 0 || (v >= 2 && v <= 4);
        case RELNN_TUNE_AGG_EPI: return v == 0 || v == 4 || v == 8;
        case RELNN_TUNE_KAHAN_MIN: return v >= 0 && v <= (1 << 30);
        case RELNN_TUNE_GROUP_SORT: return v == 0 || v == 1;
        case RELNN_TUNE_AGG_FUSE: return v >= 0 && v <= 2;
    }
    return false;
}
}  // namespace

int64_t tune_get(int knob) { return knob >= 0 && knob < kKnobs ? g_knobs[knob].load() : 0; }

void ensure_pool_cached() {
    static std::atomic<uint64_t> done_mask{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    const uint64_t bit = 1ull << dev;
    if (done_mask.load() & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done_mask.fetch_or(bit);
}

ProfToken prof_begin(int id, cudaStream_t st) {
    ProfToken t;
    if (!g_prof_on.load(std::memory_order_relaxed) || id < 0 || id >= kIds) return t;
    EvPair* e = take();
    if (!e) return t;
    e->id = id;
    cudaEventRecord(e->a, st);
    t.id = id;
    t.ev = e;
    return t;
}

void prof_end(ProfToken& tok, cudaStream_t st) {
    if (!tok.ev) return;
    EvPair* e = reinterpret_cast<EvPair*>(tok.ev);
    cudaEventRecord(e->b, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back(e);
    tok.ev = nullptr;
}

// FP32 FMA throughput probe: every thread runs kFmaChains independent chains x <- x * a + b (a and b
// are run-time values, so nothing folds), enough independent work per warp to issue an FMA every
// cycle; the sum of the chains is stored only if it equals a value it cannot take, which keeps the
// chains live without a store per thread.
constexpr int kFmaChains = 8;
__global__ void __launch_bounds__(1024) fma_peak_kernel(float* out, int iters, float a, float b) {
    float x[kFmaChains];
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) x[i] = (float)threadIdx.x * 1e-3f + (float)i;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kFmaChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) s += x[i];
    if (s == -1.2345e30f) out[blockIdx.x] = s;
}

// One CTA waits, with the library's bounded mbarrier wait, on a barrier nothing arrives at; the wait
// gives up after the budget in the status word, raises RELNN_DEV_TIMEOUT and the kernel returns.
__global__ void wait_timeout_kernel(int* status) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_u32(&bar), 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    __syncthreads();
    tc::mbar_wait(tc::smem_u32(&bar), 0, status, &abort_flag);  // phase 0 never completes
}

}  // namespace relnn

using namespace relnn;

extern "C" {

relnn_status relnn_test_wait_timeout(int32_t budget_us, void* stream) {
    RELNN_CHECK_ARG(budget_us > 0 && budget_us <= 1000000, "wait timeout test: budget must be in (0, 1 s]");
    cudaStream_t st = (cudaStream_t)stream;
    int* d = nullptr;
    RELNN_CUDA(cudaMallocAsync(&d, sizeof(int) * kStatusInts, st));
    const int h[kStatusInts] = {0, budget_us};
    int code = 0;
    cudaError_t e = cudaMemcpyAsync(d, h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        wait_timeout_kernel<<<1, 32, 0, st>>>(d);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&code, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d, st);
    RELNN_CUDA(e);
    if (code != 0) {
        set_device_error(code);
        set_error("wait timeout test: the bounded wait gave up (device code " + std::to_string(code) + ")");
        return RELNN_EDEVICE;
    }
    return RELNN_OK;
}

relnn_status relnn_tune_set(int32_t knob, int64_t value) {
    RELNN_CHECK_ARG(knob_ok(knob, value), "tune: unknown knob or value out of range");
    g_knobs[knob].store(value);
    return RELNN_OK;
}

relnn_status relnn_tune_get(int32_t knob, int64_t* value) {
    RELNN_CHECK_ARG(knob >= 0 && knob < kKnobs && value, "tune: unknown knob");
    *value = g_knobs[knob].load();
    return RELNN_OK;
}

relnn_status relnn_peak_fma_f32(int32_t iters, double* tflops, double* ms, void* stream) {
    RELNN_CHECK_ARG(iters > 0 && tflops, "peak fma: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = 2 * num_sms(), threads = 1024;
    float* sink = nullptr;
    RELNN_CUDA(cudaMallocAsync(&sink, sizeof(float) * blocks, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RELNN_CUDA(cudaEventCreate(&e0));
    RELNN_CUDA(cudaEventCreate(&e1));
    // a = 1 - 2^-20 and b = 2^-10 keep the chains bounded (x converges to b / (1 - a) = 1024)
    const float a = 1.0f - 9.5367431640625e-07f, b = 9.765625e-04f;
    { fma_peak_kernel<<<blocks, threads, 0, st>>>(sink, iters, a, b); note_launch(); }
    cudaEventRecord(e0, st);
    { fma_peak_kernel<<<blocks, threads, 0, st>>>(sink, iters, a, b); note_launch(); }
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    RELNN_CUDA(err);
    const double flop = 2.0 * kFmaChains * (double)iters * blocks * threads;
    *tflops = flop / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return RELNN_OK;
}

uint64_t relnn_launch_count(void) { return g_launches.load(); }

relnn_status relnn_profile_enable(int32_t on) {
    g_prof_on.store(on ? 1 : 0);
    return RELNN_OK;
}

relnn_status relnn_profile_read(int32_t id, double* total_ms, int64_t* launches) {
    RELNN_CHECK_ARG(id >= 0 && id < kIds, "profile: bad id");
    std::vector<EvPair*> done;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        done.swap(g_pending);
    }
    for (EvPair* e : done) {
        cudaEventSynchronize(e->b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e->a, e->b) == cudaSuccess) {
            g_total_ms[e->id] += ms;
            g_count[e->id] += 1;
        }
        std::lock_guard<std::mutex> lk(g_mu);
        g_free.push_back(e);
    }
    if (total_ms) *total_ms = g_total_ms[id];
    if (launches) *launches = g_count[id];
    return RELNN_OK;
}

relnn_status relnn_profile_reset(void) {
    relnn_profile_read(0, nullptr, nullptr);
    for (int i = 0; i < kIds; ++i) {
        g_total_ms[i] = 0.0;
        g_count[i] = 0;
    }
    return RELNN_OK;
}

}  // extern "C"
