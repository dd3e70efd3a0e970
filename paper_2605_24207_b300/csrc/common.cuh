// Internal helpers shared by the librelnn translation units: status plumbing, device status word,
// bounded waits, key encodings and small device utilities.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "../../include/relnn.h"

namespace relnn {

// ----------------------------------------------------------------------------------- host errors
void set_error(const std::string& msg);
void set_device_error(int32_t code);

// Counts every kernel launch made by the library (relnn_launch_count).
void note_launch();

// Optional CUDA-event timing of the main kernels (relnn_profile_*): a token brackets one launch.
struct ProfToken {
    int id = -1;
    void* ev = nullptr;
};
ProfToken prof_begin(int id, cudaStream_t st);
void prof_end(ProfToken& tok, cudaStream_t st);

#define RELNN_CHECK_ARG(cond, msg)                  \
    do {                                           \
        if (!(cond)) {                             \
            ::relnn::set_error(msg);               \
            return RELNN_EINVAL;                   \
        }                                          \
    } while (0)

#define RELNN_CUDA(call)                                                                      \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            ::relnn::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));           \
            return e_ == cudaErrorMemoryAllocation ? RELNN_ENOMEM : RELNN_ECUDA;              \
        }                                                                                     \
    } while (0)

#define RELNN_TRY(expr)                     \
    do {                                    \
        relnn_status s_ = (expr);           \
        if (s_ != RELNN_OK) return s_;      \
    } while (0)

// Current value of a tuning knob (RELNN_TUNE_*; relnn_tune_set).
int64_t tune_get(int knob);

// Keeps freed blocks of the device's default memory pool cached (no return to the OS at syncs), so
// repeated plan builds reuse memory instead of mapping it again.
void ensure_pool_cached();

// Device buffer drawn from the device's default memory pool.
//   alloc(n, s):     persistent (owned by a handle, usable on any stream once alloc returns; freed
//                    with cudaFree, which synchronises, so only from destroy paths or on growth)
//   alloc_tmp(n, s): temporary, allocated and freed in the order of stream s only
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    bool ordered = false;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), st(o.st), ordered(o.ordered) {
        o.p = nullptr;
        o.bytes = 0;
    }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            st = o.st;
            ordered = o.ordered;
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (ordered) cudaFreeAsync(p, st);
            else cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
    }
    relnn_status alloc(size_t n, cudaStream_t s = nullptr) {
        if (n <= bytes && p) return RELNN_OK;
        release();
        if (n == 0) n = 16;
        ensure_pool_cached();
        cudaError_t e = cudaMallocAsync(&p, n, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            if (p) cudaFree(p);
            p = nullptr;
            set_error(std::string("device allocation of ") + std::to_string(n) + " bytes: " + cudaGetErrorString(e));
            return RELNN_ENOMEM;
        }
        bytes = n;
        ordered = false;
        return RELNN_OK;
    }
    relnn_status alloc_tmp(size_t n, cudaStream_t s) {
        release();
        if (n == 0) n = 16;
        ensure_pool_cached();
        cudaError_t e = cudaMallocAsync(&p, n, s);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error(std::string("device allocation of ") + std::to_string(n) + " bytes: " + cudaGetErrorString(e));
            return RELNN_ENOMEM;
        }
        bytes = n;
        st = s;
        ordered = true;
        return RELNN_OK;
    }
    // Long-lived buffer allocated in the order of stream s without a synchronisation: usable on s
    // at once and on other streams only after s has been synchronised (the plan builders end with
    // one). Freed by cudaFree like alloc().
    relnn_status alloc_nosync(size_t n, cudaStream_t s) {
        if (n <= bytes && p) return RELNN_OK;
        release();
        if (n == 0) n = 16;
        ensure_pool_cached();
        cudaError_t e = cudaMallocAsync(&p, n, s);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error(std::string("device allocation of ") + std::to_string(n) + " bytes: " + cudaGetErrorString(e));
            return RELNN_ENOMEM;
        }
        bytes = n;
        ordered = false;
        return RELNN_OK;
    }
    template <class T>
    T* as() const { return reinterpret_cast<T*>(p); }
};

inline int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

// ----------------------------------------------------------------------------------- device side
// Wall-clock budget for any spin or mbarrier wait inside a kernel (nanoseconds).
constexpr unsigned long long kWaitBudgetNs = 2000000000ull;

// A kernel's device status word is two ints: [0] the status code it raises (RELNN_DEV_*), [1] the
// budget of its bounded waits in microseconds (0: kWaitBudgetNs). Only the wait-timeout test entry
// point sets [1]; every other status word keeps it 0.
constexpr int kStatusInts = 2;
__device__ __forceinline__ unsigned long long wait_budget_ns(const int* status) {
    const int us = status ? *reinterpret_cast<const volatile int*>(status + 1) : 0;
    return us > 0 ? (unsigned long long)us * 1000ull : kWaitBudgetNs;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void raise_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Checked build (compiled with -DRELNN_CHECKED, librelnn_checked.so): gathered row indices and output
// rows are tested on the device; one outside [0, n) raises RELNN_DEV_BOUNDS in the status word and the
// access is skipped (a zero row is read, nothing is written), so a bad plan or input ends as
// RELNN_EDEVICE instead of a fault. In the regular build the test compiles away.
#ifdef RELNN_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, int* status) {
    if (!kChecked) return true;
    if (i >= 0 && i < n) return true;
    raise_status(status, RELNN_DEV_BOUNDS);
    return false;
}

// Order-preserving maps from signed keys to unsigned integers (for radix sorting).
__device__ __forceinline__ uint64_t ordered64(int64_t k) { return (uint64_t)k ^ 0x8000000000000000ull; }
__device__ __forceinline__ uint32_t ordered32(int32_t k) { return (uint32_t)k ^ 0x80000000u; }

// Load key i of a column as int64 (RELNN_I32 columns are sign-extended).
__device__ __forceinline__ int64_t load_key(const void* keys, int kt, int64_t i) {
    return kt == RELNN_I64 ? reinterpret_cast<const int64_t*>(keys)[i]
                           : (int64_t) reinterpret_cast<const int32_t*>(keys)[i];
}

// splitmix64 finalizer (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014) used as the hash of a 64-bit key.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ float bf16_to_f32(uint16_t h) {
    return __uint_as_float(((uint32_t)h) << 16);
}

// Writes one output element. Single-branch rules write every output row exactly once (streaming
// store); unions add every branch into the zeroed output with a reduction (no load on the path).
__device__ __forceinline__ void emit_out(float* dst, float v, int accumulate) {
    if (accumulate) {
        // one add per element per launch and the launches are stream-ordered, so the sum over the
        // branches is taken in branch order (a fire-and-forget reduction: no load on the path)
        atomicAdd(dst, v);
    } else {
        __stcs(dst, v);
    }
}

// Kahan step: sum += v with compensation c (never contracted into FMA).
__device__ __forceinline__ void kahan_add(float& sum, float& c, float v) {
    float y = __fsub_rn(v, c);
    float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

}  // namespace relnn
