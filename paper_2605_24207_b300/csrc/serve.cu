// Serving engine (relnn_server_*): memory-admitted continuous batching of independent rule queries
// that share one Linear.
//
// Host side: submit() queues a query after checking that its device-memory estimate can ever fit the
// budget; n_workers host threads each own a non-blocking CUDA stream and repeatedly take, in arrival
// order, as many queued queries as fit (E tuples, query count, free budget), evaluate them as ONE
// batch and publish per-query results. Queries that arrive while batches run are picked up by the
// next free worker, so batches overlap on the device.
//
// A batch is one rule over disjoint key ranges: key k of the i-th query of the batch becomes
// (i << kb) + (k - kmin_i) (int64, order-preserving; kmin_i the query's least H key, kb the width of
// the widest query's H key span, so dense queries make a dense batch), the queries' H.z rows are
// concatenated, and the usual content track (relnn plan) and fused persistent forward run once over
// all of it. The output keys come out sorted by (query, key); a binary search per query cuts them
// back into per-query results (keys restored to int32).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fwd.cuh"
#include "primitives.cuh"

namespace relnn {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kPollUs = 2000;  // how long an idle worker polls the queue before it sleeps

// Key k of the i-th query of a batch becomes (i << kb) + (k - kmin_i), kmin_i the least H key of
// the query and kb the width of the widest query's H key span, so that the batch's key space stays as
// dense as its queries' (the join build then addresses it directly). An E key outside its query's H
// span matches nothing: it becomes -1, below every batch key.
__global__ void batch_keys_kernel(const int32_t* __restrict__ in, int64_t n, int64_t prefix, int32_t kmin,
                                  int32_t kmax, int64_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = in[i];
        out[i] = (k < kmin || k > kmax) ? -1 : prefix + ((int64_t)k - kmin);
    }
}

__global__ void strip_keys_kernel(const int64_t* __restrict__ in, int64_t n, int64_t mask, int32_t kmin,
                                  int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)((in[i] & mask) + kmin);
}

// Least and largest H key of every query of a batch (blockIdx.y = query): mm[2 i] / mm[2 i + 1] hold
// them order-preserved as unsigned (k + 2^31), reduced by warp then atomics.
struct QKeys {
    const int32_t* k;
    int64_t n;
};
__global__ void query_minmax_kernel(const QKeys* __restrict__ qs, unsigned* __restrict__ mm) {
    const QKeys q = qs[blockIdx.y];
    unsigned lo = 0xffffffffu, hi = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q.n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned u = (unsigned)q.k[i] ^ 0x80000000u;
        lo = min(lo, u);
        hi = max(hi, u);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mm + 2 * blockIdx.y, lo);
        atomicMax(mm + 2 * blockIdx.y + 1, hi);
    }
}

// lo[q] = first output row of query q (keys are sorted by query prefix); lo[nq] = n.
__global__ void ranges_kernel(const int64_t* __restrict__ keys, int64_t n, int nq, int kb, int64_t* __restrict__ lo) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > nq) return;
    const int64_t target = (int64_t)q << kb;
    int64_t a = 0, b = n;
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (keys[mid] < target) a = mid + 1;
        else b = mid;
    }
    lo[q] = (q == nq) ? n : a;
}

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 148 * 8)); }

struct Query {
    uint64_t ticket = 0;
    relnn_query q{};
    int64_t mem = 0;
    Clock::time_point t_submit;
    int state = 0;  // 0 queued, 1 running, 2 done
    relnn_status st = RELNN_OK;
    DevBuf keys, z;
    int64_t n_out = 0;
    double latency_us = 0;
    int batch_q = 0;
};

}  // namespace
}  // namespace relnn

using namespace relnn;

struct relnn_server_s {
    relnn_server_cfg cfg{};
    int dev = 0;
    size_t z_esz = 4;
    int64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Query*> queue;
    std::unordered_map<uint64_t, Query*> all;
    uint64_t next_ticket = 1;
    int64_t mem_in_use = 0;
    int in_system = 0;
    bool stopping = false;
    // the device's free memory as last read (cudaMemGetInfo), and when; re-read when older than
    // 2 ms or when a batch would take more than half of it
    int64_t free_seen = 0;
    std::chrono::steady_clock::time_point free_when{};
    // queued queries and the stop request, read without the lock by idle workers polling for work
    std::atomic<int> n_queued{0};
    std::atomic<bool> stopping_flag{false};
    std::vector<std::thread> workers;
};

namespace relnn {
namespace {

// Device bytes a query may need while its batch runs (keys, sort temporaries, plan, outputs).
int64_t query_mem(const relnn_server_s* S, const relnn_query& q) {
    const int64_t T = q.n_tuples, K = q.n_h;
    return T * 112 + K * (96 + (int64_t)S->cfg.d * (int64_t)S->z_esz) + K * (int64_t)S->cfg.d_out * 8 + (1 << 20);
}

relnn_status run_batch(relnn_server_s* S, std::vector<Query*>& batch, cudaStream_t st) {
    const int nq = (int)batch.size();
    const int d = S->cfg.d, d_out = S->cfg.d_out;
    int64_t K = 0, T = 0;
    std::vector<int64_t> h_off(nq), t_off(nq);
    for (int i = 0; i < nq; ++i) {
        h_off[i] = K;
        t_off[i] = T;
        K += batch[i]->q.n_h;
        T += batch[i]->q.n_tuples;
    }
    DevBuf hk, zb, sk, dk, lo;
    RELNN_TRY(hk.alloc_tmp(sizeof(int64_t) * std::max<int64_t>(K, 1), st));
    RELNN_TRY(zb.alloc_tmp(S->z_esz * d * std::max<int64_t>(K, 1), st));
    RELNN_TRY(sk.alloc_tmp(sizeof(int64_t) * std::max<int64_t>(T, 1), st));
    RELNN_TRY(dk.alloc_tmp(sizeof(int64_t) * std::max<int64_t>(T, 1), st));
    RELNN_TRY(lo.alloc_tmp(sizeof(int64_t) * (nq + 1), st));
    // every query's H key range (one launch, one synchronisation), then the batch key width
    std::vector<QKeys> qk(nq);
    for (int i = 0; i < nq; ++i) qk[i] = QKeys{(const int32_t*)batch[i]->q.d_h_ids, batch[i]->q.n_h};
    DevBuf qd, mmb;
    RELNN_TRY(qd.alloc_tmp(sizeof(QKeys) * nq, st));
    RELNN_TRY(mmb.alloc_tmp(sizeof(unsigned) * 2 * nq, st));
    std::vector<unsigned> mm(2 * nq);
    for (int i = 0; i < nq; ++i) {
        mm[2 * i] = 0xffffffffu;
        mm[2 * i + 1] = 0u;
    }
    RELNN_CUDA(cudaMemcpyAsync(qd.p, qk.data(), sizeof(QKeys) * nq, cudaMemcpyHostToDevice, st));
    RELNN_CUDA(cudaMemcpyAsync(mmb.p, mm.data(), sizeof(unsigned) * 2 * nq, cudaMemcpyHostToDevice, st));
    int64_t kmax_n = 1;
    for (int i = 0; i < nq; ++i) kmax_n = std::max<int64_t>(kmax_n, batch[i]->q.n_h);
    { query_minmax_kernel<<<dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(kmax_n, 256 * 8), 64)), (unsigned)nq),
                            256, 0, st>>>(qd.as<QKeys>(), mmb.as<unsigned>()); note_launch(); }
    RELNN_CUDA(cudaMemcpyAsync(mm.data(), mmb.p, sizeof(unsigned) * 2 * nq, cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> qmin(nq), qmax(nq);
    int kb = 1;
    for (int i = 0; i < nq; ++i) {
        if (batch[i]->q.n_h == 0) {
            qmin[i] = 1;
            qmax[i] = 0;  // an empty H: every E key is out of range
            continue;
        }
        qmin[i] = (int32_t)(mm[2 * i] ^ 0x80000000u);
        qmax[i] = (int32_t)(mm[2 * i + 1] ^ 0x80000000u);
        const uint64_t span = (uint64_t)((int64_t)qmax[i] - qmin[i]);
        kb = std::max(kb, bit_length(span));
    }
    for (int i = 0; i < nq; ++i) {
        const relnn_query& q = batch[i]->q;
        const int64_t prefix = (int64_t)i << kb;
        if (q.n_h > 0) {
            { batch_keys_kernel<<<grid_for(q.n_h), 256, 0, st>>>((const int32_t*)q.d_h_ids, q.n_h, prefix, qmin[i], qmax[i],
                                                                hk.as<int64_t>() + h_off[i]); note_launch(); }
            RELNN_CUDA(cudaMemcpyAsync(zb.as<uint8_t>() + h_off[i] * d * S->z_esz, q.d_z, q.n_h * d * S->z_esz,
                                       cudaMemcpyDeviceToDevice, st));
        }
        if (q.n_tuples > 0) {
            { batch_keys_kernel<<<grid_for(q.n_tuples), 256, 0, st>>>((const int32_t*)q.d_src, q.n_tuples, prefix, qmin[i], qmax[i],
                                                                     sk.as<int64_t>() + t_off[i]); note_launch(); }
            { batch_keys_kernel<<<grid_for(q.n_tuples), 256, 0, st>>>((const int32_t*)q.d_dst, q.n_tuples, prefix, qmin[i], qmax[i],
                                                                     dk.as<int64_t>() + t_off[i]); note_launch(); }
        }
    }
    RELNN_CUDA(cudaGetLastError());
    relnn_branch_desc bd{sk.p, dk.p, T, 0, 0, nullptr};
    relnn_rule_desc desc{};
    desc.key_type = RELNN_I64;
    desc.d_h_ids = hk.p;
    desc.n_h = K;
    desc.d = d;
    desc.d_out = d_out;
    desc.n_branches = 1;
    desc.branches = &bd;
    desc.act = S->cfg.act;
    desc.flags = S->cfg.flags & (RELNN_FLAG_BF16 | RELNN_FLAG_KAHAN);
    if (T < S->cfg.tile128_below) desc.flags |= RELNN_FLAG_TILE128;
    Plan P;
    // on every exit the plan's buffers go back to the pool in stream order (no device-wide sync)
    struct Retire {
        Plan& p;
        cudaStream_t s;
        ~Retire() { p.retire_on(s); }
    } retire{P, st};
    RELNN_TRY(build_plan(P, &desc, st));
    DevBuf bo;
    RELNN_TRY(bo.alloc_tmp(sizeof(float) * std::max<int64_t>(P.n_out, 1) * d_out, st));
    if (P.n_out > 0) {
        CallIO io;
        io.z = zb.p;
        io.z_bf16 = S->cfg.z_dtype == RELNN_BF16;
        io.w_bf16 = S->cfg.w_dtype == RELNN_BF16;
        io.br.resize(1);
        io.br[0].W = S->cfg.d_W;
        io.br[0].b = S->cfg.d_b;
        if (P.bf16) RELNN_TRY(forward_tc(P, io, bo.as<float>(), st));
        else RELNN_TRY(forward_fp32(P, io, bo.as<float>(), st));
    }
    { ranges_kernel<<<(nq + 1 + 127) / 128, 128, 0, st>>>(P.out_keys.as<int64_t>(), P.n_out, nq, kb, lo.as<int64_t>()); note_launch(); }
    std::vector<int64_t> hlo(nq + 1);
    RELNN_CUDA(cudaMemcpyAsync(hlo.data(), lo.p, sizeof(int64_t) * (nq + 1), cudaMemcpyDeviceToHost, st));
    // the forward's device checks arrive with the same synchronisation (the kernels after it raise none)
    int dev_status = 0;
    RELNN_CUDA(cudaMemcpyAsync(&dev_status, P.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RELNN_CUDA(cudaStreamSynchronize(st));
    if (dev_status) {
        set_device_error(dev_status);
        return RELNN_EDEVICE;
    }
    for (int i = 0; i < nq; ++i) {
        Query* q = batch[i];
        q->n_out = hlo[i + 1] - hlo[i];
        q->batch_q = nq;
        if (q->n_out > 0) {
            RELNN_TRY(q->keys.alloc_tmp(sizeof(int32_t) * q->n_out, st));
            RELNN_TRY(q->z.alloc_tmp(sizeof(float) * q->n_out * d_out, st));
            { strip_keys_kernel<<<grid_for(q->n_out), 256, 0, st>>>(P.out_keys.as<int64_t>() + hlo[i], q->n_out,
                                                                    ((int64_t)1 << kb) - 1, qmin[i], q->keys.as<int32_t>()); note_launch(); }
            RELNN_CUDA(cudaMemcpyAsync(q->z.p, bo.as<float>() + hlo[i] * d_out, sizeof(float) * q->n_out * d_out,
                                       cudaMemcpyDeviceToDevice, st));
        }
    }
    RELNN_CUDA(cudaGetLastError());
    RELNN_CUDA(cudaStreamSynchronize(st));
    return RELNN_OK;
}

void worker_main(relnn_server_s* S) {
    cudaSetDevice(S->dev);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    while (true) {
        std::vector<Query*> batch;
        int64_t bmem = 0, btup = 0;
        // An idle worker polls the queue for up to kPollUs before it sleeps on the condition
        // variable: queries arriving within that time are taken by a thread that is still running
        // (a thread woken from sleep starts its next batch's host work several times slower).
        {
            const Clock::time_point p0 = Clock::now();
            while (S->n_queued.load(std::memory_order_acquire) == 0 && !S->stopping_flag.load(std::memory_order_acquire) &&
                   Clock::now() - p0 < std::chrono::microseconds(kPollUs))
                std::this_thread::yield();
        }
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                return (S->stopping && S->queue.empty()) ||
                       (!S->queue.empty() && S->mem_in_use + S->queue.front()->mem <= S->budget);
            });
            if (S->queue.empty()) break;  // stopping and drained
            // the device's free memory (other batches and other processes hold some of it): a batch
            // is admitted only while its estimate fits in 90 % of it as well as in the budget. The
            // reading is refreshed at an admission when it is older than 2 ms or when the front
            // query alone would take more than half of it (a driver query per admission otherwise
            // serialises the workers' launches)
            const Clock::time_point now0 = Clock::now();
            if (now0 - S->free_when > std::chrono::milliseconds(2) || 2 * S->queue.front()->mem > S->free_seen) {
                lk.unlock();
                size_t free_b = 0, total_b = 0;
                if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
                    (void)cudaGetLastError();
                    free_b = (size_t)S->budget;
                }
                lk.lock();
                S->free_seen = (int64_t)free_b;
                S->free_when = now0;
                if (S->queue.empty()) continue;
            }
            const int64_t avail = (int64_t)(0.9 * (double)S->free_seen);
            while (!S->queue.empty()) {
                Query* q = S->queue.front();
                if (!batch.empty() && ((int)batch.size() >= S->cfg.max_batch_queries ||
                                       btup + q->q.n_tuples > S->cfg.max_batch_tuples))
                    break;
                if (S->mem_in_use + bmem + q->mem > S->budget) break;
                // the first query of a batch always goes (its estimate fits the budget, and a
                // smaller free figure only means other batches still hold memory they will free)
                if (!batch.empty() && bmem + q->mem > avail) break;
                S->queue.pop_front();
                S->n_queued.fetch_sub(1, std::memory_order_release);
                q->state = 1;
                batch.push_back(q);
                bmem += q->mem;
                btup += q->q.n_tuples;
            }
            if (batch.empty()) continue;  // another worker took the front query meanwhile
            S->mem_in_use += bmem;
        }
        relnn_status s = run_batch(S, batch, st);
        cudaStreamSynchronize(st);
        for (Query* q : batch) {
            // results outlive this batch; their later frees need no ordering against this stream
            q->keys.st = nullptr;
            q->z.st = nullptr;
        }
        const Clock::time_point now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->mem_in_use -= bmem;
            for (Query* q : batch) {
                q->st = s;
                q->latency_us = std::chrono::duration<double, std::micro>(now - q->t_submit).count();
                q->state = 2;
            }
            S->in_system -= (int)batch.size();
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    cudaStreamDestroy(st);
}

}  // namespace
}  // namespace relnn

extern "C" {

relnn_status relnn_server_create(const relnn_server_cfg* cfg, relnn_server_t* out) {
    RELNN_CHECK_ARG(cfg && out, "server: null argument");
    RELNN_CHECK_ARG(cfg->d > 0 && cfg->d % 8 == 0 && cfg->d_out > 0 && cfg->d_out <= 256, "server: bad widths");
    RELNN_CHECK_ARG(cfg->d_W, "server: null W");
    RELNN_CHECK_ARG(cfg->n_workers >= 1 && cfg->n_workers <= 16, "server: 1..16 workers");
    RELNN_CHECK_ARG(cfg->max_queue >= 1 && cfg->max_batch_queries >= 1 && cfg->max_batch_tuples >= 1,
                    "server: bad queue / batch limits");
    *out = nullptr;
    relnn_server_s* S = new (std::nothrow) relnn_server_s();
    if (!S) return RELNN_ENOMEM;
    S->cfg = *cfg;
    S->z_esz = cfg->z_dtype == RELNN_BF16 ? 2 : 4;
    cudaGetDevice(&S->dev);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    S->budget = cfg->mem_budget_bytes > 0 ? cfg->mem_budget_bytes : (int64_t)(0.8 * (double)free_b);
    // The device's memory pool keeps freed blocks (ensure_pool_cached); it is grown here, once, to
    // what n_workers batches of max_batch_tuples tuples may hold together, so that the first burst of
    // large batches does not map new memory while queries wait (at most half of the budget).
    {
        relnn_query big{};
        big.n_tuples = cfg->max_batch_tuples;
        big.n_h = std::max<int64_t>(1, cfg->max_batch_tuples / 8);
        const int64_t want = std::min<int64_t>((int64_t)cfg->n_workers * query_mem(S, big), S->budget / 2);
        ensure_pool_cached();
        // memory freed on one worker's stream is reused by another only once its free has completed
        // (no event waits inserted between the workers' streams, which would serialise their batches)
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, S->dev) == cudaSuccess) {
            int off = 0;
            cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &off);
        }
        void* p = nullptr;
        if (want > 0 && cudaMallocAsync(&p, (size_t)want, nullptr) == cudaSuccess) {
            cudaFreeAsync(p, nullptr);
            cudaStreamSynchronize(nullptr);
        }
        (void)cudaGetLastError();
    }
    // One small batch of two queries runs before the workers start, so that the kernels of the
    // batched path (the key range of every query, the batch keys, the plan and the result split) are
    // loaded before the first query arrives.
    {
        const int64_t n = 64;
        DevBuf keys, z;
        cudaStream_t st = nullptr;
        bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
                  keys.alloc_tmp(sizeof(int32_t) * n, st) == RELNN_OK &&
                  z.alloc_tmp(S->z_esz * (size_t)cfg->d * n, st) == RELNN_OK;
        if (ok) {
            std::vector<int32_t> hk(n);
            for (int64_t i = 0; i < n; ++i) hk[i] = (int32_t)i;
            ok = cudaMemcpyAsync(keys.p, hk.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                 cudaMemsetAsync(z.p, 0, S->z_esz * (size_t)cfg->d * n, st) == cudaSuccess;
        }
        if (ok) {
            Query q0, q1;
            for (Query* q : {&q0, &q1}) {
                q->q.d_h_ids = keys.p;
                q->q.n_h = n;
                q->q.d_z = z.p;
                q->q.d_src = keys.p;
                q->q.d_dst = keys.p;
                q->q.n_tuples = n;
            }
            std::vector<Query*> warm = {&q0, &q1};
            (void)run_batch(S, warm, st);
            cudaStreamSynchronize(st);
            q0.keys.st = q0.z.st = q1.keys.st = q1.z.st = nullptr;
        }
        keys.release();
        z.release();
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
        (void)cudaGetLastError();
    }
    for (int i = 0; i < cfg->n_workers; ++i) S->workers.emplace_back(worker_main, S);
    *out = S;
    return RELNN_OK;
}

relnn_status relnn_serve_submit(relnn_server_t S, const relnn_query* q, uint64_t* ticket) {
    RELNN_CHECK_ARG(S && q && ticket, "submit: null argument");
    RELNN_CHECK_ARG(q->n_h >= 0 && q->n_tuples >= 0 && q->n_h < (1ll << 31) && q->n_tuples < (1ll << 31),
                    "submit: bad sizes");
    RELNN_CHECK_ARG((q->n_h == 0 || (q->d_h_ids && q->d_z)) && (q->n_tuples == 0 || (q->d_src && q->d_dst)),
                    "submit: null relation");
    const int64_t mem = query_mem(S, *q);
    if (mem > S->budget) {
        set_error("submit: query needs ~" + std::to_string(mem) + " device bytes, budget is " + std::to_string(S->budget));
        return RELNN_ENOMEM;
    }
    Query* Q = new (std::nothrow) Query();
    if (!Q) return RELNN_ENOMEM;
    Q->q = *q;
    Q->mem = mem;
    Q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) {
            delete Q;
            set_error("submit: server is stopping");
            return RELNN_EINVAL;
        }
        if (S->in_system >= S->cfg.max_queue) {
            delete Q;
            set_error("submit: queue full");
            return RELNN_EAGAIN;
        }
        Q->ticket = S->next_ticket++;
        S->all[Q->ticket] = Q;
        S->queue.push_back(Q);
        S->n_queued.fetch_add(1, std::memory_order_release);
        ++S->in_system;
        *ticket = Q->ticket;
    }
    S->cv_work.notify_one();
    return RELNN_OK;
}

relnn_status relnn_serve_poll(relnn_server_t S, uint64_t ticket, relnn_result* res, uint32_t timeout_us) {
    RELNN_CHECK_ARG(S && res, "poll: null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    RELNN_CHECK_ARG(it != S->all.end(), "poll: unknown ticket");
    Query* Q = it->second;
    if (Q->state != 2) {
        if (timeout_us == 0) return RELNN_EAGAIN;
        const bool done = S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return Q->state == 2; });
        if (!done) return RELNN_ETIMEDOUT;
    }
    res->n_out = Q->n_out;
    res->d_out_keys = Q->keys.as<int32_t>();
    res->d_out_z = Q->z.as<float>();
    res->latency_us = Q->latency_us;
    res->batch_queries = Q->batch_q;
    if (Q->st != RELNN_OK) set_error("poll: the query's batch failed");
    return Q->st;
}

relnn_status relnn_serve_release(relnn_server_t S, uint64_t ticket) {
    RELNN_CHECK_ARG(S, "release: null server");
    Query* Q = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->all.find(ticket);
        RELNN_CHECK_ARG(it != S->all.end(), "release: unknown ticket");
        RELNN_CHECK_ARG(it->second->state == 2, "release: query still running");
        Q = it->second;
        S->all.erase(it);
    }
    delete Q;
    return RELNN_OK;
}

relnn_status relnn_server_destroy(relnn_server_t S) {
    if (!S) return RELNN_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->stopping_flag.store(true, std::memory_order_release);
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    cudaDeviceSynchronize();
    for (auto& kv : S->all) delete kv.second;
    delete S;
    return RELNN_OK;
}

}  // extern "C"
