// Streaming a relation larger than device memory (relnn_stream_*; paper Sec. 6 names scaling for
// memory, by streaming the data to the GPU in mini-batches, as future work).
//
// E stays in host memory. H (ids, z) is device-resident and its build side is made once. A pass
// walks E in chunks with two device slots: while chunk i is planned (probe against the shared H
// table, grouping) and evaluated on the caller's stream, chunk i + 1's key columns (and r rows) are
// copied into the other slot on a copy stream; events order slot reuse. Chunk plans index their
// output rows by H's distinct keys, so every chunk adds its rows (one add per element, chunks in
// order) into one [U, d_out] accumulator and marks its keys present; the pass ends with a
// compaction to the present keys in ascending order, which is exactly the unchunked rule's output
// key set. The backward scatters dOut to the same distinct-key rows and re-plans each chunk,
// adding dz across chunks and the chunks' dW / db partials in order.
#include <cstring>
#include <new>
#include <vector>

#include "bwd.cuh"
#include "mean.cuh"
#include "primitives.cuh"

using namespace relnn;

struct relnn_stream_s {
    relnn_stream_desc d{};
    std::vector<relnn_filter> filters;
    JoinTable H;
    int64_t U = 0, chunk = 0, n_chunks = 0;
    int d_in = 0, d_out = 0, kbytes = 4;
    bool bf16 = false, identity = false, concat_dst = true, mean = false;
    DevBuf keys[2][2];  // [slot][src, dst]
    DevBuf rrow[2];     // [slot] r rows of the chunk
    DevBuf acc, present, cnt, iota, out_row, ddense, scratch, zbf, dw_tmp, db_tmp, dr_buf;
    int64_t n_out = -1;  // rows of the last forward (-1: none yet)
    cudaStream_t copy_st = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    ~relnn_stream_s() {
        for (int i = 0; i < 2; ++i) {
            if (copied[i]) cudaEventDestroy(copied[i]);
            if (consumed[i]) cudaEventDestroy(consumed[i]);
        }
        if (copy_st) cudaStreamDestroy(copy_st);
    }
};

namespace relnn {
namespace {

int grid_of(int64_t n) { return (int)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), 256), (int64_t)num_sms() * 8); }

__global__ void iota_i32_kernel(int32_t* v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (int32_t)i;
}

// Rows of present distinct keys, in key order: keys[r] = ukeys[u], out[r] = acc[u] (MEAN: / cnt[u]).
__global__ void compact_kernel(const int32_t* __restrict__ present, const int32_t* __restrict__ out_row,
                               const int64_t* __restrict__ ukeys, const float* __restrict__ acc,
                               const int32_t* __restrict__ cnt, int64_t U, int d_out, int key64, void* keys,
                               float* __restrict__ out) {
    const int64_t total = U * d_out;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = i / d_out;
        if (!present[u]) continue;
        const int o = (int)(i - u * d_out);
        const int64_t r = out_row[u];
        const float v = acc[i];
        out[r * d_out + o] = cnt ? v / (float)cnt[u] : v;
        if (o == 0 && keys) {
            if (key64) reinterpret_cast<int64_t*>(keys)[r] = ukeys[u];
            else reinterpret_cast<int32_t*>(keys)[r] = (int32_t)ukeys[u];
        }
    }
}

// dOut of the compacted rows back onto distinct-key rows (MEAN: / cnt), for the chunks' backward.
__global__ void spread_kernel(const int32_t* __restrict__ present, const int32_t* __restrict__ out_row,
                              const float* __restrict__ dout, const int32_t* __restrict__ cnt, int64_t U, int d_out,
                              float* __restrict__ dd) {
    const int64_t total = U * d_out;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = i / d_out;
        const int o = (int)(i - u * d_out);
        float v = 0.f;
        if (present[u]) {
            v = dout[(int64_t)out_row[u] * d_out + o];
            if (cnt) v /= (float)cnt[u];
        }
        dd[i] = v;
    }
}

__global__ void add_kernel(float* __restrict__ y, const float* __restrict__ x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

// Copies chunk i's keys (and r rows) into slot i & 1 on the copy stream, after the compute stream
// is done with the slot's previous chunk.
relnn_status issue_copy(relnn_stream_s* S, int64_t i, const void* h_r, int r_esz) {
    const int slot = (int)(i & 1);
    const int64_t lo = i * S->chunk, n = std::min(S->chunk, S->d.n_tuples - lo);
    RELNN_CUDA(cudaStreamWaitEvent(S->copy_st, S->consumed[slot], 0));
    const uint8_t* hs = reinterpret_cast<const uint8_t*>(S->d.h_src) + lo * S->kbytes;
    const uint8_t* hd = reinterpret_cast<const uint8_t*>(S->d.h_dst) + lo * S->kbytes;
    RELNN_CUDA(cudaMemcpyAsync(S->keys[slot][0].p, hs, n * S->kbytes, cudaMemcpyHostToDevice, S->copy_st));
    RELNN_CUDA(cudaMemcpyAsync(S->keys[slot][1].p, hd, n * S->kbytes, cudaMemcpyHostToDevice, S->copy_st));
    if (h_r && S->d.d_r > 0) {
        const size_t row = (size_t)S->d.d_r * r_esz;
        RELNN_CUDA(cudaMemcpyAsync(S->rrow[slot].p, reinterpret_cast<const uint8_t*>(h_r) + lo * row, n * row,
                                   cudaMemcpyHostToDevice, S->copy_st));
    }
    RELNN_CUDA(cudaEventRecord(S->copied[slot], S->copy_st));
    return RELNN_OK;
}

// Plans chunk `slot` (n tuples) against the stream's H side into P.
relnn_status plan_chunk(relnn_stream_s* S, int slot, int64_t n, uint32_t extra_flags, Plan& P, cudaStream_t st) {
    relnn_branch_desc bd{S->keys[slot][0].p, S->keys[slot][1].p, n, S->d.d_r, (int32_t)S->filters.size(),
                         S->filters.empty() ? nullptr : S->filters.data()};
    relnn_rule_desc rd{};
    rd.key_type = S->d.key_type;
    rd.d_h_ids = nullptr;
    rd.n_h = S->d.n_h;
    rd.d = S->d.d;
    rd.d_out = S->d.d_out;
    rd.n_branches = 1;
    rd.branches = &bd;
    rd.act = S->d.act;
    rd.flags = (S->d.flags & ~RELNN_FLAG_MEAN) | extra_flags;
    P.Hx = &S->H;
    P.dense_out = true;
    P.acc_out = true;
    P.present_ext = S->present.as<int32_t>();
    P.iota_ext = S->iota.as<int32_t>();
    return build_plan(P, &rd, st);
}

// Runs body(P, slot, lo, n) for every chunk, with the next chunk's copy in flight.
template <class F>
relnn_status for_each_chunk(relnn_stream_s* S, const void* h_r, int r_esz, uint32_t extra_flags, cudaStream_t st,
                            F&& body) {
    if (S->n_chunks == 0) return RELNN_OK;
    RELNN_TRY(issue_copy(S, 0, h_r, r_esz));
    for (int64_t i = 0; i < S->n_chunks; ++i) {
        const int slot = (int)(i & 1);
        const int64_t lo = i * S->chunk, n = std::min(S->chunk, S->d.n_tuples - lo);
        if (i + 1 < S->n_chunks) RELNN_TRY(issue_copy(S, i + 1, h_r, r_esz));
        RELNN_CUDA(cudaStreamWaitEvent(st, S->copied[slot], 0));
        {
            Plan P;
            relnn_status rc = plan_chunk(S, slot, n, extra_flags, P, st);
            if (rc == RELNN_OK) rc = body(P, slot, lo, n);
            P.retire_on(st);  // the chunk plan's buffers are freed in stream order
            if (rc != RELNN_OK) {
                cudaStreamSynchronize(S->copy_st);
                return rc;
            }
        }
        RELNN_CUDA(cudaEventRecord(S->consumed[slot], st));
    }
    RELNN_CUDA(cudaStreamSynchronize(S->copy_st));
    return RELNN_OK;
}

relnn_status resolve_stream_io(relnn_stream_s* S, const relnn_rule_params* prm, CallIO& io, const void** h_r,
                               int* r_esz, cudaStream_t st) {
    RELNN_CHECK_ARG(prm, "stream: null params");
    RELNN_CHECK_ARG(S->d.n_h == 0 || prm->d_z, "stream: null z");
    io.z = prm->d_z;
    io.z_bf16 = prm->z_dtype == RELNN_BF16;
    io.r_bf16 = prm->r_dtype == RELNN_BF16;
    io.w_bf16 = prm->w_dtype == RELNN_BF16;
    io.br.resize(1);
    *h_r = nullptr;
    *r_esz = io.r_bf16 ? 2 : 4;
    if (S->d.d_r > 0) {
        RELNN_CHECK_ARG(prm->d_r && prm->d_r[0], "stream: the rule needs its per-tuple embedding r (host)");
        *h_r = prm->d_r[0];
    }
    if (!S->identity) {
        RELNN_CHECK_ARG(prm->d_W && prm->d_W[0], "stream: null W");
        io.br[0].W = prm->d_W[0];
        io.br[0].b = prm->d_b ? prm->d_b[0] : nullptr;
    }
    // the BF16 form gathers bf16 rows: an f32 z is rounded once per pass, not once per chunk
    if (S->bf16 && !io.z_bf16 && S->d.n_h > 0) {
        const int64_t n = S->d.n_h * (int64_t)S->d.d;
        RELNN_CHECK_ARG(n % 4 == 0 && (reinterpret_cast<uintptr_t>(io.z) & 15u) == 0, "stream: z layout");
        RELNN_TRY(S->zbf.alloc(sizeof(uint16_t) * n));
        f32_to_bf16(reinterpret_cast<const float*>(io.z), n, S->zbf.as<uint16_t>(), st);
        io.z = S->zbf.p;
        io.z_bf16 = 1;
    }
    return RELNN_OK;
}

// Slot buffers for chunks of S->chunk tuples.
relnn_status alloc_slots(relnn_stream_s* S, int r_esz) {
    for (int s = 0; s < 2; ++s) {
        RELNN_TRY(S->keys[s][0].alloc((size_t)S->chunk * S->kbytes));
        RELNN_TRY(S->keys[s][1].alloc((size_t)S->chunk * S->kbytes));
        if (S->d.d_r > 0) RELNN_TRY(S->rrow[s].alloc((size_t)S->chunk * S->d.d_r * r_esz));
    }
    return RELNN_OK;
}

}  // namespace
}  // namespace relnn

extern "C" {

relnn_status relnn_stream_create(const relnn_stream_desc* desc, void* stream, relnn_stream_t* out) {
    RELNN_CHECK_ARG(desc && out, "stream create: null argument");
    *out = nullptr;
    RELNN_CHECK_ARG(desc->key_type == RELNN_I32 || desc->key_type == RELNN_I64, "stream: bad key type");
    RELNN_CHECK_ARG(desc->n_h >= 0 && (desc->n_h == 0 || desc->d_h_ids), "stream: bad H");
    RELNN_CHECK_ARG(desc->n_tuples >= 0 && (desc->n_tuples == 0 || (desc->h_src && desc->h_dst)), "stream: bad E");
    RELNN_CHECK_ARG(desc->d > 0 && desc->d <= 4096 && desc->d_r >= 0 && desc->d_r <= 4096, "stream: bad widths");
    RELNN_CHECK_ARG(desc->act == RELNN_ACT_NONE || desc->act == RELNN_ACT_RELU, "stream: bad act");
    const uint32_t allowed = RELNN_FLAG_BF16 | RELNN_FLAG_KAHAN | RELNN_FLAG_IDENTITY | RELNN_FLAG_NO_CONCAT_DST |
                             RELNN_FLAG_MEAN | RELNN_FLAG_TILE128;
    RELNN_CHECK_ARG((desc->flags & ~allowed) == 0,
                    "stream: flags outside BF16 | KAHAN | IDENTITY | NO_CONCAT_DST | MEAN | TILE128");
    RELNN_CHECK_ARG(desc->n_filters >= 0 && desc->n_filters <= RELNN_MAX_FILTERS &&
                        (desc->n_filters == 0 || desc->filters), "stream: bad filter list");
    cudaStream_t st = (cudaStream_t)stream;
    relnn_stream_s* S = new (std::nothrow) relnn_stream_s();
    if (!S) return RELNN_ENOMEM;
    S->d = *desc;
    S->filters.assign(desc->filters, desc->filters + desc->n_filters);
    S->kbytes = desc->key_type == RELNN_I64 ? 8 : 4;
    S->bf16 = (desc->flags & RELNN_FLAG_BF16) != 0;
    S->identity = (desc->flags & RELNN_FLAG_IDENTITY) != 0;
    S->mean = (desc->flags & RELNN_FLAG_MEAN) != 0;
    S->concat_dst = !(desc->flags & RELNN_FLAG_NO_CONCAT_DST);
    S->d_in = desc->d * (S->concat_dst ? 2 : 1) + desc->d_r;
    S->d_out = S->identity ? S->d_in : desc->d_out;
    auto fail = [&](relnn_status s) {
        cudaStreamSynchronize(st);
        delete S;
        return s;
    };
    if (S->d_out <= 0 || S->d_out > 4096) {
        set_error("stream: bad d_out");
        return fail(RELNN_EINVAL);
    }
    relnn_status rc = join_table_build(S->H, desc->d_h_ids, desc->n_h, desc->key_type, st);
    if (rc != RELNN_OK) return fail(rc);
    S->U = S->H.n_unique;
    const int64_t U = S->U;
    const size_t rows = sizeof(float) * (size_t)std::max<int64_t>(U, 1) * S->d_out;
    // accumulator, dense dOut, and (BF16 with ReLU) the scratch output of the backward's re-forward
    const bool need_scratch = S->bf16 && desc->act == RELNN_ACT_RELU;
    int64_t fixed = (int64_t)rows * (2 + (need_scratch ? 1 : 0)) + 16 * (U + 1);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(RELNN_ECUDA);
    const int64_t budget = desc->mem_budget_bytes > 0 ? desc->mem_budget_bytes : (int64_t)(free_b / 4);
    // device bytes per chunk tuple: two slots of keys and r rows, plus the chunk plan's arrays, sort
    // temporaries, boundary partials and masks (the serving path's per-tuple estimate)
    const int64_t per_tuple = 2 * (2 * S->kbytes + (int64_t)desc->d_r * 4) + 112 + (need_scratch ? 32 : 0);
    if (desc->chunk_tuples > 0) {
        S->chunk = desc->chunk_tuples;
    } else {
        if (budget <= fixed + per_tuple * 4096) {
            set_error("stream: memory budget below the accumulators and a minimal chunk");
            return fail(RELNN_ENOMEM);
        }
        S->chunk = (budget - fixed) / per_tuple;
    }
    S->chunk = std::max<int64_t>(1, std::min<int64_t>(S->chunk, std::min<int64_t>((1ll << 31) - 2, std::max<int64_t>(desc->n_tuples, 1))));
    S->n_chunks = ceil_div(desc->n_tuples, S->chunk);
    if ((rc = S->acc.alloc(rows)) != RELNN_OK) return fail(rc);
    if ((rc = S->ddense.alloc(rows)) != RELNN_OK) return fail(rc);
    if (need_scratch) {
        if ((rc = S->scratch.alloc(rows)) != RELNN_OK) return fail(rc);
        if (cudaMemsetAsync(S->scratch.p, 0, rows, st) != cudaSuccess) return fail(RELNN_ECUDA);
    }
    if ((rc = S->present.alloc(sizeof(int32_t) * (U + 1))) != RELNN_OK) return fail(rc);
    if ((rc = S->out_row.alloc(sizeof(int32_t) * (U + 1))) != RELNN_OK) return fail(rc);
    if ((rc = S->iota.alloc(sizeof(int32_t) * (U + 1))) != RELNN_OK) return fail(rc);
    if (S->mean && (rc = S->cnt.alloc(sizeof(int32_t) * std::max<int64_t>(U, 1))) != RELNN_OK) return fail(rc);
    { iota_i32_kernel<<<grid_of(U + 1), 256, 0, st>>>(S->iota.as<int32_t>(), U + 1); note_launch(); }
    if (cudaStreamCreateWithFlags(&S->copy_st, cudaStreamNonBlocking) != cudaSuccess) return fail(RELNN_ECUDA);
    for (int i = 0; i < 2; ++i)
        if (cudaEventCreateWithFlags(&S->copied[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&S->consumed[i], cudaEventDisableTiming) != cudaSuccess)
            return fail(RELNN_ECUDA);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(RELNN_ECUDA);
    *out = S;
    return RELNN_OK;
}

relnn_status relnn_stream_info(relnn_stream_t s, int64_t* max_out_rows, int64_t* chunk_tuples, int64_t* n_chunks) {
    RELNN_CHECK_ARG(s, "stream info: null stream");
    if (max_out_rows) *max_out_rows = s->U;
    if (chunk_tuples) *chunk_tuples = s->chunk;
    if (n_chunks) *n_chunks = s->n_chunks;
    return RELNN_OK;
}

relnn_status relnn_stream_forward(relnn_stream_t S, const relnn_rule_params* prm, void* d_out_keys, float* d_out_z,
                                  int64_t* h_n_out, void* stream) {
    RELNN_CHECK_ARG(S && (S->U == 0 || d_out_z), "stream forward: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    CallIO io;
    const void* h_r = nullptr;
    int r_esz = 4;
    RELNN_TRY(resolve_stream_io(S, prm, io, &h_r, &r_esz, st));
    RELNN_TRY(alloc_slots(S, r_esz));
    const int64_t U = S->U;
    S->n_out = -1;
    RELNN_CUDA(cudaMemsetAsync(S->acc.p, 0, sizeof(float) * (size_t)std::max<int64_t>(U, 1) * S->d_out, st));
    RELNN_CUDA(cudaMemsetAsync(S->present.p, 0, sizeof(int32_t) * (U + 1), st));
    if (S->mean) RELNN_CUDA(cudaMemsetAsync(S->cnt.p, 0, sizeof(int32_t) * std::max<int64_t>(U, 1), st));
    RELNN_TRY(for_each_chunk(S, h_r, r_esz, 0u, st, [&](Plan& P, int slot, int64_t, int64_t) -> relnn_status {
        CallIO cio = io;
        cio.br[0].r = S->d.d_r > 0 ? S->rrow[slot].p : nullptr;
        if (P.br[0].m == 0) return RELNN_OK;
        if (P.bf16) RELNN_TRY(forward_tc(P, cio, S->acc.as<float>(), st));
        else RELNN_TRY(forward_fp32(P, cio, S->acc.as<float>(), st));
        if (S->mean) RELNN_TRY(count_rows_into(P.br[0].seg.as<int32_t>(), P.br[0].m, S->cnt.as<int32_t>(), st));
        return RELNN_OK;
    }));
    // compaction to the present keys, ascending
    RELNN_TRY(exclusive_scan<int32_t>(S->present.as<int32_t>(), S->out_row.as<int32_t>(), U,
                                      S->out_row.as<int32_t>() + U, st));
    int32_t n_out = 0;
    RELNN_CUDA(cudaMemcpyAsync(&n_out, S->out_row.as<int32_t>() + U, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (U > 0)
        { compact_kernel<<<grid_of(U * S->d_out), 256, 0, st>>>(S->present.as<int32_t>(), S->out_row.as<int32_t>(),
                                                               S->H.ukeys.as<int64_t>(), S->acc.as<float>(),
                                                               S->mean ? S->cnt.as<int32_t>() : nullptr, U, S->d_out,
                                                               S->kbytes == 8, d_out_keys, d_out_z); note_launch(); }
    RELNN_CUDA(cudaGetLastError());
    RELNN_CUDA(cudaStreamSynchronize(st));
    S->n_out = n_out;
    if (h_n_out) *h_n_out = n_out;
    return RELNN_OK;
}

relnn_status relnn_stream_backward(relnn_stream_t S, const relnn_rule_params* prm, const float* d_dout, float* d_dW,
                                   float* d_db, float* d_dz, float* h_dr, void* stream) {
    RELNN_CHECK_ARG(S, "stream backward: null stream");
    if (S->n_out < 0) {
        set_error("stream backward: run relnn_stream_forward first (its output rows define dOut's rows)");
        return RELNN_ENOTSUP;
    }
    RELNN_CHECK_ARG(S->n_out == 0 || d_dout, "stream backward: null output gradient");
    cudaStream_t st = (cudaStream_t)stream;
    CallIO io;
    const void* h_r = nullptr;
    int r_esz = 4;
    RELNN_TRY(resolve_stream_io(S, prm, io, &h_r, &r_esz, st));
    RELNN_TRY(alloc_slots(S, r_esz));
    const int64_t U = S->U;
    const int d_out = S->d_out, d_in = S->d_in;
    const bool want_w = !S->identity && (d_dW || d_db);
    if (U > 0)
        { spread_kernel<<<grid_of(U * d_out), 256, 0, st>>>(S->present.as<int32_t>(), S->out_row.as<int32_t>(), d_dout,
                                                           S->mean ? S->cnt.as<int32_t>() : nullptr, U, d_out,
                                                           S->ddense.as<float>()); note_launch(); }
    if (d_dz) RELNN_CUDA(cudaMemsetAsync(d_dz, 0, sizeof(float) * S->d.n_h * S->d.d, st));
    if (d_dW) RELNN_CUDA(cudaMemsetAsync(d_dW, 0, sizeof(float) * d_out * d_in, st));
    if (d_db) RELNN_CUDA(cudaMemsetAsync(d_db, 0, sizeof(float) * d_out, st));
    if (want_w) {
        RELNN_TRY(S->dw_tmp.alloc(sizeof(float) * d_out * d_in));
        RELNN_TRY(S->db_tmp.alloc(sizeof(float) * d_out));
    }
    if (h_r && h_dr) RELNN_TRY(S->dr_buf.alloc(sizeof(float) * (size_t)S->chunk * S->d.d_r));
    // a BF16 rule with ReLU needs each chunk's ReLU mask: the chunk's forward runs again first
    const bool refwd = S->bf16 && S->d.act == RELNN_ACT_RELU;
    RELNN_TRY(for_each_chunk(S, h_r, r_esz, refwd ? RELNN_FLAG_RELU_MASK : 0u, st,
                             [&](Plan& P, int slot, int64_t lo, int64_t n) -> relnn_status {
        CallIO cio = io;
        cio.br[0].r = S->d.d_r > 0 ? S->rrow[slot].p : nullptr;
        float* dr = (h_r && h_dr) ? S->dr_buf.as<float>() : nullptr;
        if (P.br[0].m > 0) {
            if (refwd) RELNN_TRY(forward_tc(P, cio, S->scratch.as<float>(), st));
            GradIO g;
            g.dout = S->ddense.as<float>();
            g.dz = d_dz;
            g.accumulate_dz = true;
            g.dW.assign(1, want_w && d_dW ? S->dw_tmp.as<float>() : nullptr);
            g.db.assign(1, want_w && d_db ? S->db_tmp.as<float>() : nullptr);
            g.dr.assign(1, dr);
            if (P.bf16) RELNN_TRY(backward_tc(P, cio, g, st));
            else RELNN_TRY(backward_fp32(P, cio, g, st));
            if (want_w && d_dW) { add_kernel<<<grid_of((int64_t)d_out * d_in), 256, 0, st>>>(d_dW, S->dw_tmp.as<float>(), (int64_t)d_out * d_in); note_launch(); }
            if (want_w && d_db) { add_kernel<<<grid_of(d_out), 256, 0, st>>>(d_db, S->db_tmp.as<float>(), d_out); note_launch(); }
            RELNN_CUDA(cudaGetLastError());
        } else if (dr) {
            RELNN_CUDA(cudaMemsetAsync(dr, 0, sizeof(float) * n * S->d.d_r, st));
        }
        if (dr)
            RELNN_CUDA(cudaMemcpyAsync(h_dr + lo * S->d.d_r, dr, sizeof(float) * n * S->d.d_r, cudaMemcpyDeviceToHost, st));
        return RELNN_OK;
    }));
    RELNN_CUDA(cudaStreamSynchronize(st));
    return RELNN_OK;
}

relnn_status relnn_stream_destroy(relnn_stream_t s) {
    if (!s) return RELNN_OK;
    cudaDeviceSynchronize();
    delete s;
    return RELNN_OK;
}

}  // extern "C"
