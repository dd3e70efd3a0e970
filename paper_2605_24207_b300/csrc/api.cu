// C ABI entry points of librelnn.so (declared in include/relnn.h).
#include <cstring>
#include <new>
#include <string>

#include "bwd.cuh"
#include "maxagg.cuh"
#include "mean.cuh"
#include "primitives.cuh"

namespace relnn {

static thread_local std::string g_last_error;
static thread_local int32_t g_last_dev_error = 0;

void set_error(const std::string& msg) { g_last_error = msg; }
void set_device_error(int32_t code) { g_last_dev_error = code; }

relnn_status join_probe_pairs(const JoinTable& jt, const void* probe, int64_t m, int32_t* probe_idx,
                              int32_t* build_idx, int64_t capacity, int64_t* d_count, cudaStream_t st);

namespace {

__global__ void keys_to_i32_kernel(const int64_t* in, int64_t n, int32_t* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

relnn_status copy_out_keys(const Plan& p, void* d_out_keys, cudaStream_t st) {
    if (!d_out_keys || p.n_out == 0) return RELNN_OK;
    if (p.kt == RELNN_I64) {
        RELNN_CUDA(cudaMemcpyAsync(d_out_keys, p.out_keys.p, sizeof(int64_t) * p.n_out, cudaMemcpyDeviceToDevice, st));
    } else {
        const int blocks = (int)std::min<int64_t>(ceil_div(p.n_out, 256), 4096);
        { keys_to_i32_kernel<<<blocks, 256, 0, st>>>(p.out_keys.as<int64_t>(), p.n_out, reinterpret_cast<int32_t*>(d_out_keys)); note_launch(); }
        RELNN_CUDA(cudaGetLastError());
    }
    return RELNN_OK;
}

relnn_status resolve_io(const Plan& p, const relnn_rule_params* prm, CallIO& io) {
    RELNN_CHECK_ARG(prm, "null params");
    RELNN_CHECK_ARG(p.n_h == 0 || prm->d_z, "params: null z");
    io.z = prm->d_z;
    io.z_bf16 = prm->z_dtype == RELNN_BF16;
    io.r_bf16 = prm->r_dtype == RELNN_BF16;
    io.w_bf16 = prm->w_dtype == RELNN_BF16;
    io.br.resize(p.br.size());
    for (size_t i = 0; i < p.br.size(); ++i) {
        if (p.br[i].d_r > 0) {
            RELNN_CHECK_ARG(prm->d_r && prm->d_r[i], "params: branch needs its per-tuple embedding r");
            io.br[i].r = prm->d_r[i];
        }
        if (!p.identity) {
            RELNN_CHECK_ARG(prm->d_W && prm->d_W[i], "params: null W");
            io.br[i].W = prm->d_W[i];
            io.br[i].b = prm->d_b ? prm->d_b[i] : nullptr;
        }
    }
    return RELNN_OK;
}

}  // namespace
}  // namespace relnn

using namespace relnn;

extern "C" {

int32_t relnn_version(void) { return 100; }

int32_t relnn_build_flags(void) { return kChecked ? 1 : 0; }

const char* relnn_status_string(relnn_status s) {
    switch (s) {
        case RELNN_OK: return "ok";
        case RELNN_EINVAL: return "invalid argument";
        case RELNN_ENOMEM: return "out of memory";
        case RELNN_ENOSPC: return "output capacity too small";
        case RELNN_EAGAIN: return "try again";
        case RELNN_ETIMEDOUT: return "timed out";
        case RELNN_ECUDA: return "CUDA error";
        case RELNN_EDEVICE: return "device-side check failed";
        case RELNN_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

const char* relnn_last_error(void) { return g_last_error.c_str(); }
int32_t relnn_last_device_error(void) { return g_last_dev_error; }

relnn_status relnn_join_build(const void* d_keys, int64_t n, relnn_key_t kt, void* stream, relnn_join_t* out) {
    RELNN_CHECK_ARG(out, "join build: null out");
    RELNN_CHECK_ARG(kt == RELNN_I32 || kt == RELNN_I64, "join build: bad key type");
    *out = nullptr;
    relnn_join_s* j = new (std::nothrow) relnn_join_s();
    if (!j) return RELNN_ENOMEM;
    relnn_status s = join_table_build(j->t, d_keys, n, kt, (cudaStream_t)stream);
    if (s != RELNN_OK) {
        delete j;
        return s;
    }
    *out = j;
    return RELNN_OK;
}

relnn_status relnn_join_probe(relnn_join_t j, const void* d_probe_keys, int64_t m, int32_t* d_probe_idx,
                              int32_t* d_build_idx, int64_t capacity, int64_t* d_count, void* stream) {
    RELNN_CHECK_ARG(j, "join probe: null join");
    RELNN_CHECK_ARG(m >= 0 && m < (1ll << 31) - 1, "join probe: m out of range");
    RELNN_CHECK_ARG(m == 0 || d_probe_keys, "join probe: null keys");
    RELNN_CHECK_ARG(capacity >= 0 && (capacity == 0 || (d_probe_idx && d_build_idx)), "join probe: null outputs");
    return join_probe_pairs(j->t, d_probe_keys, m, d_probe_idx, d_build_idx, capacity, d_count, (cudaStream_t)stream);
}

relnn_status relnn_join_destroy(relnn_join_t j) {
    if (!j) return RELNN_OK;
    cudaDeviceSynchronize();
    delete j;
    return RELNN_OK;
}

relnn_status relnn_rule_plan(const relnn_rule_desc* desc, void* stream, relnn_plan_t* out) {
    RELNN_CHECK_ARG(out, "rule plan: null out");
    *out = nullptr;
    relnn_plan_s* p = new (std::nothrow) relnn_plan_s();
    if (!p) return RELNN_ENOMEM;
    ProfToken pt = prof_begin(RELNN_PROF_PLAN, (cudaStream_t)stream);
    relnn_status s = build_plan(p->p, desc, (cudaStream_t)stream);
    prof_end(pt, (cudaStream_t)stream);
    if (s != RELNN_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        delete p;
        return s;
    }
    *out = p;
    return RELNN_OK;
}

relnn_status relnn_plan_info(relnn_plan_t p, int64_t* n_out, int64_t* n_matched_total, int64_t* h_matched) {
    RELNN_CHECK_ARG(p, "plan info: null plan");
    if (n_out) *n_out = p->p.n_out;
    if (n_matched_total) *n_matched_total = p->p.total_matched();
    if (h_matched)
        for (size_t i = 0; i < p->p.br.size(); ++i) h_matched[i] = p->p.br[i].m;
    return RELNN_OK;
}

relnn_status relnn_plan_out_keys(relnn_plan_t p, void* d_out_keys, void* stream) {
    RELNN_CHECK_ARG(p && d_out_keys, "plan out keys: null argument");
    return copy_out_keys(p->p, d_out_keys, (cudaStream_t)stream);
}

relnn_status relnn_plan_check(relnn_plan_t p, void* stream) {
    RELNN_CHECK_ARG(p, "plan check: null plan");
    RELNN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int v = 0;
    RELNN_CUDA(cudaMemcpy(&v, p->p.status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        RELNN_CUDA(cudaMemset(p->p.status.p, 0, sizeof(int)));
        set_device_error(v);
        set_error("device-side check failed with code " + std::to_string(v));
        return RELNN_EDEVICE;
    }
    return RELNN_OK;
}

relnn_status relnn_plan_set_z_version(relnn_plan_t p, uint64_t version) {
    RELNN_CHECK_ARG(p, "set z version: null plan");
    p->p.z_version = version;
    return RELNN_OK;
}

relnn_status relnn_rule_forward(relnn_plan_t p, const relnn_rule_params* prm, void* d_out_keys, float* d_out_z,
                                int64_t* d_out_count, void* stream) {
    RELNN_CHECK_ARG(p, "forward: null plan");
    Plan& P = p->p;
    RELNN_CHECK_ARG(P.n_out == 0 || d_out_z, "forward: null output");
    cudaStream_t st = (cudaStream_t)stream;
    CallIO io;
    RELNN_TRY(resolve_io(P, prm, io));
    const bool mean = (P.flags & RELNN_FLAG_MEAN) != 0;
    if (mean) RELNN_TRY(ensure_inv_count(P, st));
    if (P.n_out > 0) {
        if (P.flags & RELNN_FLAG_PUSHDOWN) RELNN_TRY(forward_pushdown(P, io, d_out_z, st));
        else if (P.bf16) RELNN_TRY(forward_tc(P, io, d_out_z, st));
        else RELNN_TRY(forward_fp32(P, io, d_out_z, st));
        if (mean) RELNN_TRY(scale_rows(d_out_z, P.inv_cnt.as<float>(), P.n_out, P.d_out, d_out_z, st));
    }
    if (P.flags & RELNN_FLAG_MAX) P.max_ready = true;
    RELNN_TRY(copy_out_keys(P, d_out_keys, st));
    if (d_out_count)
        RELNN_CUDA(cudaMemcpyAsync(d_out_count, &P.n_out, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    return RELNN_OK;
}

relnn_status relnn_rule_backward(relnn_plan_t p, const relnn_rule_params* prm, const float* d_dout, float* const* d_dW,
                                 float* const* d_db, float* d_dz, float* const* d_dr, void* stream) {
    RELNN_CHECK_ARG(p, "backward: null plan");
    Plan& P = p->p;
    cudaStream_t st = (cudaStream_t)stream;
    CallIO io;
    RELNN_TRY(resolve_io(P, prm, io));
    GradIO g;
    g.dout = d_dout;
    g.dz = d_dz;
    const size_t nb = P.br.size();
    g.dW.assign(nb, nullptr);
    g.db.assign(nb, nullptr);
    g.dr.assign(nb, nullptr);
    for (size_t i = 0; i < nb; ++i) {
        if (d_dW) g.dW[i] = d_dW[i];
        if (d_db) g.db[i] = d_db[i];
        if (d_dr) g.dr[i] = d_dr[i];
    }
    RELNN_CHECK_ARG(P.n_out == 0 || d_dout, "backward: null output gradient");
    if ((P.flags & RELNN_FLAG_MEAN) && P.n_out > 0) {  // MEAN: the SUM backward of dOut[k] / n_k
        RELNN_TRY(ensure_inv_count(P, st));
        RELNN_TRY(P.mean_dout.alloc(sizeof(float) * (size_t)P.n_out * P.d_out));
        RELNN_TRY(scale_rows(d_dout, P.inv_cnt.as<float>(), P.n_out, P.d_out, P.mean_dout.as<float>(), st));
        g.dout = P.mean_dout.as<float>();
    }
    if (P.flags & RELNN_FLAG_MAX) RELNN_TRY(build_win_mask(P, st));  // MAX: dOut to the argmax only
    if (P.bf16) return backward_tc(P, io, g, st);
    return backward_fp32(P, io, g, st);
}

relnn_status relnn_attention_forward(relnn_plan_t p, const relnn_attn_params* prm, float* d_out, float* d_lse,
                                     void* stream) {
    RELNN_CHECK_ARG(p, "attention: null plan");
    return attention_forward(p->p, prm, d_out, d_lse, (cudaStream_t)stream);
}

relnn_status relnn_attention_backward(relnn_plan_t p, const relnn_attn_params* prm, const float* d_fwd_out,
                                      const float* d_lse, const float* d_dout, float* d_dq, float* d_dk, float* d_dv,
                                      void* stream) {
    RELNN_CHECK_ARG(p, "attention backward: null plan");
    return attention_backward(p->p, prm, d_fwd_out, d_lse, d_dout, d_dq, d_dk, d_dv, (cudaStream_t)stream);
}

relnn_status relnn_plan_release(relnn_plan_t p, void* stream) {
    if (!p) return RELNN_OK;
    p->p.retire_on((cudaStream_t)stream);
    delete p;
    return RELNN_OK;
}

relnn_status relnn_plan_destroy(relnn_plan_t p) {
    if (!p) return RELNN_OK;
    cudaDeviceSynchronize();
    delete p;
    return RELNN_OK;
}

}  // extern "C"
