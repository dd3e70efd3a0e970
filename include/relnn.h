/*
 * relnn.h -- C ABI of librelnn.so: evaluation of RelaNN rules over embedded relations on one
 * NVIDIA B300 (sm_103a).
 *
 * The operation (paper Sec. 2.2 and Sec. 3.1): a join rule
 *
 *     H'(dst; SUM(tau(Concat(z_src, z_dst [, r])))) :- E(src, dst [; r]), H(src; z_src), H(dst; z_dst)
 *
 * compiles to U_{SUM,dst}(T_tau(E |><| H |><| H)): an integer-key equi-join of the tuple relation E
 * with the embedded relation H on both src and dst (bag semantics: duplicate keys all match, a key
 * absent from H drops the tuple), the concatenation of the matched embeddings (Sec. 2.2, Join), a
 * per-tuple Linear tau(x) = x W^T + b with optional ReLU (Sec. 2.2, Transformation), and a SUM
 * group-by on the dst key (Sec. 2.2, Projected union). Several tuple relations E_1..E_n with their
 * own Linear each ("union rule" / "|..." replicator, Sec. 3.1 and Sec. 3.7) add into one output.
 *
 * Conventions for every entry point:
 *   - Returns relnn_status; no C++ exception crosses the ABI. relnn_last_error() gives a message.
 *   - Pointers named d_* are DEVICE pointers owned by the caller (the library never frees them);
 *     h_* pointers are host memory. Handles (join, plan, server) are owned by the library and are
 *     released only by the matching *_destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls marked
 *     "async" only enqueue work on it; calls marked "sync" return after the stream has drained.
 *     A plan's workspaces are allocated and grown in the order of the stream of the call that
 *     needs them, so calls on one plan must be ordered by the caller: issued on one stream, or
 *     ordered across streams (events, or a synchronisation) before a call on another stream.
 *   - Keys are int32 (RELNN_I32) or int64 (RELNN_I64). INT64_MAX is reserved and rejected as an H
 *     key. Embeddings are row-major [rows, width] with contiguous rows, f32 or bf16.
 *   - W uses the torch nn.Linear layout [d_out, d_in] row-major; b is f32 [d_out].
 *   - Device-side checks never trap: a failed check writes a code to the plan's status word and the
 *     kernel returns; relnn_plan_check() reports it as RELNN_EDEVICE with relnn_last_device_error().
 */
#ifndef RELNN_H
#define RELNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum relnn_status {
    RELNN_OK = 0,
    RELNN_EINVAL = 1,     /* invalid argument (null pointer, bad size, unsupported shape)        */
    RELNN_ENOMEM = 2,     /* device allocation failed, or a query can never fit the memory budget */
    RELNN_ENOSPC = 3,     /* caller-provided output capacity too small (required size reported)   */
    RELNN_EAGAIN = 4,     /* try again: serving queue full, or a ticket not finished yet           */
    RELNN_ETIMEDOUT = 5,  /* a bounded wait ran out                                                */
    RELNN_ECUDA = 6,      /* a CUDA runtime/driver call failed                                     */
    RELNN_EDEVICE = 7,    /* a device-side check failed; code in relnn_last_device_error()         */
    RELNN_ENOTSUP = 8     /* feature/shape combination the library does not support               */
} relnn_status;

typedef enum relnn_key_t { RELNN_I32 = 0, RELNN_I64 = 1 } relnn_key_t;
typedef enum relnn_float_t { RELNN_F32 = 0, RELNN_BF16 = 1 } relnn_float_t;
typedef enum relnn_act_t { RELNN_ACT_NONE = 0, RELNN_ACT_RELU = 1 } relnn_act_t;

/* relnn_rule_desc.flags */
#define RELNN_FLAG_BF16 0x1u          /* Linear on tcgen05 tensor cores: bf16 operands, f32 accumulate.
                                         Without it: the FP32 form (f32 FMA on CUDA cores, no TF32). */
#define RELNN_FLAG_KAHAN 0x2u         /* compensated (Kahan) f32 summation in the SUM group-by        */
#define RELNN_FLAG_IDENTITY 0x4u      /* tau = identity: no Linear, d_out = width of the Concat        */
#define RELNN_FLAG_NO_JOIN_DST 0x8u   /* dst is content only: not joined with H, no z_dst; the output
                                         is keyed by the raw dst value (e.g. a readout into groups)    */
#define RELNN_FLAG_NO_CONCAT_DST 0x10u /* join H(dst) (it filters tuples) but leave z_dst out of Concat */
#define RELNN_FLAG_RELU_MASK 0x20u    /* forward stores the per-tuple ReLU mask for a later backward   */
#define RELNN_FLAG_TILE128 0x40u      /* BF16 forward: 128 matched tuples per tile instead of 256      */
#define RELNN_FLAG_PUSHDOWN 0x80u     /* forward with the Linear pushed below the join (paper Sec. 6):
                                         P = Z W_src^T, Q = Z W_dst^T + b once per H row on tensor
                                         cores (bf16 operands, f32 accumulate), then Out[k] = SUM
                                         over the tuples of k of act(P[src] + Q[dst]) in f32. No
                                         per-tuple embedding; d_out a multiple of 32, at most 128.
                                         The backward is the per-tuple one (RELNN_FLAG_RELU_MASK is
                                         honoured).                                                */
#define RELNN_FLAG_MEAN 0x100u        /* aggregator MEAN instead of SUM (paper Sec. 2.2 alpha): each
                                         output row is the SUM divided by its number of matched
                                         tuples; single-branch rules only (EINVAL otherwise)       */
#define RELNN_FLAG_MAX 0x200u         /* aggregator MAX instead of SUM (paper Sec. 2.2 alpha; Sec. 4.2
                                         scatter-max): per output row and feature, the maximum of
                                         tau(...) over its matched tuples. Single-branch rules; not
                                         with MEAN or PUSHDOWN (EINVAL). The forward records, per row
                                         and feature, the first tuple reaching the maximum in the
                                         plan's order (dst H row, then E row, then src H row); the
                                         backward sends dOut there only (times ReLU' at it), so it
                                         needs a forward of the same plan first.                   */

#define RELNN_FLAG_PER_TUPLE 0x400u   /* BF16 form without an activation: apply the Linear to every
                                         matched tuple and then SUM (the order of the rule as
                                         written), instead of the default for such rules, which
                                         sums each output row's Concat rows first and applies the
                                         Linear once per row (SUM commutes with a linear map;
                                         paper Sec. 2.2 alpha, Sec. 6 hybrid rewrites). Both give
                                         the rule's result; they differ in the order of f32
                                         additions and in speed.                                   */

/* Device status codes (relnn_last_device_error) */
#define RELNN_DEV_OK 0
#define RELNN_DEV_TIMEOUT 1           /* a bounded spin/mbarrier wait gave up                         */
#define RELNN_DEV_BOUNDS 2            /* an index failed its bounds check                             */
#define RELNN_DEV_HASH_FULL 3         /* hash insert found no free slot                               */

typedef struct relnn_join_s* relnn_join_t;
typedef struct relnn_plan_s* relnn_plan_t;
typedef struct relnn_server_s* relnn_server_t;
typedef struct relnn_stream_s* relnn_stream_t;
typedef struct relnn_tri_s* relnn_tri_t;

/* ---------------------------------------------------------------------------------------------
 * Library
 * ------------------------------------------------------------------------------------------- */
int32_t relnn_version(void);                      /* 100 * major + minor                          */
int32_t relnn_build_flags(void);                  /* bit 0: the checked build (-DRELNN_CHECKED:
                                                     gathered indices and output rows are tested
                                                     on the device, a failing one raises
                                                     RELNN_DEV_BOUNDS and the access is skipped)  */
const char* relnn_status_string(relnn_status s);  /* static string                                */
const char* relnn_last_error(void);               /* calling thread's last error message          */
int32_t relnn_last_device_error(void);            /* RELNN_DEV_* of the last RELNN_EDEVICE        */

/* ---------------------------------------------------------------------------------------------
 * Join (paper Sec. 2.2 "Join": natural join on shared attributes; Sec. 4.2: the join emits row-index
 * tensors). Build side: a key column. Probe side: another key column. Bag semantics.
 * ------------------------------------------------------------------------------------------- */

/* sync. Builds a lookup structure over d_keys[0..n) (radix-sorted (key,row) pairs plus a hash
 * table, or a direct-address table when the key range is small). d_keys may be freed after return.
 * Errors: EINVAL (null/negative n, INT64_MAX key), ENOMEM, ECUDA. */
relnn_status relnn_join_build(const void* d_keys, int64_t n, relnn_key_t kt, void* stream,
                              relnn_join_t* out);

/* sync. Emits every matching (probe row, build row) pair of d_probe_keys[0..m) against the build
 * side into d_probe_idx / d_build_idx (int32, capacity entries each), ordered by probe row and then
 * by build row. *d_count (device int64) receives the number of pairs. If it exceeds `capacity`,
 * nothing is written to the index arrays, *d_count holds the required size and RELNN_ENOSPC is
 * returned. Probe keys must have the build's key type. */
relnn_status relnn_join_probe(relnn_join_t j, const void* d_probe_keys, int64_t m,
                              int32_t* d_probe_idx, int32_t* d_build_idx, int64_t capacity,
                              int64_t* d_count, void* stream);

/* Releases the join's device memory (waits for the device first). */
relnn_status relnn_join_destroy(relnn_join_t j);

/* ---------------------------------------------------------------------------------------------
 * Rules (paper Sec. 3.1 join rule, union rule; Sec. 3.7 "|..." replicator).
 * ------------------------------------------------------------------------------------------- */
/* Selection (paper Sec. 3.1 filter expressions, Sec. 4.2 sigma): an atomic predicate
 * lhs op rhs over the tuple's content variables (its src and dst keys) and integer constants; a
 * branch's predicates are conjunctive. A tuple that fails one is dropped before the join. */
typedef enum relnn_term_t { RELNN_TERM_SRC = 0, RELNN_TERM_DST = 1, RELNN_TERM_CONST = 2 } relnn_term_t;
typedef enum relnn_cmp_t {
    RELNN_CMP_EQ = 0, RELNN_CMP_NE = 1, RELNN_CMP_LT = 2, RELNN_CMP_LE = 3, RELNN_CMP_GT = 4, RELNN_CMP_GE = 5
} relnn_cmp_t;
#define RELNN_MAX_FILTERS 4
typedef struct relnn_filter {
    int32_t lhs, op, rhs;  /* relnn_term_t, relnn_cmp_t, relnn_term_t                             */
    int32_t reserved;      /* 0                                                                    */
    int64_t lhs_const;     /* value of lhs when lhs == RELNN_TERM_CONST (compared as signed keys)  */
    int64_t rhs_const;     /* value of rhs when rhs == RELNN_TERM_CONST                            */
} relnn_filter;

typedef struct relnn_branch_desc {
    const void* d_src;     /* [n_tuples] keys of E.src (device)                                   */
    const void* d_dst;     /* [n_tuples] keys of E.dst (device)                                   */
    int64_t n_tuples;      /* rows of this E relation (< 2^31)                                     */
    int32_t d_r;           /* width of the per-tuple embedding r (0 = none)                        */
    int32_t n_filters;     /* 0..RELNN_MAX_FILTERS predicates in `filters`                         */
    const relnn_filter* filters;  /* host array [n_filters] or NULL                               */
} relnn_branch_desc;

typedef struct relnn_rule_desc {
    relnn_key_t key_type;  /* type of H.id, E.src, E.dst                                          */
    const void* d_h_ids;   /* [n_h] keys of H (device)                                            */
    int64_t n_h;
    int32_t d;             /* width of H.z                                                        */
    int32_t d_out;         /* width of the output embedding (ignored with RELNN_FLAG_IDENTITY)     */
    int32_t n_branches;    /* >= 1; branches share H and the output key space                     */
    const relnn_branch_desc* branches;  /* host array [n_branches]                                */
    relnn_act_t act;
    uint32_t flags;        /* RELNN_FLAG_*                                                        */
} relnn_rule_desc;

/* sync. The content track of the rule (join build on H.id, probe of every branch's src and dst,
 * grouping of the matched tuples by output key), cached in the plan and reused by every forward and
 * backward (the paper's content caching across training iterations). Key columns may be freed
 * after return. Errors: EINVAL, ENOTSUP (shape the kernels do not cover), ENOMEM, ECUDA, EDEVICE. */
relnn_status relnn_rule_plan(const relnn_rule_desc* desc, void* stream, relnn_plan_t* out);

/* Host-side sizes of a plan: number of output rows, total matched (join-output) tuples over all
 * branches, and the matched tuples of branch i in h_matched[i] (may be NULL). */
relnn_status relnn_plan_info(relnn_plan_t p, int64_t* n_out, int64_t* n_matched_total,
                             int64_t* h_matched);

/* async. Writes the sorted output keys ([n_out], plan key type) to d_out_keys. */
relnn_status relnn_plan_out_keys(relnn_plan_t p, void* d_out_keys, void* stream);

/* sync. Drains `stream` and reports a device-side failure of any earlier call on this plan as
 * RELNN_EDEVICE (and clears it). */
relnn_status relnn_plan_check(relnn_plan_t p, void* stream);

/* sync (host only). The caller's promise about H.z for the following calls on this plan: an f32 table
 * passed at the same address with the same nonzero `version` holds the same values. The BF16 form
 * then converts the table to bf16 once per version and reuses the copy across forwards and
 * backwards (a training step's forward and backward share one conversion). version 0 (the default)
 * promises nothing: the table is converted on every call. Changing the table without changing the
 * version gives results computed from the stale copy. */
relnn_status relnn_plan_set_z_version(relnn_plan_t p, uint64_t version);

typedef struct relnn_rule_params {
    const void* d_z;               /* H.z [n_h, d]                                                 */
    relnn_float_t z_dtype;
    const void* const* d_r;        /* host array [n_branches] of device [n_tuples_i, d_r] or NULL   */
    relnn_float_t r_dtype;
    const void* const* d_W;        /* host array [n_branches] of device W_i [d_out, d_in]           */
    relnn_float_t w_dtype;
    const float* const* d_b;       /* host array [n_branches] of device b_i [d_out] (or NULL = 0)   */
} relnn_rule_params;

/* async. Forward of the rule: d_out_z [n_out, d_out] f32 receives, for each output key (sorted as
 * relnn_plan_out_keys), the SUM (MEAN, MAX with those flags) over every branch's matched tuples with
 * that dst key of tau(Concat(...)). d_out_keys (may be NULL) receives the keys; d_out_count (device int64, may be
 * NULL) receives n_out. d_out_z is fully overwritten. Concat widths: the BF16 form needs d and d_r
 * to be multiples of 8 and d_in, d_out <= 256; the FP32 form needs d_in, d_out <= 256. */
relnn_status relnn_rule_forward(relnn_plan_t p, const relnn_rule_params* prm, void* d_out_keys,
                                float* d_out_z, int64_t* d_out_count, void* stream);

/* async. Backward of relnn_rule_forward for the output gradient d_dout [n_out, d_out] f32:
 * d_dW[i] [d_out, d_in] f32, d_db[i] [d_out] f32, d_dz [n_h, d] f32 and d_dr[i] [n_tuples_i, d_r]
 * f32 are OVERWRITTEN with the gradients (any of the host arrays or entries may be NULL to skip).
 * The gathered Concat rows are recomputed, not stored. With act = RELU the BF16 form's forward must
 * have run with RELNN_FLAG_RELU_MASK (the mask is kept in the plan); with RELNN_FLAG_MAX the plan's
 * last forward must have run (its argmax is kept in the plan), ENOTSUP otherwise. */
relnn_status relnn_rule_backward(relnn_plan_t p, const relnn_rule_params* prm, const float* d_dout,
                                 float* const* d_dW, float* const* d_db, float* d_dz,
                                 float* const* d_dr, void* stream);

/* Attention over a rule's join (paper Sec. 1: Score(p, t; q*k) :- Treat(p, t), Queries(p; q),
 * Keys(t; k) and Attention(p; sum(a*v)) :- Score(p, t; a), Values(t; v); Sec. 5: the HGT head).
 * On a single-branch plan with a dst join and no per-tuple embedding, E(src = t, dst = p): every
 * output key p attends over its matched tuples, with q from the dst side's H row and k, v from the
 * src side's H row (rows of d_q, d_k, d_v are aligned with H's rows).
 *   RELNN_ATTN_PRODUCT: Out[p] = sum_t q_t * k_t * v_t (element-wise).
 *   RELNN_ATTN_SOFTMAX: per head h (features [h d/H, (h+1) d/H)), a_t = softmax over p's tuples of
 *                       scale * q_t . k_t, Out[p][h] = sum_t a_t v_t[h]; lse[p][h] = log sum_t exp. */
#define RELNN_ATTN_SOFTMAX 0
#define RELNN_ATTN_PRODUCT 1
typedef struct relnn_attn_params {
    const void* d_q;         /* [n_h, d] (device, 16-byte aligned)                                 */
    const void* d_k;         /* [n_h, d]                                                           */
    const void* d_v;         /* [n_h, d_val]                                                       */
    relnn_float_t dtype;     /* of q, k and v                                                      */
    int32_t d;               /* 32, 64, 128 or 256                                                 */
    int32_t d_val;           /* width of v; = d                                                    */
    int32_t n_heads;         /* softmax: a power of two <= 32 (ignored by the product head)        */
    float scale;             /* softmax: multiplies q . k (e.g. 1 / sqrt(d / n_heads))             */
    int32_t mode;            /* RELNN_ATTN_SOFTMAX or RELNN_ATTN_PRODUCT                           */
} relnn_attn_params;

/* async. d_out [n_out, d] f32 (rows in relnn_plan_out_keys order, 16-byte aligned) and, for the
 * softmax head, d_lse [n_out, n_heads] f32 (may be NULL when no backward follows). Deterministic.
 * Errors: EINVAL (plan or shape outside the above). */
relnn_status relnn_attention_forward(relnn_plan_t p, const relnn_attn_params* prm, float* d_out, float* d_lse,
                                     void* stream);
/* async. Gradients of sum(d_dout * Out) for the forward's inputs: d_dq, d_dk, d_dv [n_h, d] f32 are
 * OVERWRITTEN (each may be NULL to skip); the softmax head needs that forward's d_out and d_lse.
 * Contributions are added with f32 atomics (run order may vary in the last bits). */
relnn_status relnn_attention_backward(relnn_plan_t p, const relnn_attn_params* prm, const float* d_fwd_out,
                                      const float* d_lse, const float* d_dout, float* d_dq, float* d_dk, float* d_dv,
                                      void* stream);

/* Releases the plan's device memory (waits for the device first). */
relnn_status relnn_plan_destroy(relnn_plan_t p);
/* Releases the plan without waiting: its device memory is freed in the order of `stream`, after
 * the work already queued there. Every call that used the plan must have been issued on that
 * stream (or be complete); the handle is invalid on return. */
relnn_status relnn_plan_release(relnn_plan_t p, void* stream);

/* async. Loss relation of content arity 0 (paper Sec. 3.2 fit statement; Sec. 3.6 loss rule):
 *     L(; mean((z_p - z_t)^2)) :- Pred(g; z_p), Target(g; z_t)
 * Pred and Target are embedded relations with unique keys sorted ascending (d_pred_keys [n_pred],
 * d_target_keys [n_target], type kt) and f32 rows of `width`. The join pairs rows with equal keys;
 * *d_loss (device f32) receives the mean of the squared differences over every cell of the joined
 * pairs (0 if none join), and d_grad (may be NULL) [n_pred, width] the gradient with respect to
 * d_pred (zero rows for predictions that join no target). Intended for small readout relations. */
relnn_status relnn_mse_loss(const float* d_pred, const void* d_pred_keys, int64_t n_pred, const float* d_target,
                            const void* d_target_keys, int64_t n_target, int32_t width, relnn_key_t kt,
                            float* d_loss, float* d_grad, void* stream);

/* async. Allocation-free FP32-form forward (the paper has no counterpart: this is a deployment aid).
 * Some callers cannot call cudaMalloc: a host that handed all device memory to another allocator at
 * start-up and works within that fixed budget, or a latency-critical loop that cannot afford the
 * device-wide synchronisation a cudaMalloc/cudaFree may cause. This entry point allocates nothing:
 * its scratch (the transposed W and the tile-boundary partial sums) is one fixed 4 MiB device array
 * inside the library, which every GPU that loads the library keeps until the process exits.
 * Inputs are the join output already grouped by output row (e.g. the grouping of relnn_rule_plan, or
 * the caller's own): for m matched tuples, d_hs / d_hd = src / dst H rows and d_seg = output row, with
 * d_seg non-decreasing; z f32 [n_h, d]; W f32 [d_out, 2d]; b f32 [d_out] (may be NULL). d_out_z
 * [n_out, d_out] receives, for every output row present in d_seg, the SUM over its tuples of
 * act(Concat(z[hs], z[hd]) W^T + b); rows absent from d_seg are not written.
 * Limits: d_out <= 256, 2d <= 1024, and (2d + 2 ceil(m/32)) * d_out * 4 bytes <= 4 MiB; larger calls
 * return RELNN_ENOSPC before any device work. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and must come before any stream capture. All calls share the one
 * array and nothing in it needs to start at zero (each call writes every slot it reads), but calls
 * that overlap on the device race on it: issue them on one stream or otherwise serialise them. */
relnn_status relnn_rule_forward_noalloc(const float* d_z, int32_t d, const int32_t* d_hs, const int32_t* d_hd,
                                        const int32_t* d_seg, int64_t m, const float* d_W, const float* d_b,
                                        int32_t d_out, relnn_act_t act, float* d_out_z, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Serving: a stream of independent rule queries evaluated with one shared Linear (the `?pred`
 * statement of paper Sec. 3.3 issued by many clients against a fitted rule). Queries of uneven
 * sizes are admitted by device memory and batched: the admitted queries' relations are placed in
 * disjoint key ranges of one batch, which is planned and evaluated by one fused persistent launch;
 * several batches run concurrently on separate streams while new queries keep arriving.
 * ------------------------------------------------------------------------------------------- */
typedef struct relnn_server_cfg {
    int32_t d;                  /* width of every query's H.z                                       */
    int32_t d_out;              /* width of the output embeddings                                   */
    const void* d_W;            /* shared Linear [d_out, 2d] (device, caller-owned, must outlive the server) */
    relnn_float_t w_dtype;
    const float* d_b;           /* shared bias [d_out] or NULL                                      */
    relnn_act_t act;
    uint32_t flags;             /* rule flags (RELNN_FLAG_BF16, RELNN_FLAG_KAHAN)                   */
    relnn_float_t z_dtype;      /* dtype of every query's H.z                                       */
    int32_t max_queue;          /* queries waiting or running; submit returns EAGAIN beyond it      */
    int64_t mem_budget_bytes;   /* device bytes batches may hold at once (0: 80% of free memory)    */
    int64_t max_batch_tuples;   /* E tuples per batch (a larger single query runs alone)            */
    int32_t max_batch_queries;  /* queries per batch                                                */
    int64_t tile128_below;      /* batches with fewer E tuples use 128-tuple tiles (autotuned)       */
    int32_t n_workers;          /* batches in flight at once (one stream and host thread each)       */
} relnn_server_cfg;

typedef struct relnn_query {
    const void* d_h_ids;        /* [n_h] int32 keys of H (device; valid until the query completes)  */
    int64_t n_h;
    const void* d_z;            /* [n_h, d] embeddings (server z_dtype)                             */
    const void* d_src;          /* [n_tuples] int32 E.src                                           */
    const void* d_dst;          /* [n_tuples] int32 E.dst                                           */
    int64_t n_tuples;
} relnn_query;

typedef struct relnn_result {
    int64_t n_out;              /* output rows                                                      */
    const int32_t* d_out_keys;  /* [n_out] sorted output keys (device, owned by the server)         */
    const float* d_out_z;       /* [n_out, d_out] f32 (device, owned by the server)                 */
    double latency_us;          /* submit -> results ready on the device                            */
    int32_t batch_queries;      /* queries that shared this query's batch                           */
} relnn_result;

/* Creates a server (starts its worker threads on the current device). Errors: EINVAL, ENOMEM. */
relnn_status relnn_server_create(const relnn_server_cfg* cfg, relnn_server_t* out);
/* Queues a query; *ticket identifies it. EAGAIN: queue full (retry later); ENOMEM: the query can
 * never fit the memory budget; EINVAL: bad query. Never blocks on the device. */
relnn_status relnn_serve_submit(relnn_server_t s, const relnn_query* q, uint64_t* ticket);
/* Waits up to timeout_us (0 = just check) for a ticket. OK: *res filled (buffers stay valid until
 * relnn_serve_release); EAGAIN: still pending (timeout 0); ETIMEDOUT: pending after the wait;
 * EINVAL: unknown ticket; EDEVICE / ECUDA: the query's batch failed. */
relnn_status relnn_serve_poll(relnn_server_t s, uint64_t ticket, relnn_result* res, uint32_t timeout_us);
/* Frees a completed ticket's result buffers. */
relnn_status relnn_serve_release(relnn_server_t s, uint64_t ticket);
/* Stops accepting queries, finishes the queued ones, joins the workers and frees everything. */
relnn_status relnn_server_destroy(relnn_server_t s);

/* ---------------------------------------------------------------------------------------------
 * Cyclic self-join (paper Sec. 5, DHN: a triangle homomorphism as a cyclic join over an edge
 * relation, the per-position transformations Mu applied to the node embeddings beforehand):
 *     Out(n; sum(a_n * b_v * c_w)) :- E(n, v), E(v, w), E(w, n), H(n; a), H(v; b), H(w; c)
 * with element-wise products and bag semantics (every E row is a tuple, every H row of a key
 * matches; edges with a key outside H are dropped). Output keys: the n with at least one match,
 * ascending. The plan intersects sorted adjacency lists per edge (a worst-case-optimal join).
 * ------------------------------------------------------------------------------------------- */
typedef struct relnn_tri_desc {
    relnn_key_t key_type;   /* type of H.id, E.src, E.dst                                           */
    const void* d_h_ids;    /* [n_h] (device)                                                       */
    int64_t n_h;
    const void* d_src;      /* [n_edges] E.src = n of E(n, v) (device)                              */
    const void* d_dst;      /* [n_edges] E.dst                                                      */
    int64_t n_edges;        /* < 2^31                                                               */
} relnn_tri_desc;

/* sync. Builds the cached match records (n, v, w, multiplicity) grouped by n. Errors: EINVAL,
 * ENOMEM, ENOTSUP (2^31 records or more), EDEVICE (a multiplicity above 2^31). */
relnn_status relnn_triangle_plan(const relnn_tri_desc* desc, void* stream, relnn_tri_t* out);
/* Output rows, match records (distinct (n, v, w)) and the edges kept by the join with H. */
relnn_status relnn_triangle_info(relnn_tri_t t, int64_t* n_out, int64_t* n_records, int64_t* n_edges_kept);
/* async. The output keys [n_out] (plan key type). */
relnn_status relnn_triangle_out_keys(relnn_tri_t t, void* d_out_keys, void* stream);
/* async. d_a, d_b, d_c [n_h, d] rows aligned with H (dtype f32 or bf16; d in {32, 64, 128, 256});
 * d_out [n_out, d] f32 (16-byte aligned), fully overwritten. Deterministic. */
relnn_status relnn_triangle_forward(relnn_tri_t t, const void* d_a, const void* d_b, const void* d_c,
                                    relnn_float_t dtype, int32_t d, float* d_out, void* stream);
/* async. Gradients of sum(d_dout * Out): d_da, d_db, d_dc [n_h, d] f32 OVERWRITTEN (each may be
 * NULL). Contributions are added with f32 atomics. */
relnn_status relnn_triangle_backward(relnn_tri_t t, const void* d_a, const void* d_b, const void* d_c,
                                     relnn_float_t dtype, int32_t d, const float* d_dout, float* d_da,
                                     float* d_db, float* d_dc, void* stream);
/* Frees the plan (waits for the device first). */
relnn_status relnn_triangle_destroy(relnn_tri_t t);

/* ---------------------------------------------------------------------------------------------
 * Streaming a relation larger than device memory (paper Sec. 6, future work on scaling for memory:
 * streaming the data from the database to the GPU in mini-batches). E (src, dst and the optional
 * per-tuple embedding r) stays in HOST memory; H (ids, z) is device-resident. A forward or backward
 * walks E in chunks: the next chunk's columns are copied while the current one is planned (join
 * against the shared H build side, grouping) and evaluated, and every chunk adds its rows into one
 * device accumulator indexed by H's distinct keys, so the result equals the unchunked rule's up to
 * the order of f32 additions (chunks are added in order: deterministic). Single branch, dst joined
 * (the output key space is H's), SUM or MEAN; no MAX, no PUSHDOWN.
 * ------------------------------------------------------------------------------------------- */
typedef struct relnn_stream_desc {
    relnn_key_t key_type;       /* type of H.id, E.src, E.dst                                       */
    const void* d_h_ids;        /* [n_h] keys of H (device; used by relnn_stream_create only)      */
    int64_t n_h;
    int32_t d;                  /* width of H.z                                                     */
    int32_t d_out;              /* output width (ignored with RELNN_FLAG_IDENTITY)                  */
    relnn_act_t act;
    uint32_t flags;             /* RELNN_FLAG_BF16, KAHAN, IDENTITY, NO_CONCAT_DST, MEAN, TILE128   */
    const void* h_src;          /* [n_tuples] keys of E.src (HOST; pinned memory overlaps copies)   */
    const void* h_dst;          /* [n_tuples] keys of E.dst (HOST); both must outlive the stream    */
    int64_t n_tuples;           /* any size (chunks hold < 2^31 tuples each)                        */
    int32_t d_r;                /* width of the per-tuple embedding r (0 = none)                    */
    int32_t n_filters;          /* selection predicates (as relnn_branch_desc)                      */
    const relnn_filter* filters;
    int64_t chunk_tuples;       /* E rows per chunk; 0: from mem_budget_bytes                       */
    int64_t mem_budget_bytes;   /* device bytes the chunk pipeline may hold; 0: a quarter of free   */
} relnn_stream_desc;

/* sync. Builds the H side (join build over H.id) and the device accumulators ([U, d_out] f32 per
 * role, U = distinct keys of H). Errors: EINVAL (unsupported flags / shapes), ENOMEM. */
relnn_status relnn_stream_create(const relnn_stream_desc* desc, void* stream, relnn_stream_t* out);
/* Distinct keys of H (the output capacity a forward needs), tuples per chunk and chunks per pass. */
relnn_status relnn_stream_info(relnn_stream_t s, int64_t* max_out_rows, int64_t* chunk_tuples, int64_t* n_chunks);
/* sync. Forward over all of E: d_out_keys [max_out_rows] (may be NULL) and d_out_z
 * [max_out_rows, d_out] f32 receive the n_out (*h_n_out) output rows, keys ascending, as
 * relnn_rule_forward would for the whole E. prm holds z, W, b as for a rule (one branch); its r
 * entry, if any, is a HOST pointer [n_tuples, d_r] (streamed with the keys). */
relnn_status relnn_stream_forward(relnn_stream_t s, const relnn_rule_params* prm, void* d_out_keys, float* d_out_z,
                                  int64_t* h_n_out, void* stream);
/* sync. Backward of the last relnn_stream_forward for d_dout [n_out, d_out] f32 (rows as that
 * forward returned them): d_dW [d_out, d_in], d_db [d_out], d_dz [n_h, d] (device, OVERWRITTEN) and
 * h_dr [n_tuples, d_r] (HOST, overwritten; may be NULL), each may be NULL to skip. The chunks are
 * re-planned; a BF16 rule with ReLU re-runs each chunk's forward for its ReLU mask. */
relnn_status relnn_stream_backward(relnn_stream_t s, const relnn_rule_params* prm, const float* d_dout, float* d_dW,
                                   float* d_db, float* d_dz, float* h_dr, void* stream);
/* Frees the stream's device memory (waits for the device first). */
relnn_status relnn_stream_destroy(relnn_stream_t s);

/* ---------------------------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper; used to report roofline fractions).
 * ------------------------------------------------------------------------------------------- */
#define RELNN_PROF_FWD_TC 0      /* fused tcgen05 forward kernel                                   */
#define RELNN_PROF_FWD_FP32 1    /* FP32-form forward kernel                                       */
#define RELNN_PROF_FIXUP 2       /* tile-boundary fix-up of split segments                         */
#define RELNN_PROF_BWD_TC 3      /* tensor-core backward kernels                                   */
#define RELNN_PROF_BWD_FP32 4    /* FP32-form backward kernels                                     */
#define RELNN_PROF_PLAN 5        /* content track (whole relnn_rule_plan)                          */
#define RELNN_PROF_AGG_FWD 6     /* aggregate-first forward kernel (linear SUM rules)              */
#define RELNN_PROF_AGG_BWD 7     /* aggregate-first backward kernel (one launch per pass)          */
#define RELNN_PROF_AGG_SUM 8     /* aggregate-first gather-sum kernel (per-row sums of the src rows) */

/* Number of kernels this library has launched since it was loaded (host counter). */
uint64_t relnn_launch_count(void);
/* Turns CUDA-event timing of the kernels above on (1) or off (0). Events are recorded on the stream
 * each kernel is launched on; timing adds two event records per launch. */
relnn_status relnn_profile_enable(int32_t on);
/* sync (waits for the recorded events). Total device milliseconds and launch count of kernel `id`
 * accumulated since the last reset. */
relnn_status relnn_profile_read(int32_t id, double* total_ms, int64_t* launches);
relnn_status relnn_profile_reset(void);
/* Process-wide tuning knobs (no counterpart in the paper): choices of the kernels' host code that
 * change speed, never results beyond the order of f32 additions. Set by the autotuner or the
 * caller; thread-safe; a value outside the knob's range is rejected with EINVAL.
 *   RELNN_TUNE_SORT_BITS   widest digit of a radix-sort pass (4..11, default 8): the content track's
 *                          group sort takes ceil(key bits / this) passes of equal width; narrower
 *                          digits make longer runs per 4096-key tile in the scatter
 *   RELNN_TUNE_AGG_ROWS    output rows per tile of the aggregate-first GEMM (0 = the largest that
 *                          fits, or 32 / 64 / 128)
 *   RELNN_TUNE_AGG_STAGES  shared-memory pipeline stages of that GEMM (0 = as many as fit, at most
 *                          4; or 2..4, capped at what fits)
 *   RELNN_TUNE_AGG_EPI     epilogue warps of that GEMM: 4 (one per TMEM lane quarter) or 8 (two per
 *                          quarter, each on every other 32-row chunk); 0 = 8
 *   RELNN_TUNE_KAHAN_MIN   with RELNN_FLAG_KAHAN, the aggregate-first form's gather-sum compensates
 *                          inside a chunk of at most 32 tuples only for rows of at least this many
 *                          tuples (and the chunks of cut rows); above 32 (default 33) no chunk is
 *                          compensated inside, and the compensation is where a row's error grows:
 *                          the fix-up adding the chunk partials of rows longer than 32 tuples
 *   RELNN_TUNE_GROUP_SORT  group-by of a single-branch plan over unique H keys: 0 = the stable radix
 *                          sort (groups in E order; default); 1 = by counting (a count per group key
 *                          during the emission, one scan, an atomic scatter, each group then ordered
 *                          by src H row), falling back to the radix sort when a tuple does not match
 *                          or a group holds more than 4096 tuples
 *   RELNN_TUNE_AGG_FUSE    aggregate-first forward of a unique-key plan: 0 = two kernels (the
 *                          gather-sum writes each row's bf16 pair to memory, the GEMM reads it back;
 *                          default); 1 / 2 = one kernel whose producer warps write the pairs straight
 *                          into the GEMM's shared-memory stages (4 epilogue + 8 producer warps, or
 *                          8 + 4); plans with Kahan summation inside chunks stay with two kernels   */
#define RELNN_TUNE_SORT_BITS 0
#define RELNN_TUNE_AGG_ROWS 1
#define RELNN_TUNE_AGG_STAGES 2
#define RELNN_TUNE_AGG_EPI 3
#define RELNN_TUNE_KAHAN_MIN 4
#define RELNN_TUNE_GROUP_SORT 5
#define RELNN_TUNE_AGG_FUSE 6
relnn_status relnn_tune_set(int32_t knob, int64_t value);
relnn_status relnn_tune_get(int32_t knob, int64_t* value);

/* sync. Test of the bounded waits (no counterpart in the paper): one CTA waits, with the bounded
 * mbarrier wait every tensor-core kernel of the library uses, on a barrier that nothing arrives at,
 * under a budget of budget_us microseconds (0 < budget_us <= 1e6) instead of the kernels' 2 s. The
 * wait gives up, the kernel returns and RELNN_EDEVICE is returned with relnn_last_device_error() ==
 * RELNN_DEV_TIMEOUT after about budget_us; the device and the context stay usable. Errors: EINVAL,
 * ECUDA. */
relnn_status relnn_test_wait_timeout(int32_t budget_us, void* stream);

/* sync. FP32 CUDA-core throughput probe: one launch of 2 x SMs blocks of 1024 threads, each thread
 * running 8 independent FMA chains for `iters` steps, timed by CUDA events on `stream` after one
 * warm-up launch. *tflops = 16 x iters x threads / time (FMA = 2 FLOP); *ms (may be NULL) = the
 * launch's time. The denominator of the FP32 form's roofline. Errors: EINVAL, ECUDA. */
relnn_status relnn_peak_fma_f32(int32_t iters, double* tflops, double* ms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RELNN_H */
