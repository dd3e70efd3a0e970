// Rule plan: the cached content track of a join rule (paper Sec. 3.1 compiled as
// U_{SUM,dst}(T_tau(E |><| H |><| H)); Sec. 4.2 join row indices and group indices).
//
// Per branch, the matched (join-output) tuples are stored once, sorted by output key, as
//   hs[m]   int32  H row of the src side
//   hd[m]   int32  H row of the dst side (-1 without a dst join)
//   er[m]   int32  E row (index into the per-tuple embedding r)
//   seg[m]  int32  output row of the tuple (position of its dst key among the output keys)
// Within one output key the tuples are ordered by dst H row, then E row, then src H row, so runs of
// equal hd are contiguous (used by the backward's scatter to z_dst). er is kept only for branches
// with a per-tuple embedding r (d_r > 0). For the backward's scatter to z_src the same tuples are
// also kept in src order (built on the first backward, stable):
//   src_perm[m] int32  position in the order above of the k-th tuple in src order
//   hs_src[m]   int32  its src H row (non-decreasing)
//   seg_src[m]  int32  its output row
#pragma once

#include <memory>
#include <vector>

#include "join.cuh"

namespace relnn {

// Virtual rows of an ordered tuple list for the aggregate-first kernels (agg.cu): the tuples of
// one destination row (a run of equal keys) cut into chunks of at most a fixed number of tuples.
//   vr[v]    int4 {first tuple, tuples, destination row, partial slot (-1: the row is one chunk)}
//   fix1/2   fix-up jobs of rows cut into several chunks (int4 {row, first slot, count, level-2 slot
//            or -1}), level 2 only for rows with more chunks than one fix-up block adds
//   cnt[r]   int32 tuples of row r (lists whose keys ascend over rows 0..R-1)
//   d1[v]    int32 dst H row of virtual row v (forward lists of plans with unique H keys), or -1
// Built once per list and cached (nv < 0: not built yet).
struct VRows {
    int64_t nv = -1, n_parts = 0, n_l2 = 0, n_fix1 = 0, n_fix2 = 0;
    DevBuf vr, fix1, fix2, cnt, d1;
    bool has_d1 = false;
};

struct BranchPlan {
    int64_t n_tuples = 0;
    int64_t m = 0;  // matched tuples
    int32_t d_r = 0;
    DevBuf hs, hd, er, seg;
    DevBuf src_perm, hs_src, seg_src;
    DevBuf relu_mask;  // uint32 [m][ceil(d_out/32)] when RELNN_FLAG_RELU_MASK
    // aggregate-first evaluation: output rows (forward), H rows in src order and runs of equal dst H
    // rows (backward)
    VRows vr_out, vr_src, vr_dst;
};

// Internal plan flag (above the public RELNN_FLAG_* bits): every tuple is its own output row (the
// identity plan of a dense per-row product), so the forward stores rows without a SUM walk.
constexpr uint32_t kPlanDense = 1u << 30;

struct Plan {
    int kt = RELNN_I32;
    uint32_t flags = 0;
    int act = RELNN_ACT_NONE;
    int d = 0, d_out = 0, d_in = 0;
    bool join_dst = true, concat_dst = true, identity = false, bf16 = false, kahan = false;
    int64_t n_h = 0;
    JoinTable H;
    int64_t n_out = 0;
    DevBuf out_keys;  // int64 [n_out] (converted to the key type on copy-out)
    std::vector<BranchPlan> br;
    DevBuf status;    // device status word
    // forward/backward workspace (grown on demand, reused across calls)
    DevBuf carry;     // f32 [tiles][2][d_out] partial sums of segments cut by tile boundaries
    DevBuf wpack;     // bf16 packed/padded weights for the tensor-core kernels
    DevBuf scratch;   // misc per-call scratch
    DevBuf zbf;       // bf16 copy of an f32 H embedding for the tensor-core kernels
    // the caller's promise (relnn_plan_set_z_version): an f32 H.z passed at the same address with the
    // same nonzero version is unchanged, so zbf (converted from zbf_src at zbf_version) is reused
    uint64_t z_version = 0, zbf_version = 0;
    const void* zbf_src = nullptr;
    DevBuf doutbf;    // bf16 copy of the output gradient for the backward's src pass
    DevBuf fixjobs;   // long segments handed from the fix-up to its block-per-segment pass
    DevBuf vpart;     // aggregate-first: f32 partial rows of chunks (and their level-2 sums)
    DevBuf sbuf;      // aggregate-first: per virtual row the bf16 pair of its src sums
    // transformation push-down (RELNN_FLAG_PUSHDOWN): the identity plan of the per-H-row products,
    // the products P = Z W_src^T and Q = Z W_dst^T + b, and one column block of W
    std::unique_ptr<Plan> pd;
    DevBuf pdP, pdQ, pdW;
    // MEAN aggregator (RELNN_FLAG_MEAN): 1 / matched tuples per output row, and the scaled dOut
    DevBuf inv_cnt, mean_dout;
    // MAX aggregator (RELNN_FLAG_MAX): int32 [n_out][d_out] plan position of each maximum's first
    // tuple (-1: no gradient), the positions of the boundary partials (twin of carry), and the
    // winner mask the backward reads in place of a ReLU mask (uint32 [m][mask_words])
    DevBuf max_arg, carry_pos, win_mask;
    bool max_ready = false;  // a forward has filled max_arg
    // Chunk of a streamed relation: the H build side is the stream's (Hx); with dense_out the
    // output rows are H's distinct-key indices (n_out = U, seg = distinct index, the present flags
    // go to present_ext, iota_ext is the identity map 0..U); with acc_out the forward adds into its
    // output instead of overwriting it
    const JoinTable* Hx = nullptr;
    bool dense_out = false, acc_out = false;
    int32_t* present_ext = nullptr;
    const int32_t* iota_ext = nullptr;
    const JoinTable& Ht() const { return Hx ? *Hx : H; }
    int64_t total_matched() const {
        int64_t s = 0;
        for (auto& b : br) s += b.m;
        return s;
    }
    // Frees every buffer of the plan in the order of stream s when the plan is destroyed (instead of
    // a synchronising cudaFree), for plans whose work all ran on s.
    void retire_on(cudaStream_t s) {
        DevBuf* bufs[] = {&H.rows_sorted, &H.run_start, &H.uid_of_pos, &H.ukeys, &H.slot_keys, &H.slot_vals,
                          &H.status, &out_keys, &status, &carry, &wpack, &scratch, &zbf, &doutbf, &fixjobs, &vpart, &sbuf, &pdP, &pdQ, &pdW, &inv_cnt, &mean_dout,
                          &max_arg, &carry_pos, &win_mask};
        for (DevBuf* b : bufs) {
            b->ordered = true;
            b->st = s;
        }
        if (pd) pd->retire_on(s);
        for (auto& b : br) {
            DevBuf* bb[] = {&b.hs, &b.hd, &b.er, &b.seg, &b.src_perm, &b.hs_src, &b.seg_src, &b.relu_mask,
                            &b.vr_out.vr, &b.vr_out.fix1, &b.vr_out.fix2, &b.vr_out.cnt, &b.vr_out.d1, &b.vr_src.vr, &b.vr_src.fix1,
                            &b.vr_src.fix2, &b.vr_src.cnt, &b.vr_dst.vr, &b.vr_dst.fix1, &b.vr_dst.fix2,
                            &b.vr_dst.cnt};
            for (DevBuf* x : bb) {
                x->ordered = true;
                x->st = s;
            }
        }
    }
};

relnn_status build_plan(Plan& p, const relnn_rule_desc* desc, cudaStream_t st);

// Builds b.src_perm / hs_src / seg_src once (no-op afterwards); synchronises st when it builds.
relnn_status ensure_src_order(const Plan& p, BranchPlan& b, cudaStream_t st);

}  // namespace relnn

struct relnn_plan_s {
    relnn::Plan p;
};
