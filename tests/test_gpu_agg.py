"""GPU parity of the aggregate-first evaluation of linear SUM rules (the BF16 form's default for rules
without an activation: each output row's Concat rows are summed first and the Linear is applied once
per row, since SUM commutes with a linear map, paper Sec. 2.2 and the hybrid rewrites of Sec. 6).

Bars as for the BF16 form: join output and key sets bit-exact, <= 2e-2 relative Frobenius error
against the FP64 oracle on the original inputs, and <= 1e-4 against the oracle fed the same
bf16-rounded operands (the per-row sums are kept as a bf16 pair, about 16 significant bits). The
per-tuple form (RELNN_FLAG_PER_TUPLE) computes the same rule and is compared as well. Shapes cover
virtual rows cut into chunks (heavy rows), the two-level fix-up (rows of more than 256 chunks), the
backward's src-order hubs, unions, MEAN, Kahan, every supported width and the fallbacks."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import OBr, bf16_round, oracle_rule, rel_frob, run_rule, to_dev

pytestmark = pytest.mark.gpu

BF16_TOL = 2e-2
SAME_INPUT_TOL = 1e-4


def _fwd(rel, flags=0, z_dtype=torch.bfloat16, **kw):
    keys, out, plan, t = run_rule(rel, flags=flags | R.FLAG_BF16, z_dtype=z_dtype, **kw)
    ok, oo, sizes = oracle_rule(rel)
    assert np.array_equal(keys, ok)
    assert plan.matched == sizes
    assert rel_frob(out, oo) <= BF16_TOL
    _, oo_r, _ = oracle_rule(rel, round_z=True, round_w=True)
    err = rel_frob(out, oo_r)
    assert err <= SAME_INPUT_TOL, err
    return keys, out, plan, t


@pytest.mark.parametrize("d,d_out", [(128, 128), (64, 64), (32, 96), (256, 64), (8, 16), (16, 256), (64, 200)])
def test_forward_widths(gpu, d, d_out):
    rel = W.make_rule(101, 20_011, 1500, d, d_out, np.int32, src_dist="zipf", src_s=1.1)
    _fwd(rel)


@pytest.mark.parametrize("d,d_out", [(8, 16), (16, 64), (32, 32)])
def test_forward_narrow_rows_padding_reads_zero(gpu, d, d_out):
    """Rows narrower than a 64-column K block: the GEMM's dst block is padded with zeros it writes
    itself (the gather-sum before it leaves index words in shared memory, and with more than 2^15 H
    rows some of them are NaN patterns as bf16; a stale NaN times a zero weight would be NaN)."""
    rel = W.make_rule(107, 200_000, 70_000, d, d_out, np.int32, src_dist="zipf", src_s=1.1)
    keys, out, _, _ = _fwd(rel)
    assert np.isfinite(out).all()


@pytest.mark.parametrize("d", [16, 64, 128, 256])
def test_forward_table_alignment_same_sums(gpu, d):
    """Rows of 64 .. 256 elements in a 32-byte aligned bf16 table take the gather-sum with 32-byte lane
    chunks, a table 16 bytes off that boundary (and rows of 16) the one with 16-byte chunks: the same
    sums in the same order, so the outputs are equal bit for bit, and both meet the oracle bars."""
    rel = W.make_rule(108, 60_000, 5000, d, 64, np.int32, src_dist="zipf", src_s=1.2)
    keys, out, plan, t = _fwd(rel)
    z = t["z"]
    assert z.data_ptr() % 32 == 0
    buf = torch.empty(z.numel() + 8, dtype=z.dtype, device=z.device)
    z_off = buf[8:].view(z.shape)
    z_off.copy_(z)
    assert z_off.data_ptr() % 32 == 16
    out2 = plan.forward(z_off, t["W"], t["b"]).cpu().numpy()
    plan.check()
    assert np.array_equal(out, out2)
    # the backward's src pass gathers dOut rows from the plan's own (aligned) copy; both tables give
    # the same gradients
    dout = torch.randn(out.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    g1 = plan.backward(dout, z, t["W"], t["b"])
    g2 = plan.backward(dout, z_off, t["W"], t["b"])
    assert torch.equal(g1[0][0], g2[0][0])
    if d % 32 == 0:  # the aggregate-first backward: no atomics, the same dz bit for bit
        assert torch.equal(g1[2], g2[2])
    else:  # d = 16 takes the per-tuple backward, which adds dz rows by atomics (order varies)
        assert rel_frob(g2[2].cpu().numpy(), g1[2].cpu().double().numpy()) <= 1e-6


def test_forward_same_as_per_tuple(gpu):
    rel = W.make_rule(102, 50_000, 4000, 128, 128, np.int64, src_dist="zipf", src_s=1.1)
    keys, out, _, _ = _fwd(rel)
    keys2, out2, _, _ = run_rule(rel, flags=R.FLAG_BF16 | R.FLAG_PER_TUPLE, z_dtype=torch.bfloat16)
    assert np.array_equal(keys, keys2)
    assert rel_frob(out, out2.astype(np.float64)) <= SAME_INPUT_TOL


@pytest.mark.parametrize("kahan", [False, True])
def test_forward_heavy_rows_two_level_fixup(gpu, kahan):
    """Zipf(2.0) dst over 200 keys: the largest row holds most of the 40k tuples, i.e. more than 256
    chunks of 32, so its chunk partials go through both fix-up levels."""
    rel = W.make_rule(103, 40_000, 200, 64, 64, np.int32, dst_dist="zipf", dst_s=2.0)
    _fwd(rel, flags=R.FLAG_KAHAN if kahan else 0)


def test_forward_f32_table_and_duplicate_keys(gpu):
    """f32 z (the plan's bf16 copy is gathered) and duplicate H keys (a row's tuples name several
    dst H rows: the dst part sums distinct rows with their multiplicities)."""
    rel = W.make_rule(104, 8000, 600, 64, 64, np.int64, dup_frac=0.3, missing_frac=0.1, sparse_keys=True)
    _fwd(rel, z_dtype=torch.float32)


def test_forward_union_without_edge_embedding(gpu):
    rel = W.make_rule(105, 0, 3000, 64, 96, np.int32, dst_dist="zipf", dst_s=1.0,
                      branch_tuples=[20_000, 10_000, 5000])
    _fwd(rel)


def test_forward_no_concat_dst_and_readout_shape(gpu):
    rel = W.make_rule(106, 10_000, 900, 64, 64, np.int32)
    rel.branches[0].W = np.ascontiguousarray(rel.branches[0].W[:, :64])  # Concat = z_src only
    keys, out, plan, _ = run_rule(rel, flags=R.FLAG_BF16 | R.FLAG_NO_CONCAT_DST, z_dtype=torch.bfloat16)
    ok, oo, _ = oracle_rule(rel, round_z=True, round_w=True, concat_dst=False)
    assert np.array_equal(keys, ok)
    assert rel_frob(out, oo) <= SAME_INPUT_TOL


def test_forward_mean(gpu):
    rel = W.make_rule(107, 30_000, 2500, 64, 64, np.int32, src_dist="zipf", src_s=1.2, dst_dist="zipf", dst_s=1.3)
    keys, out, plan, _ = run_rule(rel, flags=R.FLAG_BF16 | R.FLAG_MEAN, z_dtype=torch.bfloat16)
    brs = [OBr(b.src, b.dst, bf16_round(b.W), b.b, None) for b in rel.branches]
    ok, oo, _ = O.rule_forward(rel.h_ids, bf16_round(rel.z), brs, agg="mean")
    assert np.array_equal(keys, ok)
    assert rel_frob(out, oo) <= SAME_INPUT_TOL


def test_forward_unaligned_output_takes_per_tuple_form(gpu):
    """An output pointer that is not 16-byte aligned runs the per-tuple form (same result)."""
    rel = W.make_rule(108, 6000, 500, 64, 64, np.int32)
    br = rel.branches[0]
    plan = R.RulePlan(to_dev(rel.h_ids), [(to_dev(br.src), to_dev(br.dst))], 64, 64, flags=R.FLAG_BF16)
    buf = torch.empty(plan.n_out * 64 + 1, dtype=torch.float32, device="cuda")
    out = buf[1:].view(plan.n_out, 64)
    plan.forward(to_dev(rel.z, torch.bfloat16), [to_dev(br.W)], [to_dev(br.b)], out=out)
    torch.cuda.synchronize()
    plan.check()
    _, oo, _ = oracle_rule(rel, round_z=True, round_w=True)
    assert rel_frob(out.cpu().numpy(), oo) <= SAME_INPUT_TOL


def test_empty_branch_in_union(gpu):
    """A union whose first branch matches nothing: the first launch still writes every output row."""
    rel = W.make_rule(109, 0, 800, 64, 64, np.int32, branch_tuples=[3000, 4000])
    b0 = rel.branches[0]
    b0.src = np.full_like(b0.src, 10 ** 6)  # no H key matches
    _fwd(rel)


# ------------------------------------------------------------------------------ backward
def _bwd(rel, flags=0, z_dtype=torch.bfloat16, seed=3):
    keys, out, plan, t = run_rule(rel, flags=flags | R.FLAG_BF16, z_dtype=z_dtype)
    dout = np.random.default_rng(seed).standard_normal(out.shape).astype(np.float32)
    dW, db, dz, _ = plan.backward(to_dev(dout), t["z"], t["W"], t["b"], t["r"])
    torch.cuda.synchronize()
    plan.check()
    agg = "mean" if flags & R.FLAG_MEAN else "sum"
    brs = [OBr(b.src, b.dst, bf16_round(b.W), b.b, None) for b in rel.branches]
    oW, ob, oz, _ = O.rule_backward(rel.h_ids, bf16_round(rel.z), brs, keys, dout, act=rel.act, agg=agg)
    return (dW, db, dz), (oW, ob, oz), (plan, t, dout)


@pytest.mark.parametrize("d,d_out,src_s", [(128, 128, 1.1), (64, 64, 1.2), (32, 8, 1.1), (256, 128, 1.1), (64, 256, 1.3)])
def test_backward_matches_oracle(gpu, d, d_out, src_s):
    rel = W.make_rule(111, 30_011, 3000, d, d_out, np.int32, src_dist="zipf", src_s=src_s)
    (dW, db, dz), (oW, ob, oz), _ = _bwd(rel)
    # dOut is gathered as bf16 (the per-tuple form's dY rounding); the sums are a bf16 pair
    assert rel_frob(dW[0].cpu().numpy(), oW[0]) <= 5e-3
    assert rel_frob(db[0].cpu().numpy(), ob[0]) <= 5e-3
    assert rel_frob(dz.cpu().numpy(), oz) <= 5e-3


def test_backward_same_as_per_tuple(gpu):
    rel = W.make_rule(112, 40_000, 3000, 128, 128, np.int64, src_dist="zipf", src_s=1.1)
    (dW, db, dz), _, (plan, t, dout) = _bwd(rel)
    keys, out, plan2, t2 = run_rule(rel, flags=R.FLAG_BF16 | R.FLAG_PER_TUPLE, z_dtype=torch.bfloat16)
    dW2, db2, dz2, _ = plan2.backward(to_dev(dout), t2["z"], t2["W"], t2["b"], t2["r"])
    torch.cuda.synchronize()
    assert rel_frob(dW[0].cpu().numpy(), dW2[0].cpu().numpy().astype(np.float64)) <= 2e-2
    assert rel_frob(db[0].cpu().numpy(), db2[0].cpu().numpy().astype(np.float64)) <= 1e-4
    assert rel_frob(dz.cpu().numpy(), dz2.cpu().numpy().astype(np.float64)) <= 2e-2


def test_backward_src_hub_two_level_fixup(gpu):
    """Zipf(2.5) src over 2000 keys: the top src row holds most of the 60k tuples (more than 256
    chunks), so the src pass's dz row of that hub goes through both fix-up levels."""
    rel = W.make_rule(113, 60_000, 2000, 64, 64, np.int32, src_dist="zipf", src_s=2.5)
    (dW, db, dz), (oW, ob, oz), _ = _bwd(rel)
    assert rel_frob(dW[0].cpu().numpy(), oW[0]) <= 5e-3
    assert rel_frob(dz.cpu().numpy(), oz) <= 5e-3


@pytest.mark.parametrize("kind", ["union", "mean", "kahan", "dup_keys"])
def test_backward_variants(gpu, kind):
    flags = 0
    if kind == "union":
        rel = W.make_rule(114, 0, 2000, 64, 64, np.int32, dst_dist="zipf", dst_s=1.0, branch_tuples=[9000, 5000, 2500])
    elif kind == "mean":
        rel = W.make_rule(115, 20_000, 1500, 64, 64, np.int32, dst_dist="zipf", dst_s=1.3)
        flags = R.FLAG_MEAN
    elif kind == "kahan":
        rel = W.make_rule(116, 20_000, 1500, 64, 64, np.int32, src_dist="zipf", src_s=1.5)
        flags = R.FLAG_KAHAN
    else:
        rel = W.make_rule(117, 8000, 600, 64, 64, np.int64, dup_frac=0.3, missing_frac=0.1, sparse_keys=True)
    (dW, db, dz), (oW, ob, oz), _ = _bwd(rel, flags=flags)
    for i in range(len(rel.branches)):
        assert rel_frob(dW[i].cpu().numpy(), oW[i]) <= 5e-3
        assert rel_frob(db[i].cpu().numpy(), ob[i]) <= 5e-3
    assert rel_frob(dz.cpu().numpy(), oz) <= 5e-3


def test_backward_repeat_is_deterministic(gpu):
    rel = W.make_rule(118, 30_000, 2000, 64, 64, np.int32, src_dist="zipf", src_s=1.4)
    (dW, db, dz), _, (plan, t, dout) = _bwd(rel)
    dW2, db2, dz2, _ = plan.backward(to_dev(dout), t["z"], t["W"], t["b"], t["r"])
    torch.cuda.synchronize()
    assert torch.equal(dW[0], dW2[0]) and torch.equal(db[0], db2[0]) and torch.equal(dz, dz2)


def test_forward_repeat_is_deterministic(gpu):
    rel = W.make_rule(119, 30_000, 200, 64, 64, np.int32, dst_dist="zipf", dst_s=2.0)
    keys, out, plan, t = run_rule(rel, flags=R.FLAG_BF16, z_dtype=torch.bfloat16)
    out2 = plan.forward(t["z"], t["W"], t["b"])
    torch.cuda.synchronize()
    assert np.array_equal(out, out2.cpu().numpy())


@pytest.mark.parametrize("d,d_out,src_s", [(64, 64, 1.2), (128, 128, 1.1), (32, 32, 1.5), (64, 256, 1.1)])
def test_relu_backward_aggregate_first(gpu, d, d_out, src_s):
    """A ReLU rule whose forward kept its mask: the backward sums the masked dOut rows per H row
    (src pass: each tuple's mask bits; dst pass: per-feature counts of active tuples, which also give
    db) and runs the same GEMMs as a linear rule. Compared with the FP64 oracle's gradient and with the
    per-tuple backward (RELNN_FLAG_PER_TUPLE) from the same mask."""
    rel = W.make_rule(120, 30_011, 3000, d, d_out, np.int32, src_dist="zipf", src_s=src_s, act="relu")
    flags = R.FLAG_BF16 | R.FLAG_RELU_MASK
    keys, out, plan, t = run_rule(rel, flags=flags, z_dtype=torch.bfloat16)
    dout = np.random.default_rng(9).standard_normal(out.shape).astype(np.float32)
    dW, db, dz, _ = plan.backward(to_dev(dout), t["z"], t["W"], t["b"], t["r"])
    torch.cuda.synchronize()
    plan.check()
    brs = [OBr(b.src, b.dst, bf16_round(b.W), b.b, None) for b in rel.branches]
    oW, ob, oz, _ = O.rule_backward(rel.h_ids, bf16_round(rel.z), brs, keys, dout, act=rel.act)
    # the GPU's ReLU decisions come from its bf16 forward; a few tuples near 0 may differ
    assert rel_frob(dW[0].cpu().numpy(), oW[0]) <= 2e-2
    assert rel_frob(db[0].cpu().numpy(), ob[0]) <= 2e-2
    assert rel_frob(dz.cpu().numpy(), oz) <= 2e-2
    keys2, out2, plan2, t2 = run_rule(rel, flags=flags | R.FLAG_PER_TUPLE, z_dtype=torch.bfloat16)
    dW2, db2, dz2, _ = plan2.backward(to_dev(dout), t2["z"], t2["W"], t2["b"], t2["r"])
    torch.cuda.synchronize()
    assert rel_frob(dW[0].cpu().numpy(), dW2[0].cpu().numpy().astype(np.float64)) <= 1e-2
    assert rel_frob(db[0].cpu().numpy(), db2[0].cpu().numpy().astype(np.float64)) <= 1e-4
    assert rel_frob(dz.cpu().numpy(), dz2.cpu().numpy().astype(np.float64)) <= 1e-2


def test_relu_backward_aggregate_first_is_deterministic(gpu):
    rel = W.make_rule(121, 20_000, 1500, 64, 64, np.int32, src_dist="zipf", src_s=1.3, act="relu")
    keys, out, plan, t = run_rule(rel, flags=R.FLAG_BF16 | R.FLAG_RELU_MASK, z_dtype=torch.bfloat16)
    dout = to_dev(np.random.default_rng(2).standard_normal(out.shape).astype(np.float32))
    g1 = plan.backward(dout, t["z"], t["W"], t["b"], t["r"])
    g2 = plan.backward(dout, t["z"], t["W"], t["b"], t["r"])
    torch.cuda.synchronize()
    assert torch.equal(g1[0][0], g2[0][0]) and torch.equal(g1[1][0], g2[1][0]) and torch.equal(g1[2], g2[2])


@pytest.mark.parametrize("fuse", [1, 2])
@pytest.mark.parametrize("case", ["w128", "w64_d96", "w32", "w256", "heavy", "union", "no_concat_dst", "f32"])
def test_fused_forward(gpu, fuse, case):
    """The fused aggregate-first forward (RELNN_TUNE_AGG_FUSE = 1 or 2: the GEMM's producer warps
    sum each row's tuples straight into the shared-memory stage) against the oracle, at the same bars
    as the two-kernel form, and against the two-kernel form itself."""
    saved = R.tune_get(R.TUNE_AGG_FUSE)
    try:
        if case == "w128":
            rel, kw = W.make_rule(131, 40_000, 3000, 128, 128, np.int64, src_dist="zipf", src_s=1.1), {}
        elif case == "w64_d96":
            rel, kw = W.make_rule(132, 20_011, 1500, 64, 96, np.int32), {}
        elif case == "w32":
            rel, kw = W.make_rule(133, 20_011, 1500, 32, 64, np.int32), {}
        elif case == "w256":
            rel, kw = W.make_rule(134, 10_000, 900, 256, 64, np.int32), {}
        elif case == "heavy":
            rel, kw = W.make_rule(135, 40_000, 200, 64, 64, np.int32, dst_dist="zipf", dst_s=2.0), {}
        elif case == "union":
            rel, kw = W.make_rule(136, 0, 3000, 64, 96, np.int32, dst_dist="zipf", dst_s=1.0,
                                  branch_tuples=[20_000, 10_000, 5000]), {}
        elif case == "no_concat_dst":
            rel = W.make_rule(137, 10_000, 900, 64, 64, np.int32)
            rel.branches[0].W = np.ascontiguousarray(rel.branches[0].W[:, :64])
            R.tune_set(R.TUNE_AGG_FUSE, fuse)
            keys, out, plan, _ = run_rule(rel, flags=R.FLAG_BF16 | R.FLAG_NO_CONCAT_DST, z_dtype=torch.bfloat16)
            ok, oo, _ = oracle_rule(rel, round_z=True, round_w=True, concat_dst=False)
            assert np.array_equal(keys, ok)
            assert rel_frob(out, oo) <= SAME_INPUT_TOL
            return
        else:
            rel, kw = W.make_rule(138, 8000, 600, 64, 64, np.int64, missing_frac=0.1, sparse_keys=True), \
                dict(z_dtype=torch.float32)
        R.tune_set(R.TUNE_AGG_FUSE, 0)
        _, out2, _, _ = run_rule(rel, flags=R.FLAG_BF16, **({"z_dtype": torch.bfloat16} | kw))
        R.tune_set(R.TUNE_AGG_FUSE, fuse)
        _, out, _, _ = _fwd(rel, **kw)
        assert rel_frob(out, out2.astype(np.float64)) <= 1e-5
    finally:
        R.tune_set(R.TUNE_AGG_FUSE, saved)


FP32_TOL = 1e-5


@pytest.mark.parametrize("case", ["c1", "d4", "d8_dout64", "d32_dout256", "hubs_kahan", "two_level", "union",
                                  "no_concat_dst", "mean", "dup_keys_falls_back", "f32_instances"])
def test_fp32_aggregate_first_forward(gpu, case):
    """The FP32 form's aggregate-first forward (f32 on CUDA cores: each output row's src rows summed
    first, the Linear applied once per row) against the FP64 oracle at the FP32 bar (1e-5) and
    against the per-tuple FP32 form (RELNN_FLAG_PER_TUPLE) on the same inputs; key sets and join
    sizes bit-exact. Covers every supported width, rows cut into chunks (hubs; more than 256 chunks:
    the two-level fix-up), Kahan, unions, no dst part, MEAN and a plan with duplicate H keys (which
    takes the per-tuple form)."""
    flags, kw = 0, {}
    if case == "c1":
        rel = W.config1(0)
    elif case == "d4":
        rel = W.make_rule(151, 30_011, 2000, 4, 8, np.int32, src_dist="zipf", src_s=1.1)
    elif case == "d8_dout64":
        rel = W.make_rule(152, 20_000, 1500, 8, 64, np.int64, sparse_keys=True, missing_frac=0.05)
    elif case == "d32_dout256":
        rel = W.make_rule(153, 10_000, 800, 32, 256, np.int32)
    elif case == "hubs_kahan":
        rel, flags = W.make_rule(154, 60_000, 3000, 16, 16, np.int32, dst_dist="zipf", dst_s=1.3), R.FLAG_KAHAN
    elif case == "two_level":
        rel = W.make_rule(155, 40_000, 200, 16, 32, np.int32, dst_dist="zipf", dst_s=2.0)
    elif case == "union":
        rel = W.make_rule(156, 0, 3000, 16, 16, np.int32, dst_dist="zipf", dst_s=1.0,
                          branch_tuples=[20_000, 10_000, 5000])
    elif case == "no_concat_dst":
        rel = W.make_rule(157, 10_000, 900, 16, 16, np.int32)
        rel.branches[0].W = np.ascontiguousarray(rel.branches[0].W[:, :16])
        flags, kw = R.FLAG_NO_CONCAT_DST, dict(concat_dst=False)
    elif case == "mean":
        rel, flags = W.make_rule(158, 20_000, 1500, 16, 16, np.int32, dst_dist="zipf", dst_s=1.2), R.FLAG_MEAN
    elif case == "dup_keys_falls_back":
        rel = W.make_rule(159, 8000, 600, 16, 16, np.int64, dup_frac=0.3)
    else:
        rel = W.make_rule(160, 200_000, 30_000, 16, 16, np.int32, src_dist="zipf", src_s=1.1)
    keys, out, plan, _ = run_rule(rel, flags=flags)
    if case == "mean":
        ok, oo, sizes = O.rule_forward(rel.h_ids, rel.z, [OBr(b.src, b.dst, b.W, b.b, None) for b in rel.branches],
                                       agg="mean")
    else:
        ok, oo, sizes = oracle_rule(rel, **kw)
    assert np.array_equal(keys, ok)
    assert plan.matched == sizes
    assert rel_frob(out, oo) <= FP32_TOL
    keys2, out2, _, _ = run_rule(rel, flags=flags | R.FLAG_PER_TUPLE)
    assert np.array_equal(keys, keys2)
    assert rel_frob(out, out2.astype(np.float64)) <= FP32_TOL


def _identity_rel(seed, k, groups, d, dst_s=None):
    """Out(g; SUM z) :- H(k; z), G(k, g): every H row in one group (uniform, or Zipf over the groups)."""
    rng = np.random.default_rng(seed)
    h = rng.permutation(k).astype(np.int32)
    z = rng.standard_normal((k, d)).astype(np.float32)
    if dst_s is None:
        g = rng.integers(0, groups, size=k).astype(np.int32)
    else:
        g = (rng.zipf(dst_s, size=k) % groups).astype(np.int32)
    return W.Relations(h_ids=h, z=z, branches=[W.Branch(src=h.copy(), dst=g, W=None, b=None)])


@pytest.mark.parametrize("case", ["readout8_d64_kahan", "readout8_d64", "readout_d128", "readout_d4_hubs",
                                  "join_dst_d32", "union_d16", "mean_d64", "d48_falls_back"])
def test_fp32_identity_aggregate_first(gpu, case):
    """Identity rules of the FP32 form (no Linear: a SUM of the src rows per output row, e.g. the SUM
    readout) take the aggregate-first gather-sum for d in {4, ..., 128}: against the FP64 oracle at
    the FP32 bar and against the per-tuple FP32 form on the same inputs; key sets and join sizes
    bit-exact. Covers groups of 25,000 rows (more than 256 chunks: the two-level fix-up), Kahan,
    hub groups, a joined dst without Concat, a union of branches, MEAN and a width that takes the
    per-tuple form."""
    flags, okw, agg = R.FLAG_NO_JOIN_DST, dict(join_dst=False, concat_dst=False), "sum"
    if case == "readout8_d64_kahan":
        rel, flags = _identity_rel(170, 200_000, 8, 64), flags | R.FLAG_KAHAN
    elif case == "readout8_d64":
        rel = _identity_rel(171, 200_000, 8, 64)
    elif case == "readout_d128":
        rel = _identity_rel(172, 100_000, 3000, 128)
    elif case == "readout_d4_hubs":
        rel = _identity_rel(173, 150_000, 500, 4, dst_s=1.5)
    elif case == "join_dst_d32":
        # uniform src (about 15 tuples per src row): the per-tuple backward adds dz rows by atomics in
        # no fixed order, so src hubs of thousands of tuples would leave f32 errors above 1e-5
        rel = W.make_rule(174, 60_000, 4000, 32, 32, np.int32, dst_dist="zipf", dst_s=1.2)
        rel.branches[0].W, rel.branches[0].b = None, None
        flags, okw = R.FLAG_NO_CONCAT_DST, dict(concat_dst=False)
    elif case == "union_d16":
        rel = W.make_rule(175, 0, 3000, 16, 16, np.int32, dst_dist="zipf", dst_s=1.0,
                          branch_tuples=[20_000, 10_000, 5000])
        for b in rel.branches:
            b.W, b.b = None, None
        flags, okw = R.FLAG_NO_CONCAT_DST, dict(concat_dst=False)
    elif case == "mean_d64":
        rel, flags, agg = _identity_rel(176, 50_000, 300, 64), flags | R.FLAG_MEAN, "mean"
    else:
        rel = _identity_rel(177, 20_000, 100, 48)
    keys, out, plan, _ = run_rule(rel, flags=flags)
    if agg == "mean":
        brs = [OBr(b.src, b.dst, None, None, None) for b in rel.branches]
        ok, oo, sizes = O.rule_forward(rel.h_ids, rel.z, brs, agg="mean", **okw)
    else:
        ok, oo, sizes = oracle_rule(rel, **okw)
    assert np.array_equal(keys, ok)
    assert plan.matched == sizes
    assert rel_frob(out, oo) <= FP32_TOL
    keys2, out2, plan2, t2 = run_rule(rel, flags=flags | R.FLAG_PER_TUPLE)
    assert np.array_equal(keys, keys2)
    assert rel_frob(out, out2.astype(np.float64)) <= FP32_TOL
    # the backward (dz as the gather-sum of dOut rows in src order for d in {4, ..., 128}; the
    # per-tuple form adds dOut rows into dz by atomics) against the oracle and against each other
    dout = np.random.default_rng(7).standard_normal(out.shape).astype(np.float32)
    z = to_dev(rel.z)
    _, _, dz, _ = plan.backward(to_dev(dout), z)
    _, _, dz2, _ = plan2.backward(to_dev(dout), z)
    torch.cuda.synchronize()
    plan.check()
    brs = [OBr(b.src, b.dst, None, None, None) for b in rel.branches]
    _, _, oz, _ = O.rule_backward(rel.h_ids, rel.z, brs, keys, dout, agg=agg, **okw)
    assert rel_frob(dz.cpu().numpy(), oz) <= FP32_TOL
    assert rel_frob(dz.cpu().numpy(), dz2.cpu().double().numpy()) <= FP32_TOL
