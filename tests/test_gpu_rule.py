"""GPU parity of the rule path (plan, forward, backward) against the FP64 oracle.

Bars: join output and output key sets bit-exact; relative Frobenius error per output relation
<= 1e-5 for the FP32 form and <= 2e-2 for the BF16 form against the oracle on the original inputs.
The BF16 form is also held to 1e-4 against the oracle fed the same bf16-rounded operands, which
catches layout mistakes that a 2e-2 bar could hide."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import OBr, bf16_round, oracle_rule, rel_frob, run_rule, to_dev

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
BF16_TOL = 2e-2
BF16_SAME_INPUT_TOL = 1e-4


def _check_fp32(rel, flags=0, **kw):
    keys, out, plan, _ = run_rule(rel, flags=flags)
    ok, oo, sizes = oracle_rule(rel, **kw)
    assert np.array_equal(keys, ok)
    assert plan.matched == sizes
    assert rel_frob(out, oo) <= FP32_TOL
    return keys, out


# ------------------------------------------------------------------------------ FP32 form
def test_config1_fp32(gpu):
    _check_fp32(W.config1())


@pytest.mark.parametrize("n_tuples", [1, 31, 33, 257, 4099])
def test_fp32_ragged_sizes(gpu, n_tuples):
    _check_fp32(W.make_rule(3, n_tuples, 97, 16, 24, np.int32))


def test_fp32_bag_semantics_duplicates_and_missing(gpu):
    rel = W.make_rule(5, 3000, 400, 8, 12, np.int64, dup_frac=0.3, missing_frac=0.1, sparse_keys=True)
    _check_fp32(rel)


def test_fp32_relu_and_edge_embedding(gpu):
    _check_fp32(W.make_rule(6, 5000, 300, 16, 32, np.int32, d_r=8, act="relu"))


@pytest.mark.parametrize("kahan", [False, True])
def test_fp32_union_with_hubs(gpu, kahan):
    rel = W.make_rule(7, 0, 500, 16, 16, np.int32, dst_dist="zipf", dst_s=1.3, d_r=16,
                      branch_tuples=[6000, 3000, 1500])
    _check_fp32(rel, flags=R.FLAG_KAHAN if kahan else 0)


def test_fp32_readout_identity_no_dst_join(gpu):
    """Out(g; SUM z) :- H(k; z), G(k, g): 8 groups, so every group spans many tiles."""
    rng = np.random.default_rng(0)
    k = 5000
    h = rng.permutation(k).astype(np.int32)
    z = rng.standard_normal((k, 64)).astype(np.float32)
    g = rng.integers(0, 8, size=k).astype(np.int32)
    rel = W.Relations(h_ids=h, z=z, branches=[W.Branch(src=h.copy(), dst=g, W=None, b=None)])
    keys, out, plan, _ = run_rule(rel, flags=R.FLAG_NO_JOIN_DST | R.FLAG_KAHAN)
    ok, oo, _ = oracle_rule(rel, join_dst=False, concat_dst=False)
    assert np.array_equal(keys, ok)
    assert rel_frob(out, oo) <= FP32_TOL


@pytest.mark.parametrize("groups,kahan", [(8, False), (8, True), (3000, False), (3000, True)])
def test_fp32_readout_ranges_of_tiles(gpu, groups, kahan):
    """500k rows into few or many groups: a warp walks a range of several 32-tuple tiles, so runs
    are carried from tile to tile inside a range and from range to range by the fix-up."""
    rng = np.random.default_rng(1)
    k = 500_000
    h = rng.permutation(k).astype(np.int32)
    z = rng.standard_normal((k, 64)).astype(np.float32)
    g = rng.integers(0, groups, size=k).astype(np.int32)
    rel = W.Relations(h_ids=h, z=z, branches=[W.Branch(src=h.copy(), dst=g, W=None, b=None)])
    keys, out, plan, _ = run_rule(rel, flags=R.FLAG_NO_JOIN_DST | (R.FLAG_KAHAN if kahan else 0))
    ok, oo, _ = oracle_rule(rel, join_dst=False, concat_dst=False)
    assert np.array_equal(keys, ok)
    assert rel_frob(out, oo) <= FP32_TOL


@pytest.mark.parametrize("d,kahan", [(16, False), (16, True), (6, False)])
def test_fp32_ranges_with_hubs(gpu, d, kahan):
    """600k tuples, Zipf(1.3) dst (the largest run is about a quarter of E): ranges of tiles with
    runs inside, across and over whole ranges; d = 6 takes the scalar-load form."""
    rel = W.make_rule(16, 600_000, 20_000, d, 2 * d, np.int32, dst_dist="zipf", dst_s=1.3, act="relu")
    _check_fp32(rel, flags=R.FLAG_KAHAN if kahan else 0)


def test_empty_join(gpu):
    rel = W.make_rule(8, 100, 50, 8, 8, np.int32, missing_frac=1.0)
    keys, out, plan, _ = run_rule(rel)
    assert plan.n_out == 0 and keys.size == 0


# ------------------------------------------------------------------------------ BF16 form
def _check_bf16(rel, z_dtype=torch.bfloat16, r_dtype=torch.float32, flags=0):
    keys, out, plan, _ = run_rule(rel, flags=flags | R.FLAG_BF16, z_dtype=z_dtype, r_dtype=r_dtype,
                                  w_dtype=torch.float32)
    ok, oo, sizes = oracle_rule(rel)
    assert np.array_equal(keys, ok)
    assert plan.matched == sizes
    err = rel_frob(out, oo)
    assert err <= BF16_TOL, err
    _, oo_r, _ = oracle_rule(rel, round_z=True, round_r=True, round_w=True)
    err_same = rel_frob(out, oo_r)
    assert err_same <= BF16_SAME_INPUT_TOL, err_same
    return err


def test_bf16_scaled_config2_shape(gpu):
    """d = 128, Linear 256 -> 128, int64 keys, Zipf(1.1) src: several 256-tuple tiles + ragged tail."""
    rel = W.make_rule(11, 70_003, 6000, 128, 128, np.int64, src_dist="zipf", src_s=1.1)
    _check_bf16(rel)


def test_bf16_relu_f32_embeddings(gpu):
    rel = W.make_rule(12, 40_000, 5000, 64, 64, np.int32, src_dist="zipf", src_s=1.2, act="relu")
    _check_bf16(rel, z_dtype=torch.float32)


@pytest.mark.parametrize("kahan", [False, True])
def test_bf16_union_config4_shape(gpu, kahan):
    rel = W.make_rule(13, 0, 3000, 64, 96, np.int32, dst_dist="zipf", dst_s=1.0, d_r=64,
                      branch_tuples=[20_000, 10_000, 5000])
    _check_bf16(rel, z_dtype=torch.float32, flags=R.FLAG_KAHAN if kahan else 0)


@pytest.mark.parametrize("d,d_out,d_r", [(72, 200, 8), (64, 256, 0), (8, 16, 0), (128, 48, 24)])
def test_bf16_odd_widths(gpu, d, d_out, d_r):
    rel = W.make_rule(14, 9000, 700, d, d_out, np.int32, d_r=d_r)
    _check_bf16(rel, r_dtype=torch.bfloat16)


def test_bf16_hub_spanning_many_tiles(gpu):
    rel = W.make_rule(15, 30_000, 200, 64, 64, np.int32, dst_dist="zipf", dst_s=2.0)
    _check_bf16(rel, flags=R.FLAG_KAHAN)


# ------------------------------------------------------------------------------ backward
def _grads_oracle(rel, dout_keys, dout):
    brs = [OBr(b.src, b.dst, b.W, b.b, b.r) for b in rel.branches]
    return O.rule_backward(rel.h_ids, rel.z, brs, dout_keys, dout, act=rel.act)


@pytest.mark.parametrize("act,d_r", [("none", 0), ("relu", 8)])
def test_fp32_backward_matches_oracle(gpu, act, d_r):
    rel = W.make_rule(21, 4000, 300, 16, 24, np.int32, d_r=d_r, act=act, dup_frac=0.1)
    keys, out, plan, t = run_rule(rel)
    dout = np.random.default_rng(1).standard_normal(out.shape).astype(np.float32)
    dW, db, dz, dr = plan.backward(to_dev(dout), t["z"], t["W"], t["b"], t["r"])
    oW, ob, oz, orr = _grads_oracle(rel, keys, dout)
    assert rel_frob(dW[0].cpu().numpy(), oW[0]) <= FP32_TOL
    assert rel_frob(db[0].cpu().numpy(), ob[0]) <= FP32_TOL
    assert rel_frob(dz.cpu().numpy(), oz) <= FP32_TOL
    if d_r:
        assert rel_frob(dr[0].cpu().numpy(), orr[0]) <= FP32_TOL


def test_autograd_function_fp32(gpu):
    rel = W.make_rule(22, 3000, 200, 16, 16, np.int32, act="relu")
    keys, out, plan, t = run_rule(rel)
    z = t["z"].clone().requires_grad_(True)
    Wt = t["W"][0].clone().requires_grad_(True)
    bt = t["b"][0].clone().requires_grad_(True)
    y = R.RelnnRule.apply(plan, z, Wt, bt, None)
    C = torch.randn_like(y)
    (y * C).sum().backward()
    oW, ob, oz, _ = _grads_oracle(rel, keys, C.cpu().numpy())
    assert rel_frob(Wt.grad.cpu().numpy(), oW[0]) <= FP32_TOL
    assert rel_frob(bt.grad.cpu().numpy(), ob[0]) <= FP32_TOL
    assert rel_frob(z.grad.cpu().numpy(), oz) <= FP32_TOL


# ------------------------------------------------------------------------------ BF16 backward
def _bf16_grads(rel, flags=0):
    keys, out, plan, t = run_rule(rel, flags=flags | R.FLAG_BF16 | R.FLAG_RELU_MASK, z_dtype=torch.bfloat16,
                                  r_dtype=torch.float32, w_dtype=torch.float32)
    dout = np.random.default_rng(2).standard_normal(out.shape).astype(np.float32)
    dW, db, dz, dr = plan.backward(to_dev(dout), t["z"], t["W"], t["b"], t["r"])
    torch.cuda.synchronize()
    plan.check()
    # oracle on the bf16-rounded operands the device used
    brs = [OBr(b.src, b.dst, bf16_round(b.W), b.b, None if b.r is None else bf16_round(b.r)) for b in rel.branches]
    oW, ob, oz, orr = O.rule_backward(rel.h_ids, bf16_round(rel.z), brs, keys, dout, act=rel.act)
    return (dW, db, dz, dr), (oW, ob, oz, orr)


@pytest.mark.parametrize("shape", ["c2", "c3", "c4", "odd"])
def test_bf16_backward_matches_oracle(gpu, shape):
    if shape == "c2":
        rel = W.make_rule(41, 30_011, 3000, 128, 128, np.int64, src_dist="zipf", src_s=1.1)
    elif shape == "c3":
        rel = W.make_rule(42, 20_000, 2500, 64, 64, np.int32, src_dist="zipf", src_s=1.2, act="relu")
    elif shape == "c4":
        rel = W.make_rule(43, 0, 2000, 64, 96, np.int32, dst_dist="zipf", dst_s=1.0, d_r=64,
                          branch_tuples=[9000, 5000, 2500])
    else:
        rel = W.make_rule(44, 7000, 600, 72, 40, np.int32, d_r=8, act="relu", dup_frac=0.05)
    (dW, db, dz, dr), (oW, ob, oz, orr) = _bf16_grads(rel)
    for i in range(len(rel.branches)):
        # dY is rounded to bf16 before the tensor-core GEMMs: 2e-2 is the BF16-form bar
        assert rel_frob(dW[i].cpu().numpy(), oW[i]) <= BF16_TOL
        assert rel_frob(db[i].cpu().numpy(), ob[i]) <= 1e-5  # db is summed in f32 from unrounded dY
        if dr is not None:
            assert rel_frob(dr[i].cpu().numpy(), orr[i]) <= BF16_TOL
    assert rel_frob(dz.cpu().numpy(), oz) <= BF16_TOL


def test_plan_release_in_stream_order(gpu):
    """relnn_plan_release frees the plan after the work queued on its stream, without a device-wide
    wait: a forward issued on a side stream, then the release, then the result read back."""
    rel = W.make_rule(97, 20_000, 2000, 16, 16, np.int32)
    br = rel.branches[0]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = R.RulePlan(to_dev(rel.h_ids), [(to_dev(br.src), to_dev(br.dst))], 16, 16)
        out = plan.forward(to_dev(rel.z), [to_dev(br.W)], [to_dev(br.b)])
        keys = plan.out_keys()
        plan.release()
    s.synchronize()
    ok, oo, _ = oracle_rule(rel)
    assert np.array_equal(keys.cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5
    plan.release()  # a second release is a no-op


@pytest.mark.parametrize("n_keys", [1, 2, 1024, 1000, 4096])
@pytest.mark.parametrize("bf16", [False, True])
def test_unmatched_tuples_sorted_last(gpu, n_keys, bf16):
    """Unique H keys without a selection: tuples whose src or dst key is absent from H get a sentinel
    group key above every dst position and sort behind the matched ones, whose count is read with
    the plan's final synchronisation. Key spaces whose size is a power of two (the sentinel then
    needs one more key bit), a single key, and ragged sizes; join sizes and key sets bit-exact, values
    at the form's bar."""
    rel = W.make_rule(90 + n_keys, 3 * n_keys + 777, n_keys, 16, 16, np.int32, missing_frac=0.3)
    flags = R.FLAG_BF16 if bf16 else 0
    keys, out, plan, _ = run_rule(rel, flags=flags, z_dtype=torch.bfloat16 if bf16 else torch.float32)
    ok, oo, sizes = oracle_rule(rel, round_z=bf16, round_w=bf16)
    assert np.array_equal(keys, ok)
    assert plan.matched == sizes
    assert plan.n_out == ok.size
    assert rel_frob(out, oo) <= (1e-4 if bf16 else FP32_TOL)


@pytest.mark.parametrize("bits", [4, 7, 11])
def test_radix_digit_widths_give_the_same_plan(gpu, bits):
    """The radix sorts (the join build over sparse int64 keys and the group sort over 18-bit group
    keys) with digits of at most 4, 7 and 11 bits: 5, 3 and 2 passes, the scatter ranking each digit
    with one ballot per digit bit. A stable sort gives one order, so the key set and the forward are
    the same bit for bit as with the default width, and both meet the oracle bars."""
    rel = W.make_rule(21, 300_000, 200_000, 64, 64, np.int64, sparse_keys=True, src_dist="zipf", src_s=1.1)
    saved = R.tune_get(R.TUNE_SORT_BITS)
    try:
        R.tune_set(R.TUNE_SORT_BITS, 8)
        keys0, out0, _, _ = run_rule(rel, flags=R.FLAG_BF16, z_dtype=torch.bfloat16)
        R.tune_set(R.TUNE_SORT_BITS, bits)
        keys, out, plan, _ = run_rule(rel, flags=R.FLAG_BF16, z_dtype=torch.bfloat16)
    finally:
        R.tune_set(R.TUNE_SORT_BITS, saved)
    assert np.array_equal(keys, keys0)
    assert np.array_equal(out, out0)
    ok, oo, sizes = oracle_rule(rel)
    assert np.array_equal(keys, ok)
    assert plan.matched == sizes
    _, oo_r, _ = oracle_rule(rel, round_z=True, round_w=True)
    assert rel_frob(out, oo_r) <= BF16_SAME_INPUT_TOL
