"""GPU parity of the MAX aggregator (alpha = per-feature maximum per output row, paper Sec. 2.2 and the
scatter-max of Sec. 4.2) against the FP64 oracle.

Which tuple receives a row's gradient is an integer decision taken on floating-point values. The
exact cases use quantised inputs (z multiples of 1/4, W and b multiples of 1/16, dOut multiples of
1/8, all exact in bf16) for which every tuple output and every gradient sum is exact in f32, so the
device and the oracle take the same decisions on the same values and must agree bit for bit, ties
included (many tuples tie at these values: the first in (dst H row, E row, src H row) order wins).
The continuous cases check the forward values within the form's tolerance."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import OBr, bf16_round, rel_frob, run_rule, to_dev

pytestmark = pytest.mark.gpu

BF16 = R.FLAG_BF16


def quantise(rel):
    rel.z = np.clip(np.round(rel.z * 4) / 4, -2, 2).astype(np.float32)
    for b in rel.branches:
        b.W = np.clip(np.round(b.W * 64) / 16, -1, 1).astype(np.float32)
        b.b = np.clip(np.round(b.b * 64) / 16, -1, 1).astype(np.float32)
    return rel


def oracle_max(rel, join_dst=True, concat_dst=True):
    brs = [OBr(b.src, b.dst, b.W, b.b, b.r) for b in rel.branches]
    return O.rule_forward(rel.h_ids, rel.z, brs, act=rel.act, join_dst=join_dst, concat_dst=concat_dst, agg="max")


def oracle_max_grad(rel, keys, dout, join_dst=True, concat_dst=True):
    brs = [OBr(b.src, b.dst, b.W, b.b, b.r) for b in rel.branches]
    return O.rule_backward(rel.h_ids, rel.z, brs, keys, dout, act=rel.act, join_dst=join_dst,
                           concat_dst=concat_dst, agg="max")


def _case(seed, bf16, act, **kw):
    d, d_out = (64, 64) if bf16 else (16, 24)
    return quantise(W.make_rule(seed, kw.pop("n", 30_000), kw.pop("keys", 2500), d, d_out, np.int32, act=act, **kw))


def _run(rel, bf16, extra=0):
    flags = R.FLAG_MAX | (BF16 if bf16 else 0) | extra
    zdt = torch.bfloat16 if bf16 else torch.float32
    return run_rule(rel, flags=flags, z_dtype=zdt)


def _exact_backward(rel, keys, out, plan, t, seed, **okw):
    dout = np.clip(np.round(np.random.default_rng(seed).standard_normal(out.shape) * 8) / 8, -2, 2).astype(np.float32)
    dW, db, dz, _ = plan.backward(to_dev(dout), t["z"], t["W"], t["b"], t["r"])
    torch.cuda.synchronize()
    plan.check()
    oW, ob, oz, _ = oracle_max_grad(rel, keys, dout, **okw)
    np.testing.assert_array_equal(dW[0].cpu().numpy(), oW[0])
    np.testing.assert_array_equal(db[0].cpu().numpy(), ob[0])
    np.testing.assert_array_equal(dz.cpu().numpy(), oz)


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("act", ["none", "relu"])
def test_max_exact_forward_and_backward(gpu, bf16, act):
    rel = _case(71, bf16, act, src_dist="zipf", src_s=1.2, dup_frac=0.05, missing_frac=0.02)
    keys, out, plan, t = _run(rel, bf16)
    ok, oo, sizes = oracle_max(rel)
    assert np.array_equal(keys, ok) and plan.matched == sizes
    np.testing.assert_array_equal(out, oo)
    _exact_backward(rel, keys, out, plan, t, 5)


@pytest.mark.parametrize("bf16", [False, True])
def test_max_exact_long_segments(gpu, bf16):
    """A hub key holds most tuples: its row spans hundreds of tiles, so its (value, position)
    partials go through the block-per-segment fix-up."""
    rel = _case(72, bf16, "relu", n=60_000, keys=3000, dst_dist="zipf", dst_s=2.0)
    keys, out, plan, t = _run(rel, bf16)
    ok, oo, _ = oracle_max(rel)
    assert np.array_equal(keys, ok)
    np.testing.assert_array_equal(out, oo)
    _exact_backward(rel, keys, out, plan, t, 6)


def test_max_exact_readout_form(gpu):
    """dst as a raw group key (no dst join, no z_dst): the readout form with MAX."""
    rel = quantise(W.make_rule(73, 20_000, 2000, 16, 16, np.int32, act="relu"))
    rng = np.random.default_rng(4)
    for b in rel.branches:
        b.dst = rng.integers(0, 37, size=b.dst.size).astype(np.int32)
        b.W = np.ascontiguousarray(b.W[:, :16])
    keys, out, plan, t = run_rule(rel, flags=R.FLAG_MAX | R.FLAG_NO_JOIN_DST)
    ok, oo, _ = oracle_max(rel, join_dst=False, concat_dst=False)
    assert np.array_equal(keys, ok)
    np.testing.assert_array_equal(out, oo)
    _exact_backward(rel, keys, out, plan, t, 7, join_dst=False, concat_dst=False)


@pytest.mark.parametrize("bf16", [False, True])
def test_max_continuous_forward(gpu, bf16):
    d, d_out = (64, 128) if bf16 else (32, 48)
    rel = W.make_rule(74, 50_000, 4000, d, d_out, np.int64, act="relu", src_dist="zipf", src_s=1.1,
                      sparse_keys=True)
    keys, out, plan, _ = _run(rel, bf16)
    if bf16:
        rel.z = bf16_round(rel.z)
        for b in rel.branches:
            b.W = bf16_round(b.W)
    ok, oo, _ = oracle_max(rel)
    assert np.array_equal(keys, ok)
    # f32 tuple outputs (f32 FMA, or bf16 products accumulated in f32): a maximum is within the
    # error of one of them
    assert rel_frob(out, oo) <= (1e-5 if bf16 else 1e-6)


def test_max_rejects_unsupported_combinations(gpu):
    rel = W.make_rule(75, 0, 300, 16, 16, np.int32, branch_tuples=[2000, 1000])
    with pytest.raises(R.RelnnError):
        run_rule(rel, flags=R.FLAG_MAX)
    one = W.make_rule(76, 2000, 300, 16, 16, np.int32)
    with pytest.raises(R.RelnnError):
        run_rule(one, flags=R.FLAG_MAX | R.FLAG_MEAN)
    with pytest.raises(R.RelnnError):
        run_rule(one, flags=R.FLAG_MAX | R.FLAG_PUSHDOWN | BF16)
    h = to_dev(one.h_ids)
    br = one.branches[0]
    plan = R.RulePlan(h, [(to_dev(br.src), to_dev(br.dst))], 16, 16, flags=R.FLAG_MAX)
    z = to_dev(one.z)
    with pytest.raises(R.RelnnError):  # the argmax is recorded by a forward
        plan.backward(torch.zeros((plan.n_out, 16), device="cuda"), z, [to_dev(br.W)], [to_dev(br.b)])
