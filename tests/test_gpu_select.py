"""GPU parity of the selection (a conjunctive filter expression over each tuple's src and dst keys
and constants, evaluated during the join emission) against the FP64 oracle, on both emission paths
(unique H keys: one pass; duplicate H keys: count and emit passes), in the FP32 and BF16 forms, for
a union, a readout without a dst join and the backward."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import OBr, bf16_round, oracle_rule, rel_frob, run_rule, to_dev

pytestmark = pytest.mark.gpu

PREDS = [[("src", "<", "dst")], [("dst", "!=", 7), ("src", ">=", 40)], [(300, ">", "src"), ("dst", "<=", "src")]]


def _check(rel, filters, flags=0, z_dtype=torch.float32, tol=1e-5):
    keys, out, plan, t = run_rule(rel, flags=flags, z_dtype=z_dtype, filters=filters)
    ok, oo, sizes = oracle_rule(rel, filters=filters)
    assert np.array_equal(keys, ok)
    assert plan.matched == sizes
    assert rel_frob(out, oo) <= tol
    return keys, out, plan, t


@pytest.mark.parametrize("preds", PREDS)
def test_select_unique_keys_fp32(gpu, preds):
    _check(W.make_rule(71, 20_000, 500, 16, 24, np.int32, act="relu"), [preds])


@pytest.mark.parametrize("preds", PREDS)
def test_select_duplicate_keys_int64(gpu, preds):
    rel = W.make_rule(72, 8000, 600, 8, 12, np.int64, dup_frac=0.2, missing_frac=0.1)
    _check(rel, [preds])


def test_select_bf16_union_with_per_branch_filters(gpu):
    rel = W.make_rule(73, 0, 2000, 64, 96, np.int32, dst_dist="zipf", dst_s=1.0, d_r=64,
                      branch_tuples=[9000, 5000, 2500])
    keys, out, plan, t = run_rule(rel, flags=R.FLAG_BF16, filters=PREDS)
    ok, oo, sizes = oracle_rule(rel, filters=PREDS)
    assert np.array_equal(keys, ok) and plan.matched == sizes
    assert rel_frob(out, oo) <= 2e-2
    _, oo_r, _ = oracle_rule(rel, round_z=True, round_r=True, round_w=True, filters=PREDS)
    assert rel_frob(out, oo_r) <= 1e-4


def test_select_readout_on_group_key(gpu):
    rng = np.random.default_rng(2)
    k = 6000
    h = rng.permutation(k).astype(np.int32)
    z = rng.standard_normal((k, 32)).astype(np.float32)
    g = rng.integers(0, 10, size=k).astype(np.int32)
    rel = W.Relations(h_ids=h, z=z, branches=[W.Branch(src=h.copy(), dst=g, W=None, b=None)])
    preds = [[("dst", ">=", 3), ("dst", "<", 8)]]
    keys, out, plan, _ = run_rule(rel, flags=R.FLAG_NO_JOIN_DST, filters=preds)
    ok, oo, _ = oracle_rule(rel, join_dst=False, concat_dst=False, filters=preds)
    assert np.array_equal(keys, ok)
    assert rel_frob(out, oo) <= 1e-5


def test_select_backward(gpu):
    rel = W.make_rule(74, 4000, 300, 16, 24, np.int32, d_r=8, act="relu")
    preds = [[("src", "!=", "dst"), ("dst", ">", 20)]]
    keys, out, plan, t = run_rule(rel, filters=preds)
    dout = np.random.default_rng(1).standard_normal(out.shape).astype(np.float32)
    dW, db, dz, dr = plan.backward(to_dev(dout), t["z"], t["W"], t["b"], t["r"])
    brs = [OBr(b.src, b.dst, b.W, b.b, b.r, preds[0]) for b in rel.branches]
    oW, ob, oz, orr = O.rule_backward(rel.h_ids, rel.z, brs, keys, dout, act=rel.act)
    assert rel_frob(dW[0].cpu().numpy(), oW[0]) <= 1e-5
    assert rel_frob(db[0].cpu().numpy(), ob[0]) <= 1e-5
    assert rel_frob(dz.cpu().numpy(), oz) <= 1e-5
    assert rel_frob(dr[0].cpu().numpy(), orr[0]) <= 1e-5


def test_select_rejects_bad_filters(gpu):
    rel = W.make_rule(75, 100, 50, 8, 8, np.int32)
    with pytest.raises(AssertionError):
        run_rule(rel, filters=[[("src", "<", "dst")] * 5])
