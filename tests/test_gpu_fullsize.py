"""GPU parity at the full sizes of the measured workloads, in the launch configurations bench.py times:
the single-rule workload (16M tuples over 1M int64 keys, BF16 form), the union workload (three
relations of 2M / 1M / 0.5M tuples with a per-tuple embedding, BF16 form, Kahan), the first rule
of the stacked program (4M tuples over 500k keys, ReLU, f32 z) and the 4,096 small FP32 rules in
one plan. The oracle evaluates sampled
output keys one by one: the E rows whose dst is a sampled key, joined with the full H, give exactly
those keys' rows. Properties that hold at any size are checked on the whole output: the output
key set is the set of dst keys with a matched tuple, and every branch's matched-tuple count is the
number of E rows whose two keys are both in H."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import OBr, bf16_round, rel_frob, to_dev

pytestmark = pytest.mark.gpu

N_SAMPLE = 200


def _matched_keys(rel):
    """Properties at any size: per branch the count of E rows with both keys in H (unique H keys),
    and the union of their dst keys."""
    hk = np.asarray(rel.h_ids)
    counts, keys = [], []
    for b in rel.branches:
        ok = np.isin(b.src, hk) & np.isin(b.dst, hk)
        counts.append(int(ok.sum()))
        keys.append(np.unique(b.dst[ok]))
    return counts, np.unique(np.concatenate(keys))


def _sampled_parity(rel, keys, out, flags, act, seed, round_=True, tol=1e-4, agg="sum"):
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(keys.size, size=min(N_SAMPLE, keys.size), replace=False))
    sk = keys[pick]
    brs = []
    for b in rel.branches:
        sel = np.isin(b.dst, sk)
        brs.append(OBr(b.src[sel], b.dst[sel], bf16_round(b.W) if round_ else b.W, b.b,
                       None if b.r is None else (bf16_round(b.r[sel]) if round_ else b.r[sel])))
    z = bf16_round(rel.z) if round_ else rel.z
    ok, oo, _ = O.rule_forward(rel.h_ids, z, brs, act=act, agg=agg)
    assert np.array_equal(ok, sk)
    assert rel_frob(out[pick], oo) <= tol


def _run(rel, flags, act, z_dtype, r_dtype=torch.float32):
    h = to_dev(rel.h_ids)
    brs = [(to_dev(b.src), to_dev(b.dst)) for b in rel.branches]
    d_r = 0 if rel.branches[0].r is None else rel.branches[0].r.shape[1]
    plan = R.RulePlan(h, brs, rel.z.shape[1], rel.branches[0].W.shape[0],
                      act=R.ACT_RELU if act == "relu" else R.ACT_NONE, flags=flags, d_r=d_r)
    W_ = [to_dev(b.W) for b in rel.branches]
    b_ = [to_dev(b.b) for b in rel.branches]
    r_ = None if d_r == 0 else [to_dev(b.r, r_dtype) for b in rel.branches]
    out = plan.forward(to_dev(rel.z, z_dtype), W_, b_, r_)
    torch.cuda.synchronize()
    plan.check()
    return plan, plan.out_keys().cpu().numpy(), out.cpu().numpy()


def test_single_rule_full_size(gpu):
    rel = W.config2()
    plan, keys, out = _run(rel, R.FLAG_BF16, "none", torch.bfloat16)
    counts, all_keys = _matched_keys(rel)
    assert plan.matched == counts
    assert np.array_equal(keys.astype(np.int64), all_keys.astype(np.int64))
    _sampled_parity(rel, keys, out, R.FLAG_BF16, "none", 1)


@pytest.mark.parametrize("kahan", [False, True])
def test_union_full_size(gpu, kahan):
    rel = W.config4()
    flags = R.FLAG_BF16 | (R.FLAG_KAHAN if kahan else 0)
    plan, keys, out = _run(rel, flags, "none", torch.float32)
    counts, all_keys = _matched_keys(rel)
    assert plan.matched == counts
    assert np.array_equal(keys, all_keys)
    _sampled_parity(rel, keys, out, flags, "none", 2)


def test_stacked_first_rule_full_size(gpu):
    r1, _, _, _, _ = W.config3()
    plan, keys, out = _run(r1, R.FLAG_BF16 | R.FLAG_RELU_MASK, "relu", torch.float32)
    counts, all_keys = _matched_keys(r1)
    assert plan.matched == counts
    assert np.array_equal(keys, all_keys)
    _sampled_parity(r1, keys, out, R.FLAG_BF16, "relu", 3)


def test_single_rule_full_size_max(gpu):
    """The same workload with the MAX aggregator (bench.py --agg max): sampled maxima."""
    rel = W.config2()
    plan, keys, out = _run(rel, R.FLAG_BF16 | R.FLAG_MAX, "none", torch.bfloat16)
    _, all_keys = _matched_keys(rel)
    assert np.array_equal(keys.astype(np.int64), all_keys.astype(np.int64))
    _sampled_parity(rel, keys, out, R.FLAG_BF16 | R.FLAG_MAX, "none", 4, agg="max")


def test_many_small_rules_full_size(gpu):
    """4,096 independent instances of the small FP32 rule in one plan and one FP32-form launch (the
    bench's many-small-rules workload): sampled output keys against the oracle."""
    hs, zs, ss, ds = [], [], [], []
    for i in range(4096):
        r = W.config1(seed=i)
        br = r.branches[0]
        off = np.int32(i * 1024)
        hs.append(r.h_ids + off)
        zs.append(r.z)
        ss.append(br.src + off)
        ds.append(br.dst + off)
        if i == 0:
            Wn, bn = br.W, br.b
    rel = W.Relations(h_ids=np.concatenate(hs), z=np.concatenate(zs),
                      branches=[W.Branch(src=np.concatenate(ss), dst=np.concatenate(ds), W=Wn, b=bn, r=None)],
                      act="none")
    plan, keys, out = _run(rel, 0, "none", torch.float32)
    counts, all_keys = _matched_keys(rel)
    assert plan.matched == counts
    assert np.array_equal(keys, all_keys)
    _sampled_parity(rel, keys, out, 0, "none", 5, round_=False, tol=1e-5)
