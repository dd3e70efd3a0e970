"""GPU parity of attention over a join (relnn_attention_*; the product head of paper Sec. 1 and the
HGT softmax head of Sec. 5) against the FP64 oracle: every width the kernels take, 1 to 32 heads,
f32 and bf16 rows (the oracle sees the same bf16-rounded values), hub keys whose rows span many
ranges (merged by the fix-up), duplicate H keys, sparse int64 keys, the log-sum-exp, the backward,
and the rejected shapes."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import bf16_round, rel_frob, to_dev

pytestmark = pytest.mark.gpu


def _case(seed, n, keys, d, key_dtype=np.int32, **kw):
    rel = W.make_rule(seed, n, keys, d, 1, key_dtype, **kw)
    rng = np.random.default_rng(seed + 1000)
    n_h = rel.h_ids.size
    q, k, v = (rng.standard_normal((n_h, d)).astype(np.float32) for _ in range(3))
    return rel, q, k, v


def _run(rel, q, k, v, heads, scale, mode, bf16):
    br = rel.branches[0]
    plan = R.RulePlan(to_dev(rel.h_ids), [(to_dev(br.src), to_dev(br.dst))], q.shape[1], 1)
    dt = torch.bfloat16 if bf16 else torch.float32
    tq, tk, tv = (to_dev(x, dt) for x in (q, k, v))
    out, lse = plan.attention(tq, tk, tv, heads, scale, mode)
    torch.cuda.synchronize()
    plan.check()
    if bf16:
        q, k, v = bf16_round(q), bf16_round(k), bf16_round(v)
    return plan, (tq, tk, tv), out, lse, (q, k, v)


@pytest.mark.parametrize("d,heads", [(32, 1), (64, 4), (128, 8), (256, 32), (128, 1)])
@pytest.mark.parametrize("bf16", [False, True])
def test_softmax_head_forward(gpu, d, heads, bf16):
    rel, q, k, v = _case(91, 40_000, 3000, d, src_dist="zipf", src_s=1.2, dst_dist="zipf", dst_s=1.3)
    scale = 1.0 / np.sqrt(d // heads)
    plan, _, out, lse, (q, k, v) = _run(rel, q, k, v, heads, scale, "softmax", bf16)
    br = rel.branches[0]
    ok, oo, olse = O.attention_forward(rel.h_ids, q, k, v, br.src, br.dst, heads, scale, "softmax")
    assert np.array_equal(plan.out_keys().cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5
    np.testing.assert_allclose(lse.cpu().numpy(), olse, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("d", [32, 128, 256])
@pytest.mark.parametrize("bf16", [False, True])
def test_product_head_forward(gpu, d, bf16):
    rel, q, k, v = _case(92, 30_000, 2500, d, np.int64, src_dist="zipf", src_s=1.1, sparse_keys=True, dup_frac=0.05)
    plan, _, out, lse, (q, k, v) = _run(rel, q, k, v, 1, 1.0, "product", bf16)
    assert lse is None
    br = rel.branches[0]
    ok, oo, _ = O.attention_forward(rel.h_ids, q, k, v, br.src, br.dst, 1, 1.0, "product")
    assert np.array_equal(plan.out_keys().cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5


def test_softmax_head_hub_rows_span_many_ranges(gpu):
    """One key holds most tuples: its row is the merge of many range partials (m, l, sum)."""
    rel, q, k, v = _case(93, 200_000, 4000, 64, dst_dist="zipf", dst_s=2.2)
    plan, _, out, lse, (q, k, v) = _run(rel, q, k, v, 2, 0.5, "softmax", False)
    br = rel.branches[0]
    ok, oo, olse = O.attention_forward(rel.h_ids, q, k, v, br.src, br.dst, 2, 0.5, "softmax")
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5
    np.testing.assert_allclose(lse.cpu().numpy(), olse, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("mode,heads", [("softmax", 4), ("product", 1)])
@pytest.mark.parametrize("bf16", [False, True])
def test_attention_backward(gpu, mode, heads, bf16):
    rel, q, k, v = _case(94, 20_000, 2000, 64, dst_dist="zipf", dst_s=1.2, dup_frac=0.05)
    plan, (tq, tk, tv), out, lse, (q, k, v) = _run(rel, q, k, v, heads, 0.25, mode, bf16)
    dout = np.random.default_rng(9).standard_normal(tuple(out.shape)).astype(np.float32)
    dq, dk, dv = plan.attention_backward(to_dev(dout), out, lse, tq, tk, tv, heads, 0.25, mode)
    torch.cuda.synchronize()
    br = rel.branches[0]
    oq, ok_, ov = O.attention_backward(rel.h_ids, q, k, v, br.src, br.dst, dout, heads, 0.25, mode)
    assert rel_frob(dq.cpu().numpy(), oq) <= 1e-5
    assert rel_frob(dk.cpu().numpy(), ok_) <= 1e-5
    assert rel_frob(dv.cpu().numpy(), ov) <= 1e-5


def test_attention_rejects_unsupported_shapes(gpu):
    rel, q, k, v = _case(95, 2000, 300, 64)
    br = rel.branches[0]
    plan = R.RulePlan(to_dev(rel.h_ids), [(to_dev(br.src), to_dev(br.dst))], 64, 1)
    tq, tk, tv = (to_dev(x) for x in (q, k, v))
    with pytest.raises(R.RelnnError):
        plan.attention(tq, tk, tv, 3, 1.0)  # heads not a power of two
    with pytest.raises(R.RelnnError):
        plan.attention(tq[:, :48].contiguous(), tk[:, :48].contiguous(), tv[:, :48].contiguous(), 1, 1.0)
    with pytest.raises(R.RelnnError):
        plan.attention(tq, tk, tv[:, :32].contiguous(), 1, 1.0, "product")
    two = W.make_rule(96, 0, 300, 64, 1, np.int32, branch_tuples=[1000, 500])
    p2 = R.RulePlan(to_dev(two.h_ids), [(to_dev(b.src), to_dev(b.dst)) for b in two.branches], 64, 1)
    z = to_dev(np.zeros((two.h_ids.size, 64), np.float32))
    with pytest.raises(R.RelnnError):
        p2.attention(z, z, z, 1, 1.0)
