"""GPU parity of the transformation push-down (the Linear applied once per H row, then per-tuple
gathers and the SUM walk; the paper's future-work rewrite, Sec. 6) against the FP64 oracle of the
per-tuple definition, with the BF16 form's bars: <= 2e-2 against the oracle on the original inputs
and <= 1e-4 against the oracle fed the same bf16-rounded operands. Keys and matched counts are
bit-exact, and the per-tuple fused form on the same inputs agrees to rounding order."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import OBr, bf16_round, oracle_rule, rel_frob, run_rule, to_dev

pytestmark = pytest.mark.gpu

PD = R.FLAG_BF16 | R.FLAG_PUSHDOWN


def _check(rel, flags=0, z_dtype=torch.bfloat16):
    keys, out, plan, _ = run_rule(rel, flags=flags | PD, z_dtype=z_dtype)
    ok, oo, sizes = oracle_rule(rel)
    assert np.array_equal(keys, ok)
    assert plan.matched == sizes
    assert rel_frob(out, oo) <= 2e-2
    _, oo_r, _ = oracle_rule(rel, round_z=True, round_w=True)
    assert rel_frob(out, oo_r) <= 1e-4
    _, out_f, _, _ = run_rule(rel, flags=flags | R.FLAG_BF16, z_dtype=z_dtype)
    assert rel_frob(out, out_f) <= 1e-5
    return out


def test_pushdown_single_rule_int64_zipf(gpu):
    _check(W.make_rule(51, 50_003, 4000, 128, 128, np.int64, src_dist="zipf", src_s=1.1))


def test_pushdown_relu_f32_embeddings(gpu):
    _check(W.make_rule(52, 30_000, 2500, 64, 64, np.int32, src_dist="zipf", src_s=1.2, act="relu"),
           z_dtype=torch.float32)


def test_pushdown_union_of_branches(gpu):
    _check(W.make_rule(53, 0, 2000, 64, 64, np.int32, dst_dist="zipf", dst_s=1.0, branch_tuples=[9000, 5000]))


def test_pushdown_kahan_hub_over_many_ranges(gpu):
    _check(W.make_rule(54, 300_000, 200, 64, 64, np.int32, dst_dist="zipf", dst_s=2.0), flags=R.FLAG_KAHAN)


@pytest.mark.parametrize("d,d_out", [(64, 96), (32, 32), (128, 64)])
def test_pushdown_widths(gpu, d, d_out):
    _check(W.make_rule(55, 9000, 700, d, d_out, np.int32))


def test_pushdown_bag_semantics_and_ragged(gpu):
    _check(W.make_rule(57, 8000, 600, 64, 64, np.int32, dup_frac=0.1, missing_frac=0.05, sparse_keys=True))
    for n in (1, 33):
        _check(W.make_rule(58, n, 50, 64, 64, np.int32))


def test_pushdown_relu_mask_feeds_the_backward(gpu):
    rel = W.make_rule(59, 20_000, 2500, 64, 64, np.int32, src_dist="zipf", src_s=1.2, act="relu")
    keys, out, plan, t = run_rule(rel, flags=PD | R.FLAG_RELU_MASK, z_dtype=torch.bfloat16)
    dout = np.random.default_rng(3).standard_normal(out.shape).astype(np.float32)
    dW, db, dz, _ = plan.backward(to_dev(dout), t["z"], t["W"], t["b"], t["r"])
    torch.cuda.synchronize()
    brs = [OBr(b.src, b.dst, bf16_round(b.W), b.b, None) for b in rel.branches]
    oW, ob, oz, _ = O.rule_backward(rel.h_ids, bf16_round(rel.z), brs, keys, dout, act=rel.act)
    assert rel_frob(dW[0].cpu().numpy(), oW[0]) <= 2e-2
    assert rel_frob(db[0].cpu().numpy(), ob[0]) <= 1e-5
    assert rel_frob(dz.cpu().numpy(), oz) <= 2e-2


def test_pushdown_rejects_per_tuple_embedding(gpu):
    rel = W.make_rule(60, 1000, 100, 64, 64, np.int32, d_r=64)
    with pytest.raises(R.RelnnError):
        run_rule(rel, flags=PD, z_dtype=torch.bfloat16)


@pytest.mark.parametrize("d_out", [64, 128])
def test_pushdown_unaligned_output_takes_warp_form(gpu, d_out):
    """An output 4 bytes off a 16-byte boundary cannot take the half-warp walk (16-byte row stores):
    the one-range-per-warp walk runs instead and gives the same rows."""
    rel = W.make_rule(61, 20_000, 1500, 64, d_out, np.int32, src_dist="zipf", src_s=1.2)
    br = rel.branches[0]
    plan = R.RulePlan(to_dev(rel.h_ids), [(to_dev(br.src), to_dev(br.dst))], 64, d_out, flags=PD)
    buf = torch.empty(plan.n_out * d_out + 1, dtype=torch.float32, device="cuda")
    out = buf[1:].view(plan.n_out, d_out)
    assert out.data_ptr() % 16 == 4
    plan.forward(to_dev(rel.z, torch.bfloat16), [to_dev(br.W)], [to_dev(br.b)], out=out)
    torch.cuda.synchronize()
    plan.check()
    _, oo, _ = oracle_rule(rel, round_z=True, round_w=True)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-4
    _, out_a, _, _ = run_rule(rel, flags=PD, z_dtype=torch.bfloat16)
    assert rel_frob(out.cpu().numpy(), out_a) <= 1e-5
