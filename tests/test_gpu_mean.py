"""GPU parity of the MEAN aggregator (alpha = SUM / |B_t| per output row, paper Sec. 2.2) against
the FP64 oracle: forward in the FP32 form (<= 1e-5), the BF16 form and the push-down (<= 2e-2, and
<= 1e-4 against the oracle on the same bf16-rounded operands); backward of both forms."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import OBr, bf16_round, rel_frob, run_rule, to_dev

pytestmark = pytest.mark.gpu


def _oracle(rel, round_=False, **kw):
    z = bf16_round(rel.z) if round_ else rel.z
    brs = [OBr(b.src, b.dst, bf16_round(b.W) if round_ else b.W, b.b, None) for b in rel.branches]
    return O.rule_forward(rel.h_ids, z, brs, act=rel.act, agg="mean", **kw)


def test_mean_fp32_form(gpu):
    rel = W.make_rule(61, 5000, 400, 16, 24, np.int32, act="relu", dst_dist="zipf", dst_s=1.3)
    keys, out, plan, _ = run_rule(rel, flags=R.FLAG_MEAN)
    ok, oo, sizes = _oracle(rel)
    assert np.array_equal(keys, ok) and plan.matched == sizes
    assert rel_frob(out, oo) <= 1e-5


@pytest.mark.parametrize("extra", [0, R.FLAG_PUSHDOWN])
def test_mean_bf16_forms(gpu, extra):
    rel = W.make_rule(62, 30_000, 2500, 64, 64, np.int32, src_dist="zipf", src_s=1.2, act="relu")
    keys, out, plan, _ = run_rule(rel, flags=R.FLAG_MEAN | R.FLAG_BF16 | extra, z_dtype=torch.bfloat16)
    ok, oo, _ = _oracle(rel)
    assert np.array_equal(keys, ok)
    assert rel_frob(out, oo) <= 2e-2
    _, oo_r, _ = _oracle(rel, round_=True)
    assert rel_frob(out, oo_r) <= 1e-4


@pytest.mark.parametrize("bf16", [False, True])
def test_mean_backward(gpu, bf16):
    rel = W.make_rule(63, 6000, 500, 16 if not bf16 else 64, 16 if not bf16 else 64, np.int32, act="relu",
                      dst_dist="zipf", dst_s=1.2)
    flags = R.FLAG_MEAN | ((R.FLAG_BF16 | R.FLAG_RELU_MASK) if bf16 else 0)
    zdt = torch.bfloat16 if bf16 else torch.float32
    keys, out, plan, t = run_rule(rel, flags=flags, z_dtype=zdt)
    dout = np.random.default_rng(6).standard_normal(out.shape).astype(np.float32)
    dW, db, dz, _ = plan.backward(to_dev(dout), t["z"], t["W"], t["b"], t["r"])
    torch.cuda.synchronize()
    z = bf16_round(rel.z) if bf16 else rel.z
    brs = [OBr(b.src, b.dst, bf16_round(b.W) if bf16 else b.W, b.b, None) for b in rel.branches]
    oW, ob, oz, _ = O.rule_backward(rel.h_ids, z, brs, keys, dout, act=rel.act, agg="mean")
    tol = 2e-2 if bf16 else 1e-5
    assert rel_frob(dW[0].cpu().numpy(), oW[0]) <= tol
    assert rel_frob(db[0].cpu().numpy(), ob[0]) <= 1e-5
    assert rel_frob(dz.cpu().numpy(), oz) <= tol


def test_mean_rejects_unions(gpu):
    rel = W.make_rule(64, 0, 300, 16, 16, np.int32, branch_tuples=[2000, 1000])
    with pytest.raises(R.RelnnError):
        run_rule(rel, flags=R.FLAG_MEAN)
