"""GPU tests of the plan's counting group-by (RELNN_TUNE_GROUP_SORT = 1, a choice for one branch
over unique H keys; the default 0 is the stable radix sort): output keys bit-exact and outputs equal to the radix-sort grouping (E order
within a group) up to the order of f32 additions and to the FP64 oracle at the BF16 bars; groups
of one lane's size (<= 32 tuples), of a block's (33..4096) and larger ones (the plan then falls back to
the radix sort); two plans built from the same relation give bit-identical results."""
import numpy as np
import pytest
import torch

from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import oracle_rule, rel_frob, to_dev

pytestmark = pytest.mark.gpu


def _plan_fwd(rel, group_sort, flags=R.FLAG_BF16):
    saved = R.tune_get(R.TUNE_GROUP_SORT)
    R.tune_set(R.TUNE_GROUP_SORT, group_sort)
    try:
        br = rel.branches[0]
        plan = R.RulePlan(to_dev(rel.h_ids), [(to_dev(br.src), to_dev(br.dst))], rel.z.shape[1], br.W.shape[0],
                          flags=flags)
        out = plan.forward(to_dev(rel.z, torch.bfloat16), [to_dev(br.W)], [to_dev(br.b)])
        torch.cuda.synchronize()
        plan.check()
        return plan.out_keys().cpu().numpy(), out.cpu().numpy(), plan
    finally:
        R.tune_set(R.TUNE_GROUP_SORT, saved)


@pytest.mark.parametrize("case", ["lane", "block", "fallback", "zipf_src"])
def test_counting_matches_radix_and_oracle(gpu, case):
    if case == "lane":      # ~12 tuples per group
        rel = W.make_rule(141, 60_000, 5000, 64, 64, np.int64)
    elif case == "block":   # ~300 tuples per group
        rel = W.make_rule(142, 150_000, 500, 64, 64, np.int32)
    elif case == "fallback":  # one group holds far more than 4096 tuples
        rel = W.make_rule(143, 100_000, 3000, 64, 64, np.int32, dst_dist="zipf", dst_s=2.0)
    else:
        rel = W.make_rule(144, 80_000, 4000, 128, 64, np.int32, src_dist="zipf", src_s=1.3)
    k0, o0, _ = _plan_fwd(rel, 1)
    k1, o1, _ = _plan_fwd(rel, 0)
    ok, oo, _ = oracle_rule(rel, round_z=True, round_w=True)
    assert np.array_equal(k0, ok) and np.array_equal(k1, ok)
    # a different f32 summation order inside a group; the sums reach the tensor cores as bf16 pairs
    assert rel_frob(o0, o1.astype(np.float64)) <= 1e-5
    assert rel_frob(o0, oo) <= 1e-4


def test_counting_is_deterministic_across_plans(gpu):
    rel = W.make_rule(145, 120_000, 2000, 64, 64, np.int32, src_dist="zipf", src_s=1.1)
    _, o0, _ = _plan_fwd(rel, 1)
    _, o1, _ = _plan_fwd(rel, 1)
    assert np.array_equal(o0, o1)


def test_counting_backward_matches_radix(gpu):
    rel = W.make_rule(146, 50_000, 3000, 64, 64, np.int32, src_dist="zipf", src_s=1.2)
    grads = []
    for gs in (1, 0):
        _, out, plan = _plan_fwd(rel, gs)
        br = rel.branches[0]
        dout = to_dev(np.random.default_rng(5).standard_normal(out.shape).astype(np.float32))
        dW, db, dz, _ = plan.backward(dout, to_dev(rel.z, torch.bfloat16), [to_dev(br.W)], [to_dev(br.b)])
        torch.cuda.synchronize()
        grads.append((dW[0].cpu().numpy(), db[0].cpu().numpy(), dz.cpu().numpy()))
    for a, b in zip(*grads):
        assert rel_frob(a, b.astype(np.float64)) <= 1e-5
