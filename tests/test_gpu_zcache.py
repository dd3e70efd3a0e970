"""GPU tests of the plan's bf16 copy of an f32 embedding table (relnn_plan_set_z_version): with the
same nonzero version at the same address the copy is reused (one conversion launch fewer per call)
and results do not change; "auto" versions follow the tensor's in-place updates, so a modified table
is converted again and the result matches the FP64 oracle on the new values."""
import numpy as np
import pytest
import torch

from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import oracle_rule, rel_frob, to_dev

pytestmark = pytest.mark.gpu


def _setup(seed):
    rel = W.make_rule(seed, 20_000, 1500, 64, 64, np.int32, src_dist="zipf", src_s=1.2)
    br = rel.branches[0]
    plan = R.RulePlan(to_dev(rel.h_ids), [(to_dev(br.src), to_dev(br.dst))], 64, 64, flags=R.FLAG_BF16)
    return rel, plan, to_dev(rel.z, torch.float32), to_dev(br.W), to_dev(br.b)


def _launches(fn):
    torch.cuda.synchronize()
    n0 = R.launch_count()
    out = fn()
    torch.cuda.synchronize()
    return R.launch_count() - n0, out


def test_same_version_reuses_the_copy(gpu):
    rel, plan, z, Wt, bt = _setup(131)
    plan.forward(z, [Wt], [bt])  # the plan's one-time forward set-up (virtual rows, packed W)
    n_none, out0 = _launches(lambda: plan.forward(z, [Wt], [bt]).clone())
    n_conv, out1 = _launches(lambda: plan.forward(z, [Wt], [bt], z_version=7).clone())
    n_reuse, out2 = _launches(lambda: plan.forward(z, [Wt], [bt], z_version=7).clone())
    assert n_conv == n_none  # first call with this version: converted
    assert n_reuse == n_conv - 1
    assert torch.equal(out0, out1) and torch.equal(out0, out2)
    # the backward of the same step reuses the forward's conversion
    dout = torch.randn_like(out0)
    plan.backward(dout, z, [Wt], [bt])  # the backward's one-time set-up (src order)
    n_b0, g0 = _launches(lambda: plan.backward(dout, z, [Wt], [bt]))
    plan.forward(z, [Wt], [bt], z_version=8)
    n_b1, g1 = _launches(lambda: plan.backward(dout, z, [Wt], [bt], z_version=8))
    assert n_b1 == n_b0 - 1
    assert torch.equal(g0[2], g1[2]) and torch.equal(g0[0][0], g1[0][0])
    _, oo, _ = oracle_rule(rel, round_z=True, round_w=True)
    assert rel_frob(out0.cpu().numpy(), oo) <= 1e-4


def test_auto_version_follows_inplace_updates(gpu):
    rel, plan, z, Wt, bt = _setup(132)
    out1 = plan.forward(z, [Wt], [bt], z_version="auto").cpu().numpy()
    _, oo, _ = oracle_rule(rel, round_z=True, round_w=True)
    assert rel_frob(out1, oo) <= 1e-4
    z.mul_(-0.5)  # in place: the tensor's version counter moves
    out2 = plan.forward(z, [Wt], [bt], z_version="auto").cpu().numpy()
    rel.z = (rel.z.astype(np.float32) * np.float32(-0.5))
    _, oo2, _ = oracle_rule(rel, round_z=True, round_w=True)
    assert rel_frob(out2, oo2) <= 1e-4
    # a new tensor at (possibly) the same address gets a new version
    z2 = z.clone()
    del z
    out3 = plan.forward(z2, [Wt], [bt], z_version="auto").cpu().numpy()
    assert rel_frob(out3, oo2) <= 1e-4
