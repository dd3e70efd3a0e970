"""relnn_rule_forward_noalloc against relnn_rule_forward (FP32 form) and the FP64 oracle on the same rule.

The allocation-free entry point serves callers that cannot call cudaMalloc (a fixed device-memory
budget handed to another allocator, or a loop that cannot afford an allocation's synchronisation).
It takes the join output already grouped by output row; here that grouping is built on the host
from the oracle's join, and the result must match the regular entry point and the oracle within the
FP32-form tolerance on two calls in a row (the second call reuses the shared scratch array). One
case puts most tuples in a few output rows, so rows cover whole 32-tuple tiles and cross many tile
boundaries (the fix-up's chain), and one sits at the documented width limit (2d = 1024)."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import rel_frob, run_rule

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def _grouped_join(rel):
    """Matched tuples of the (single-branch) rule grouped by output key, as int32 device arrays."""
    br = rel.branches[0]
    e, hs, hd = O.join(br.src, br.dst, rel.h_ids)
    keys = br.dst[e]
    order = np.lexsort((e, keys))  # by output key, then E row
    out_keys, seg = np.unique(keys[order], return_inverse=True)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    return dev(hs[order]), dev(hd[order]), dev(seg.reshape(-1)), out_keys


@pytest.mark.parametrize("act,shape", [("none", "uniform"), ("relu", "uniform"), ("none", "heavy"),
                                       ("relu", "heavy"), ("none", "widest")])
def test_noalloc_matches_rule_forward_twice(gpu, act, shape):
    if shape == "uniform":
        rel = W.make_rule(31, 6000, 400, 16, 24, np.int32, act=act)
    elif shape == "heavy":
        # Zipf(2.0) dst over 300 keys: the top rows hold thousands of tuples (hundreds of tiles)
        rel = W.make_rule(32, 20_000, 300, 16, 24, np.int32, act=act, dst_dist="zipf", dst_s=2.0)
    else:
        rel = W.make_rule(33, 3000, 200, 512, 32, np.int32, act=act)  # 2d = 1024: 128 KB of shared memory
    hs, hd, seg, out_keys = _grouped_join(rel)
    ok, oo, _ = O.rule_forward(rel.h_ids, rel.z, rel.branches, act=rel.act)
    assert np.array_equal(ok, out_keys)
    out_ref = None
    if shape != "widest":  # the regular FP32 form tiles at most 220 KB of shared memory
        keys_ref, out_ref, plan, t = run_rule(rel)  # the existing entry point (plan + forward)
        assert np.array_equal(out_keys, keys_ref)
    br = rel.branches[0]
    z = torch.from_numpy(rel.z).cuda()
    Wt, bt = torch.from_numpy(br.W).cuda(), torch.from_numpy(br.b).cuda()
    a = R.ACT_RELU if act == "relu" else R.ACT_NONE
    for _ in range(2):
        out = torch.full((len(out_keys), Wt.shape[0]), float("nan"), device="cuda")
        R.rule_forward_noalloc(z, hs, hd, seg, Wt, bt, out, act=a)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        if out_ref is not None:
            assert rel_frob(got, out_ref) <= FP32_TOL
        assert rel_frob(got, oo) <= FP32_TOL


def test_noalloc_rejects_oversized_call(gpu):
    z = torch.zeros((4, 16), device="cuda")
    idx = torch.zeros(4, dtype=torch.int32, device="cuda")
    Wt = torch.zeros((256, 32), device="cuda")
    out = torch.zeros((1, 256), device="cuda")
    L = R.lib()
    # 2M tuples x 256 outputs would need ~64 MB of partial sums: refused before any device work
    st = L.relnn_rule_forward_noalloc(R._ptr(z), 16, R._ptr(idx), R._ptr(idx), R._ptr(idx), 2_000_000,
                                      R._ptr(Wt), None, 256, R.ACT_NONE, R._ptr(out), R._stream())
    assert st == 3  # RELNN_ENOSPC
    assert b"scratch" in L.relnn_last_error()
