"""Helpers for the GPU parity tests: move synthetic relations to the device, run the library, and run
the FP64 oracle on exactly the same (rounded) inputs."""
from __future__ import annotations

import numpy as np
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R


class OBr:
    def __init__(self, src, dst, W, b, r=None, filters=None):
        self.src, self.dst, self.W, self.b, self.r, self.filters = src, dst, W, b, r, filters


def rel_frob(got: np.ndarray, ref: np.ndarray) -> float:
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(np.asarray(got, np.float64) - ref) / (den if den > 0 else 1.0))


def bf16_round(a: np.ndarray) -> np.ndarray:
    """float32 -> bf16 -> float32 (round to nearest even, via torch on the CPU)."""
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def to_dev(a, dtype=None, dev="cuda"):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev)


def run_rule(rel, flags=0, z_dtype=torch.float32, r_dtype=torch.float32, w_dtype=torch.float32,
             want_plan=False, filters=None):
    """Plan + forward on the device. Returns (keys np, out np, plan, device tensors)."""
    dev = "cuda"
    h = to_dev(rel.h_ids)
    z = to_dev(rel.z, z_dtype)
    brs = [(to_dev(b.src), to_dev(b.dst)) for b in rel.branches]
    d_r = 0 if rel.branches[0].r is None else rel.branches[0].r.shape[1]
    identity = rel.branches[0].W is None
    if identity:
        flags |= R.FLAG_IDENTITY
    d_out = 0 if identity else rel.branches[0].W.shape[0]
    act = R.ACT_RELU if rel.act == "relu" else R.ACT_NONE
    plan = R.RulePlan(h, brs, rel.z.shape[1], d_out, act=act, flags=flags, d_r=d_r, filters=filters)
    W = None if identity else [to_dev(b.W, w_dtype) for b in rel.branches]
    bb = None if identity else [to_dev(b.b) for b in rel.branches]
    r = None if d_r == 0 else [to_dev(b.r, r_dtype) for b in rel.branches]
    out = plan.forward(z, W, bb, r)
    torch.cuda.synchronize()
    plan.check()
    keys = plan.out_keys().cpu().numpy()
    res = (keys, out.cpu().numpy(), plan, dict(h=h, z=z, W=W, b=bb, r=r, brs=brs))
    return res


def oracle_rule(rel, round_z=False, round_r=False, round_w=False, join_dst=True, concat_dst=True, filters=None):
    """FP64 oracle on the same inputs, optionally with the bf16 rounding the device applies."""
    z = bf16_round(rel.z) if round_z else rel.z
    brs = []
    for b in rel.branches:
        W = None if b.W is None else (bf16_round(b.W) if round_w else b.W)
        r = None if b.r is None else (bf16_round(b.r) if round_r else b.r)
        brs.append(OBr(b.src, b.dst, W, b.b, r, filters[len(brs)] if filters else None))
    keys, out, sizes = O.rule_forward(rel.h_ids, z, brs, act=rel.act, join_dst=join_dst, concat_dst=concat_dst)
    return keys, out, sizes
