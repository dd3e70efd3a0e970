"""Autotuner for the fused forward's tile shape (a host-side driver of library calls only).

The fused tcgen05 forward cuts the matched tuples into 256-tuple tiles, or 128-tuple tiles with
RELNN_FLAG_TILE128. Small batches have too few 256-tuple tiles to occupy every SM, so smaller tiles
win below some size; the crossover depends on d, d_out and the device. tune_tile128_below() times
plan + forward of synthetic serving-shaped rules over a grid of sizes with both tile shapes and
returns the smallest size from which 256-tuple tiles are at least as fast; the result is cached in a
JSON file keyed by (device name, d, d_out).
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import relnn as R
from . import workloads as W

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "relnn_b300", "autotune.json")


def _time_rule(h, z, src, dst, Wt, bt, d, d_out, flags, reps=5):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p = R.RulePlan(h, [(src, dst)], d, d_out, flags=flags)
    out = torch.empty((max(p.n_out, 1), d_out), dtype=torch.float32, device=h.device)
    p.forward(z, [Wt], [bt], out=out)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        p.forward(z, [Wt], [bt], out=out)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_tile128_below(d: int = 64, d_out: int = 64, sizes=None, cache: str | None = DEFAULT_CACHE,
                       seed: int = 0) -> int:
    """E-tuple count below which 128-tuple tiles are used (0 = never)."""
    dev = torch.cuda.current_device()
    key = f"{torch.cuda.get_device_name(dev)}|d={d}|d_out={d_out}"
    if cache and os.path.exists(cache):
        try:
            got = json.load(open(cache)).get(key)
            if got is not None:
                return int(got)
        except (OSError, ValueError):
            pass
    sizes = sizes or [4_000, 16_000, 40_000, 100_000, 250_000, 600_000]
    rng = np.random.default_rng(seed)
    Wt = torch.from_numpy((rng.standard_normal((d_out, 2 * d)) / np.sqrt(2 * d)).astype(np.float32)).cuda()
    bt = torch.zeros(d_out, device="cuda")
    threshold = 0
    for n in sizes:
        keys, src, dst, z = W.serving_query(seed, n, n, d)
        h, s, t = (torch.from_numpy(x).cuda() for x in (keys, src, dst))
        zz = torch.from_numpy(z).cuda().to(torch.bfloat16)
        t256 = _time_rule(h, zz, s, t, Wt, bt, d, d_out, R.FLAG_BF16)
        t128 = _time_rule(h, zz, s, t, Wt, bt, d, d_out, R.FLAG_BF16 | R.FLAG_TILE128)
        if t128 < t256:
            threshold = n + 1
    if cache:
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            data = json.load(open(cache)) if os.path.exists(cache) else {}
            data[key] = threshold
            json.dump(data, open(cache, "w"), indent=1)
        except (OSError, ValueError):
            pass
    return threshold
