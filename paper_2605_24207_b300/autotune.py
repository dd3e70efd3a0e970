"""Autotuner (a host-side driver of library calls only; every timed step runs in librelnn).

Two tuners, both caching their choice in a JSON file keyed by device name and shape:

tune_rule() picks, per (d, d_out, embedding dtype, Kahan, tuple-count bucket), the evaluation form of
a BF16 linear rule and the knobs of the kernels it runs:
  - form: aggregate-first (sum each output row's Concat rows, then one GEMM row per output row; the
    default for linear SUM rules), per-tuple (the Linear on every matched tuple, RELNN_FLAG_PER_TUPLE)
    or push-down (the Linear once per H row, RELNN_FLAG_PUSHDOWN);
  - for the aggregate-first GEMM: tile rows (RELNN_TUNE_AGG_ROWS), pipeline stages
    (RELNN_TUNE_AGG_STAGES) and epilogue warps (RELNN_TUNE_AGG_EPI: 4 or 8, two kernel instances),
    or the fused kernel whose producer warps write the sums into its stages (RELNN_TUNE_AGG_FUSE);
  - with Kahan summation, the degree below which rows are summed plainly (RELNN_TUNE_KAHAN_MIN);
  - for the plan, the radix digit width of the group sort (RELNN_TUNE_SORT_BITS), or the counting
    group-by instead of the radix sort (RELNN_TUNE_GROUP_SORT).
It times forward + backward (or forward alone) on a synthetic relation of the bucket's shape and
keeps the fastest; apply() sets the knobs and returns the flags to add.

tune_tile128_below() times the per-tuple fused forward's 128- vs 256-tuple tiles over a grid of
sizes and returns the smallest size from which 256-tuple tiles are at least as fast.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import relnn as R
from . import workloads as W

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "relnn_b300", "autotune.json")

# the library's defaults (what every knob is when nothing is tuned)
DEFAULTS = {"form": "agg", "agg_rows": 0, "agg_stages": 0, "agg_epi": 8, "kahan_min": 33, "sort_bits": 8,
            "tile128": False, "group_sort": 0, "agg_fuse": 0}
_FORM_FLAG = {"agg": 0, "per_tuple": R.FLAG_PER_TUPLE, "pushdown": R.FLAG_PUSHDOWN}


def _cache_get(cache, key):
    if cache and os.path.exists(cache):
        try:
            return json.load(open(cache)).get(key)
        except (OSError, ValueError):
            return None
    return None


def _cache_put(cache, key, value):
    if not cache:
        return
    try:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        data = json.load(open(cache)) if os.path.exists(cache) else {}
        data[key] = value
        json.dump(data, open(cache, "w"), indent=1)
    except (OSError, ValueError):
        pass


def apply(cfg: dict) -> int:
    """Sets the process-wide knobs of ``cfg`` (missing entries: library defaults) and returns the
    flags its form adds to RELNN_FLAG_BF16."""
    c = dict(DEFAULTS, **(cfg or {}))
    R.tune_set(R.TUNE_AGG_ROWS, int(c["agg_rows"]))
    R.tune_set(R.TUNE_AGG_STAGES, int(c["agg_stages"]))
    R.tune_set(R.TUNE_AGG_EPI, int(c["agg_epi"]))
    R.tune_set(R.TUNE_KAHAN_MIN, int(c["kahan_min"]))
    R.tune_set(R.TUNE_SORT_BITS, int(c["sort_bits"]))
    R.tune_set(R.TUNE_GROUP_SORT, int(c["group_sort"]))
    R.tune_set(R.TUNE_AGG_FUSE, int(c["agg_fuse"]))
    return _FORM_FLAG[c["form"]] | (R.FLAG_TILE128 if c["tile128"] else 0)


def size_bucket(n_tuples: int) -> int:
    """Tuple-count bucket: powers of 4 (1k-4k, 4k-16k, ...)."""
    return int(np.floor(np.log2(max(int(n_tuples), 1)) / 2.0))


def _event_ms(fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def candidates(kahan: bool, linear: bool = True, pushdown: bool = True):
    """The configurations tune_rule() times: the per-tuple form with 256- and 128-tuple tiles, the
    push-down form, and (linear rules: no activation, no per-tuple embedding) the aggregate-first
    form over its GEMM's knobs."""
    out = [dict(DEFAULTS, form="per_tuple"), dict(DEFAULTS, form="per_tuple", tile128=True)]
    if pushdown:
        out.append(dict(DEFAULTS, form="pushdown"))
    if not linear:
        return out
    for rows in (0, 32, 64):
        for stages in (0, 2, 3):
            for epi in (4, 8):
                for kmin in ((0, 33) if kahan else (33,)):
                    out.append(dict(DEFAULTS, agg_rows=rows, agg_stages=stages, agg_epi=epi, kahan_min=kmin))
    # the fused forward (measured 1.9x slower than the two kernels on the single-rule relation: its
    # producer warps cannot keep enough row loads in flight within one CTA), timed once
    out.append(dict(DEFAULTS, agg_fuse=1))
    return out


def tune_rule(d: int, d_out: int, n_tuples: int, n_keys: int | None = None, z_dtype=torch.bfloat16,
              kahan: bool = False, backward: bool = True, cache: str | None = DEFAULT_CACHE, seed: int = 0,
              reps: int = 5, rel=None, act: int = 0) -> dict:
    """Fastest configuration (a dict for apply(), plus its time and the defaults' time) for a BF16
    SUM rule of this shape (act: R.ACT_NONE or R.ACT_RELU); ``rel`` (a workloads.Relations, first
    branch) replaces the synthetic relation."""
    dev = torch.cuda.current_device()
    zname = "bf16" if z_dtype == torch.bfloat16 else "f32"
    d_r = 0 if rel is None or rel.branches[0].r is None else rel.branches[0].r.shape[1]
    key = (f"rule|{torch.cuda.get_device_name(dev)}|d={d}|d_out={d_out}|d_r={d_r}|act={act}|z={zname}"
           f"|kahan={int(kahan)}|bwd={int(backward)}|bucket={size_bucket(n_tuples)}")
    got = _cache_get(cache, key)
    if got is not None:
        return got
    if rel is None:
        n_keys = n_keys or max(1, n_tuples // 16)
        rel = W.make_rule(seed, n_tuples, n_keys, d, d_out, np.int32, src_dist="zipf", src_s=1.1)
    br = rel.branches[0]
    h, s_, t_ = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (rel.h_ids, br.src, br.dst))
    z = torch.from_numpy(rel.z).cuda().to(z_dtype)
    Wt = torch.from_numpy(br.W).cuda()
    bt = torch.from_numpy(br.b).cuda()
    rr = [torch.from_numpy(br.r).cuda().to(torch.bfloat16)] if d_r else None
    base = R.FLAG_BF16 | (R.FLAG_KAHAN if kahan else 0) | (R.FLAG_RELU_MASK if act and backward else 0)
    linear = act == 0 and d_r == 0
    saved = {k: R.tune_get(k) for k in (R.TUNE_AGG_ROWS, R.TUNE_AGG_STAGES, R.TUNE_AGG_EPI, R.TUNE_KAHAN_MIN,
                                        R.TUNE_SORT_BITS)}
    results = []
    try:
        plans = {}
        for cfg in candidates(kahan, linear=linear, pushdown=d_r == 0):
            flags = base | apply(cfg)
            try:
                if flags not in plans:
                    plans[flags] = R.RulePlan(h, [(s_, t_)], d, d_out, act=act, flags=flags, d_r=d_r)
            except R.RelnnError:
                continue
            p = plans[flags]
            out = torch.empty((max(p.n_out, 1), d_out), dtype=torch.float32, device="cuda")
            dout = torch.randn_like(out)

            def step():
                p.forward(z, [Wt], [bt], r=rr, out=out, z_version=1)
                if backward:
                    p.backward(dout, z, [Wt], [bt], r=rr, z_version=1)
            try:
                results.append((_event_ms(step, reps), cfg))
            except R.RelnnError:
                continue  # a form this shape does not support
        # the plan's sort digit width, timed on plan builds with the best numeric configuration
        best_ms, best = min(results, key=lambda x: x[0])
        plan_t = []
        for bits, gsort in ((7, 0), (8, 0), (10, 0), (11, 0), (8, 1)):
            flags = base | apply(dict(best, sort_bits=bits, group_sort=gsort))
            plan_t.append((_event_ms(lambda: R.RulePlan(h, [(s_, t_)], d, d_out, act=act, flags=flags, d_r=d_r), 3),
                           bits, gsort))
        plan_ms, bits, gsort = min(plan_t)
        # the library's own choice without tuning: aggregate-first for linear rules, else per-tuple
        default_cfg = dict(DEFAULTS) if linear else dict(DEFAULTS, form="per_tuple")
        default_ms = next((ms for ms, c in results if c == default_cfg), None)
        choice = dict(best, sort_bits=bits, group_sort=gsort, ms=best_ms, default_ms=default_ms, plan_ms=plan_ms,
                      default_plan_ms=next((ms for ms, b, g in plan_t if b == DEFAULTS["sort_bits"] and g == 0), None))
    finally:
        for k, v in saved.items():
            R.tune_set(k, v)
    _cache_put(cache, key, choice)
    return choice


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
