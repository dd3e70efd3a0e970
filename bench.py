#!/usr/bin/env python
"""Benchmark of one RelaNN rule evaluation on B300 (prints ONE JSON line on rank 0).

Workload (default): the single rule at scale -- E has 16M tuples over 1M int64 keys, src ~ Zipf(1.1),
dst uniform; H(id; z) with z bf16[128]; Linear 256 -> 128 on tcgen05 (bf16 in, f32 accumulate);
SUM group-by dst. Inputs are seeded synthetic relations (no dataset).

A step is one pass of the whole hot path over the batch: the content track (join build on H.id,
probe of src and dst, grouping by dst: relnn_rule_plan) followed by the fused gather -> Concat ->
Linear -> SUM forward (relnn_rule_forward). `value` = matched (join-output) tuples per second,
summed over ranks. Extra keys report the warm forward (content cached, as the paper caches it
across iterations) and the warm forward+backward.

--impl reference times the FP64 CPU oracle on the host cores instead (bounded sample per step).
Multi-GPU: the rule does not shard here; N ranks run N independent replicas (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rule tuples/s"
UNIT = "tuples/s"
# DRAM bytes per launch of fwd_tc_kernel from ncu (dram__bytes_read.sum + dram__bytes_write.sum),
# scaled to the 16M-tuple launch; None until a capture of the current kernel exists.
NCU_TRAFFIC_PER_LAUNCH = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="relnn", choices=["relnn", "reference"])
    ap.add_argument("--n-tuples", type=int, default=16_000_000)
    ap.add_argument("--n-keys", type=int, default=1_000_000)
    ap.add_argument("--cpu-sample", type=int, default=1_000_000, help="tuples in the CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the warm forward/backward extras")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait(timeout=10)
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(args, seed):
    from paper_2605_24207_b300 import workloads as W
    return W.config2(seed=seed, n_tuples=args.n_tuples, n_keys=args.n_keys)


def cpu_oracle_rate(rel, n_sample: int, seed: int = 1):
    """FP64 oracle (as it stands) on the first n_sample E rows with the full H; tuples/s and info."""
    import torch
    from oracle import relnn_oracle as O
    br = rel.branches[0]
    n = min(n_sample, br.src.size)

    class B:
        pass
    ob = B()
    ob.src, ob.dst, ob.r = br.src[:n], br.dst[:n], None
    ob.W = torch.from_numpy(br.W).to(torch.bfloat16).float().numpy()
    ob.b = br.b
    z = torch.from_numpy(rel.z).to(torch.bfloat16).float().numpy()
    t0 = time.perf_counter()
    _, _, sizes = O.rule_forward(rel.h_ids, z, [ob])
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return sizes[0] / dt, sizes[0], dt, cores


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, rank 0 only, bounded sample per step."""
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
    rel = make_workload(args, 0)
    sample = min(args.cpu_sample // 4, rel.branches[0].src.size)
    for _ in range(args.warmup):
        cpu_oracle_rate(rel, sample)
    tot_t, tot_n = 0.0, 0
    for _ in range(args.steps):
        rate, n, dt, cores = cpu_oracle_rate(rel, sample)
        tot_t += dt
        tot_n += n
    value = tot_n / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"single rule, E {args.n_tuples} tuples over {args.n_keys} int64 keys, "
                               f"z bf16[128], Linear 256->128, SUM by dst (oracle on {sample}-tuple samples)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {sample} E rows with the full H per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2605_24207_b300 import relnn as R

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    rel = make_workload(args, 0)
    br = rel.branches[0]
    # device-resident inputs
    h = torch.from_numpy(rel.h_ids).to(dev)
    src = torch.from_numpy(br.src).to(dev)
    dst = torch.from_numpy(br.dst).to(dev)
    z = torch.from_numpy(rel.z).to(dev).to(torch.bfloat16)
    Wt = torch.from_numpy(br.W).to(dev)
    bt = torch.from_numpy(br.b).to(dev)
    d, d_out = rel.z.shape[1], br.W.shape[0]
    flags = R.FLAG_BF16
    plan0 = R.RulePlan(h, [(src, dst)], d, d_out, flags=flags)
    matched, n_out = plan0.n_matched, plan0.n_out
    out = torch.empty((max(n_out, 1), d_out), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        p = R.RulePlan(h, [(src, dst)], d, d_out, flags=flags)
        p.forward(z, [Wt], [bt], out=out)
        return p

    # ---------------------------------------------------------------- timed region (device inputs)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    clk = Clocks(local)
    R.profile_reset()
    R.profile_enable(True)
    n_launch0 = R.launch_count()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t_wall0 = time.perf_counter()
    keep = None
    for _ in range(args.steps):
        keep = step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    gpu_launches = R.launch_count() - n_launch0
    R.profile_enable(False)
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    fwd_ms, fwd_n = R.profile_read(R.PROF_FWD_TC)
    plan_ms, plan_n = R.profile_read(R.PROF_PLAN)
    fix_ms, fix_n = R.profile_read(R.PROF_FIXUP)
    keep.check()
    t_step = ms / args.steps
    if world > 1:
        tt = torch.tensor([t_step], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())
    value = world * matched / (t_step * 1e-3)

    # ---------------------------------------------------------------- roofline of the fused kernel
    pk, pk_src = peaks()
    flops_per_launch = 2.0 * (2 * d) * d_out * matched
    fwd_avg_ms = fwd_ms / max(fwd_n, 1)
    achieved = flops_per_launch / (fwd_avg_ms * 1e-3) / 1e12
    peak = pk["bf16_tflops_sustained"]
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": NCU_TRAFFIC_PER_LAUNCH,
                "kernel": "fwd_tc_kernel", "peak_source": f"{pk_src} bf16 sustained",
                "kernel_ms": fwd_avg_ms}

    extras = {}
    if not args.no_extras:
        # warm forward (content cached) and warm forward + backward
        keep_plan = plan0
        for _ in range(3):
            keep_plan.forward(z, [Wt], [bt], out=out)
        torch.cuda.synchronize()
        e0.record(stream)
        reps = max(3, args.steps)
        for _ in range(reps):
            keep_plan.forward(z, [Wt], [bt], out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        warm_fwd_ms = e0.elapsed_time(e1) / reps
        dout = torch.ones_like(out[:n_out])
        keep_plan.backward(dout, z, [Wt], [bt])
        torch.cuda.synchronize()
        e0.record(stream)
        reps_b = 3
        for _ in range(reps_b):
            keep_plan.forward(z, [Wt], [bt], out=out)
            keep_plan.backward(dout, z, [Wt], [bt])
        e1.record(stream)
        torch.cuda.synchronize()
        warm_fb_ms = e0.elapsed_time(e1) / reps_b
        extras = {"warm_forward_tuples_per_s": matched / (warm_fwd_ms * 1e-3), "warm_forward_ms": warm_fwd_ms,
                  "warm_fwd_bwd_tuples_per_s": matched / (warm_fb_ms * 1e-3), "warm_fwd_bwd_ms": warm_fb_ms,
                  "plan_ms": plan_ms / max(plan_n, 1), "fixup_ms": fix_ms / max(fix_n, 1)}

    # ---------------------------------------------------------------- end to end (host buffers)
    hp = {k: v.cpu().pin_memory() for k, v in dict(h=h, src=src, dst=dst, z=z, W=Wt, b=bt).items()}
    dv = {k: torch.empty_like(v) for k, v in dict(h=h, src=src, dst=dst, z=z, W=Wt, b=bt).items()}
    out_host = torch.empty((n_out, d_out), dtype=torch.float32).pin_memory()
    keys_host = torch.empty(n_out, dtype=h.dtype).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in hp.values())
    d2h = out_host.numel() * 4 + keys_host.numel() * keys_host.element_size()

    def e2e_step():
        for k in hp:
            dv[k].copy_(hp[k], non_blocking=True)
        p = R.RulePlan(dv["h"], [(dv["src"], dv["dst"])], d, d_out, flags=flags)
        o = p.forward(dv["z"], [dv["W"]], [dv["b"]], out=out)
        out_host.copy_(o, non_blocking=True)
        keys_host.copy_(p.out_keys(), non_blocking=True)
        return p

    e2e_steps = max(3, args.steps // 2)
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    if world > 1:
        tt = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, n, dt, cores = cpu_oracle_rate(rel, args.cpu_sample)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {args.cpu_sample} of {args.n_tuples} E rows with the full H "
                         f"({n} matched tuples, {dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (seeded Zipf/uniform relations; no dataset)",
            "config": {"workload": f"single rule H'(dst; SUM Linear(Concat(z_src, z_dst))), E {args.n_tuples} "
                                   f"tuples over {args.n_keys} int64 keys (src Zipf 1.1, dst uniform), "
                                   f"z bf16[{d}], Linear {2 * d}->{d_out} bf16/f32-acc, SUM by dst; step = "
                                   f"plan (join build+probe+group) + fused forward",
                       "matched_tuples": matched, "out_keys": n_out,
                       "l2": "inputs larger than L2 (E 256 MB, H.z 256 MB, output 512 MB)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": world * matched / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "wall_s_timed": t_wall,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
