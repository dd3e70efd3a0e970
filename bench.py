#!/usr/bin/env python
"""Benchmark of RelaNN rule evaluation on B300; prints ONE JSON line on rank 0.

Default workload (--config c2): the single rule at scale -- E has 16M tuples over 1M int64 keys,
src ~ Zipf(1.1), dst uniform; H(id; z) with z bf16[128]; Linear 256 -> 128 on tcgen05 (bf16 in, f32
accumulate); SUM group-by dst. A step is one pass of the whole hot path over the batch: the content
track (join build on H.id, probe of src and dst, grouping by dst: relnn_rule_plan) and the fused
gather -> Concat -> Linear -> SUM forward (relnn_rule_forward). `value` = matched (join-output)
tuples per second, summed over ranks.

Other workloads (reported in the design notes, not the headline):
  --config c3   two stacked rules + SUM readout + MSE, one training step (forward + backward) with
                the content track cached across steps as the paper does; 4M tuples, 500k keys, d 64
  --config c4   union of 3 branches (2M / 1M / 0.5M tuples, 300k keys, z and r f32[64],
                Linear 192 -> 96 per branch), plan + forward, with and without Kahan summation

--impl reference times the FP64 CPU oracle on the host cores instead (a bounded sample per step).
Multi-GPU: the rule does not shard here; N ranks run N independent replicas (weak scaling).
All inputs are seeded synthetic relations (no dataset).
"""
from __future__ import annotations

import argparse
import datetime
import json
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="relnn", choices=["relnn", "reference"])
    ap.add_argument("--config", default="c2", choices=["c2", "c3", "c4", "c5", "c1b"])
    ap.add_argument("--instances", type=int, default=4096, help="c1b: independent small-rule instances")
    ap.add_argument("--n-queries", type=int, default=10_000, help="c5: queries in the serving trace")
    ap.add_argument("--cmp-queries", type=int, default=2_000, help="c5: queries for the torch comparator")
    ap.add_argument("--n-tuples", type=int, default=None, help="override the tuple count (c2, c3)")
    ap.add_argument("--n-keys", type=int, default=None, help="override the key count (c2, c3)")
    ap.add_argument("--cpu-sample", type=int, default=1_000_000, help="tuples in the CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip warm / comparator extras")
    ap.add_argument("--agg", default="sum", choices=["sum", "mean", "max"],
                    help="c2: aggregator of the rule (extras only with sum)")
    ap.add_argument("--no-tune", action="store_true", help="time the library defaults (no autotuning)")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="c2: skip the c3 / c4 / c1b / c5 records appended to the line")
    ap.add_argument("--no-serving", action="store_true", help="c2: skip the shortened c5 record")
    ap.add_argument("--sub-queries", type=int, default=2000, help="queries of the shortened c5 record")
    ap.add_argument("--workers", type=int, default=2,
                    help="c5: server worker threads (streams); 2 measured best: p99 4.3 ms against 10.3 ms with 4, "
                         "whose threads contend in the driver, at the same saturation rate")
    ap.add_argument("--sub-cmp-queries", type=int, default=300,
                    help="queries the torch comparator serves in the shortened c5 record")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class Clocks:
    """Clock sampler for a timed region: an NVML thread (the library nvidia-smi reads, queried
    in-process every 2 ms, so that even a region of a few tens of milliseconds holds samples) on the
    GPU with the CUDA device's PCI bus id; nvidia-smi every 20 ms if NVML is unavailable. Started
    before the warm-up; stop() keeps the samples taken inside [t0, t1]."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.samples, self.p, self.thread = [], None, None
        try:
            self._start_nvml(gpu_index)
            return
        except Exception:  # no NVML: the nvidia-smi command line of the profiling recipe
            self.thread = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.source = "nvidia-smi, 20 ms"
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def _start_nvml(self, gpu_index: int):
        """NVML through ctypes (libnvidia-ml.so.1, the driver's library; read-only queries)."""
        import ctypes as C
        import threading
        import torch
        nv = C.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit_v2 failed")
        pr = torch.cuda.get_device_properties(gpu_index)
        bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
        h = C.c_void_p()
        if nv.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(bus), C.byref(h)) != 0:
            raise OSError("no NVML device at " + bus.decode())
        SM = 1  # NVML_CLOCK_SM
        mx = C.c_uint()
        if nv.nvmlDeviceGetMaxClockInfo(h, SM, C.byref(mx)) != 0:
            raise OSError("nvmlDeviceGetMaxClockInfo failed")
        # clocks event reason bits (nvml.h): hw slowdown 0x8, sw thermal 0x20, hw thermal 0x40, sw power cap 0x4
        bits = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20, "sw_power_cap": 0x4}
        self.stop_ev = threading.Event()

        def run():
            clk, rs = C.c_uint(), C.c_ulonglong()
            while not self.stop_ev.is_set():
                if nv.nvmlDeviceGetClockInfo(h, SM, C.byref(clk)) != 0:
                    break
                if nv.nvmlDeviceGetCurrentClocksEventReasons(h, C.byref(rs)) != 0:
                    rs.value = 0
                self.samples.append((time.time(), float(clk.value), float(mx.value),
                                     {n for n, bt in bits.items() if rs.value & bt}))
                self.stop_ev.wait(0.002)
        self.source = f"NVML, 2 ms, GPU {bus.decode()}"
        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()
        time.sleep(0.01)

    def _smi_samples(self):
        self.p.terminate()
        self.p.wait(timeout=10)
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        parsed = []
        for r in rows:
            r = [x.strip() for x in r]
            try:
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                f_sm, f_mx = float(r[2]), float(r[3])
            except (ValueError, IndexError):
                continue
            parsed.append((ts, f_sm, f_mx, {n for n, v in zip(self.NAMES, r[6:10]) if v.lower().startswith("active")}))
        return parsed

    def stop(self, t0: float, t1: float):
        """Summary of the samples whose timestamp lies in [t0, t1] (time.time() seconds)."""
        if self.thread is not None:
            self.stop_ev.set()
            self.thread.join(timeout=5)
            parsed = list(self.samples)
        elif self.p is not None:
            parsed = self._smi_samples()
        else:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock source"], "samples": 0}
        inside = [p for p in parsed if t0 <= p[0] <= t1]
        out = {"source": self.source}
        if not inside:
            # a timed region shorter than the sampling period: the samples just before and after it
            before = [p for p in parsed if t0 - 0.25 <= p[0] < t0][-1:]
            after = [p for p in parsed if t1 < p[0] <= t1 + 0.25][:1]
            inside = before + after
            out["window"] = "nearest samples around the timed region"
        sm = [p[1] for p in inside]
        mx = [p[2] for p in inside]
        reasons = set().union(*[p[3] for p in inside]) if inside else set()
        out.update({"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                    "reasons": sorted(reasons), "samples": len(sm)})
        return out


def cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


class _Br:
    def __init__(self, src, dst, W, b, r=None):
        self.src, self.dst, self.W, self.b, self.r = src, dst, W, b, r


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()


# ===================================================================================== workloads
class C2:
    """Single rule at scale (the headline)."""
    name = "c2"

    def __init__(self, args):
        from paper_2605_24207_b300 import workloads as W
        self.n_tuples = args.n_tuples or 16_000_000
        self.n_keys = args.n_keys or 1_000_000
        self.agg = args.agg
        self.rel = W.config2(seed=0, n_tuples=self.n_tuples, n_keys=self.n_keys)

    def describe(self):
        A = self.agg.upper()
        return (f"single rule H'(dst; {A} Linear(Concat(z_src, z_dst))), E {self.n_tuples} tuples over "
                f"{self.n_keys} int64 keys (src Zipf 1.1, dst uniform), z bf16[128], Linear 256->128 "
                f"bf16/f32-acc, {A} by dst; step = plan (join build+probe+group) + fused forward")

    def to_device(self, dev):
        import torch
        from paper_2605_24207_b300 import relnn as R
        rel, br = self.rel, self.rel.branches[0]
        self.t = dict(h=torch.from_numpy(rel.h_ids).to(dev), src=torch.from_numpy(br.src).to(dev),
                      dst=torch.from_numpy(br.dst).to(dev), z=torch.from_numpy(rel.z).to(dev).to(torch.bfloat16),
                      W=torch.from_numpy(br.W).to(dev), b=torch.from_numpy(br.b).to(dev))
        self.d, self.d_out = rel.z.shape[1], br.W.shape[0]
        self.flags = R.FLAG_BF16 | {"sum": 0, "mean": R.FLAG_MEAN, "max": R.FLAG_MAX}[self.agg]
        p = R.RulePlan(self.t["h"], [(self.t["src"], self.t["dst"])], self.d, self.d_out, flags=self.flags)
        self.matched, self.n_out = p.n_matched, p.n_out
        self.plan0 = p
        self.out = torch.empty((max(self.n_out, 1), self.d_out), dtype=torch.float32, device=dev)
        # the SUM rule has no activation: the library evaluates it aggregate-first (one virtual row
        # per output row, or per 32 tuples of a heavier row)
        self.agg_form = self.agg == "sum"
        cnt = np.bincount(np.searchsorted(np.sort(self.rel.h_ids), self.rel.branches[0].dst),
                          minlength=self.rel.h_ids.size)
        self.n_vrows = int(np.maximum(1, (cnt[cnt > 0] + 31) // 32).sum())

    def tune(self):
        """The autotuner's choice for this rule (plan + forward of this relation), applied to the
        library's knobs and this workload's flags before anything is timed."""
        if self.agg != "sum":
            return None
        from paper_2605_24207_b300 import autotune as A
        c = A.tune_rule(self.d, self.d_out, self.n_tuples, rel=self.rel, backward=False, cache=None, reps=3)
        self.flags = (self.flags & ~(A.R.FLAG_PER_TUPLE | A.R.FLAG_PUSHDOWN | A.R.FLAG_TILE128)) | A.apply(c)
        return c

    def step(self):
        from paper_2605_24207_b300 import relnn as R
        t = self.t
        p = R.RulePlan(t["h"], [(t["src"], t["dst"])], self.d, self.d_out, flags=self.flags)
        p.forward(t["z"], [t["W"]], [t["b"]], out=self.out)
        # done with the plan: its memory is freed in the stream's order (relnn_plan_release), not
        # with a device-wide wait
        p.release()
        return None

    def kernels(self):
        """Library kernels of a step: id -> (name, algorithmic work per step, bound)."""
        from paper_2605_24207_b300 import relnn as R
        # aggregate-first form, two kernels (HBM): the gather-sum reads per matched tuple its 4-byte
        # src row index, per virtual row its 16-byte descriptor, each H row once (bf16) and writes
        # per virtual row the bf16 pair of its sums (2 x 2 x kpad bytes); the GEMM reads those pairs,
        # the descriptors and dst row indices (16 + 4 bytes per virtual row), the dst H row of each
        # output row (bf16) and writes each output row once (f32). Per-tuple form (tensor):
        # 2 d_in d_out FLOP per tuple.
        sb, gb = self.agg_bytes()
        if R.tune_get(R.TUNE_AGG_FUSE):
            # fused: one kernel, no pair buffer (its compulsory bytes + the descriptors and dst indices)
            return {R.PROF_AGG_FWD: ("agg_gemm_kernel fused (producer-warp gather-sum + tcgen05 GEMM)",
                                     float(self.forward_bytes() + 20 * self.n_vrows), "hbm"),
                    R.PROF_FWD_TC: ("fwd_tc_kernel", 2.0 * (2 * self.d) * self.d_out * self.matched, "tensor")}
        return {R.PROF_AGG_SUM: ("seg_sum_kernel (gather-sum)", float(sb), "hbm"),
                R.PROF_AGG_FWD: ("agg_gemm_kernel (TMA + tcgen05 GEMM)", float(gb), "hbm"),
                R.PROF_FWD_TC: ("fwd_tc_kernel", 2.0 * (2 * self.d) * self.d_out * self.matched, "tensor")}

    def ncu_traffic(self):
        """DRAM bytes (read + write) per launch of the step's kernels, from one ncu capture
        (dram__bytes_read.sum + dram__bytes_write.sum, one pass) of this workload at its default size:
        the two-kernel aggregate-first forward only; None for other sizes or forms."""
        from paper_2605_24207_b300 import relnn as R
        if (self.n_tuples, self.n_keys, self.agg) != (16_000_000, 1_000_000, "sum") or not self.agg_form:
            return None
        if self.flags & (R.FLAG_PER_TUPLE | R.FLAG_PUSHDOWN) or R.tune_get(R.TUNE_AGG_FUSE):
            return None
        return {R.PROF_AGG_SUM: 472_517_376 + 467_636_992, R.PROF_AGG_FWD: 788_276_992 + 462_302_208}

    def agg_bytes(self):
        """(gather-sum bytes, GEMM bytes) per forward."""
        n_h = int(self.t["h"].numel())
        kpad = (self.d + 63) // 64 * 64
        pair = 2 * 2 * kpad * self.n_vrows
        sb = 4 * self.matched + 16 * self.n_vrows + n_h * self.d * 2 + pair
        gb = pair + 20 * self.n_vrows + self.n_out * self.d * 2 + self.n_out * self.d_out * 4
        return sb, gb

    def forward_bytes(self):
        """Compulsory bytes of the whole forward (no intermediate): per matched tuple its src row and
        output row indices, each H row once, each output row once."""
        n_h = int(self.t["h"].numel())
        return 8 * self.matched + n_h * self.d * 2 + self.n_out * self.d_out * 4

    def e2e_setup(self):
        # two slots (device inputs, device output, pinned result, stream) used in turn, so that one
        # step's result copy back to the host overlaps the next step's input copy to the device
        import torch
        self.hp = {k: v.cpu().pin_memory() for k, v in self.t.items()}
        self.slots = []
        for _ in range(2):
            self.slots.append(dict(
                dv={k: torch.empty_like(v) for k, v in self.t.items()},
                out=torch.empty((max(self.n_out, 1), self.d_out), dtype=torch.float32, device=self.out.device),
                out_host=torch.empty((self.n_out, self.d_out), dtype=torch.float32).pin_memory(),
                keys_host=torch.empty(self.n_out, dtype=self.t["h"].dtype).pin_memory(),
                stream=torch.cuda.Stream()))
        self.e2e_i, self.e2e_n = 0, 0
        h2d = sum(v.numel() * v.element_size() for v in self.hp.values())
        sl = self.slots[0]
        d2h = sl["out_host"].numel() * 4 + sl["keys_host"].numel() * sl["keys_host"].element_size()
        return h2d, d2h

    def e2e_begin(self, stream, n_steps):
        for sl in self.slots:
            sl["stream"].wait_stream(stream)
        self.e2e_i, self.e2e_n = 0, n_steps

    def _copy_in(self, i):
        import torch
        sl = self.slots[i % 2]
        with torch.cuda.stream(sl["stream"]):
            for k in self.hp:
                sl["dv"][k].copy_(self.hp[k], non_blocking=True)

    def e2e_end(self, stream):
        for sl in self.slots:
            stream.wait_stream(sl["stream"])

    def e2e_step(self):
        # one step through the public API: inputs copied in from pinned host memory, plan + fused
        # forward, the output rows and keys copied back; the plan is released in stream order. The
        # next step's inputs are copied in (on the other slot's stream) before this step's plan
        # waits for its own, as a data loader prefetching one batch ahead would
        import torch
        from paper_2605_24207_b300 import relnn as R
        i = self.e2e_i
        self.e2e_i += 1
        if i == 0:
            self._copy_in(0)
        if i + 1 < self.e2e_n:
            self._copy_in(i + 1)
        sl = self.slots[i % 2]
        with torch.cuda.stream(sl["stream"]):
            dv = sl["dv"]
            p = R.RulePlan(dv["h"], [(dv["src"], dv["dst"])], self.d, self.d_out, flags=self.flags)
            o = p.forward(dv["z"], [dv["W"]], [dv["b"]], out=sl["out"])
            sl["out_host"].copy_(o, non_blocking=True)
            sl["keys_host"].copy_(p.out_keys(), non_blocking=True)
            p.release()
        return None

    def extras(self, timer, steps):
        """Warm forward (content cached), warm forward + backward, and the unfused FP32 torch form."""
        import torch
        if self.agg != "sum":
            return {}
        from paper_2605_24207_b300 import relnn as R
        t, p = self.t, self.plan0

        def ktime(fn, reps, kid):
            """(ms per call, ms per launch of library kernel kid)."""
            R.profile_reset()
            R.profile_enable(True)
            ms = timer(fn, reps)
            R.profile_enable(False)
            k_ms, k_n = R.profile_read(kid)
            return ms, (k_ms / k_n if k_n else None)

        fwd = lambda: p.forward(t["z"], [t["W"]], [t["b"]], out=self.out)
        ms_f, k_f = ktime(fwd, max(3, steps), R.PROF_AGG_FWD)
        _, k_fs = ktime(fwd, max(3, steps), R.PROF_AGG_SUM)
        dout = torch.randn_like(self.out[: self.n_out])
        bwd = lambda: p.backward(dout, t["z"], [t["W"]], [t["b"]])
        ms_b, k_b = ktime(bwd, max(3, steps), R.PROF_AGG_BWD)
        _, k_bs = ktime(bwd, max(3, steps), R.PROF_AGG_SUM)

        def fb():
            fwd()
            bwd()
        ms_fb = timer(fb, max(3, steps))
        # the per-tuple form of the same rule (the Linear on every matched tuple, then the SUM walk)
        ppt = R.RulePlan(t["h"], [(t["src"], t["dst"])], self.d, self.d_out, flags=self.flags | R.FLAG_PER_TUPLE)
        ms_pt, k_pt = ktime(lambda: ppt.forward(t["z"], [t["W"]], [t["b"]], out=self.out), max(3, steps), R.PROF_FWD_TC)
        ms_ptb, k_ptb = ktime(lambda: ppt.backward(dout, t["z"], [t["W"]], [t["b"]]), 3, R.PROF_BWD_TC)
        del ppt
        pk, _ = peaks()
        pt_flop = 2.0 * (2 * self.d) * self.d_out * self.matched
        # backward compulsory bytes: per pass and tuple one 4-byte index, the dOut rows (bf16) and
        # H rows (bf16) once per pass, dz written by the src pass and read and written by the dst pass
        n_h = int(t["h"].numel())
        b_bytes = 2 * (4 * self.matched + self.n_out * self.d_out * 2 + n_h * self.d * 2) + n_h * self.d * 4 * 3
        f_bytes = self.forward_bytes()
        ms_torch = timer(self.torch_step, 3)
        # the push-down rewrite (Linear once per H row, then per-tuple gathers of the f32 products)
        from paper_2605_24207_b300 import relnn as R
        ppd = R.RulePlan(t["h"], [(t["src"], t["dst"])], self.d, self.d_out, flags=self.flags | R.FLAG_PUSHDOWN)
        ms_pd = timer(lambda: ppd.forward(t["z"], [t["W"]], [t["b"]], out=self.out), max(3, steps))
        del ppd
        pmx = R.RulePlan(t["h"], [(t["src"], t["dst"])], self.d, self.d_out, flags=self.flags | R.FLAG_MAX)
        ms_mx = timer(lambda: pmx.forward(t["z"], [t["W"]], [t["b"]], out=self.out), max(3, steps))
        del pmx
        # E streamed from pinned host memory in 4 chunks (plan + forward per chunk, copies overlapped)
        src_h, dst_h = t["src"].cpu().pin_memory(), t["dst"].cpu().pin_memory()
        chunk = (src_h.numel() + 3) // 4
        stm = R.StreamRule(t["h"], src_h, dst_h, self.d, self.d_out, flags=self.flags, chunk_tuples=chunk)
        ms_st = timer(lambda: stm.forward(t["z"], t["W"], t["b"]), 3)
        h2d = 2 * src_h.numel() * src_h.element_size()
        dev_keys = torch.empty(2 * src_h.numel(), dtype=src_h.dtype, device=t["src"].device)
        host_keys = torch.cat([src_h, dst_h]).pin_memory()
        ms_cp = timer(lambda: dev_keys.copy_(host_keys, non_blocking=True), 3)
        del stm, dev_keys, host_keys
        # attention over the same join (HGT softmax head, 8 heads, bf16 rows q = k = v = z; product head)
        zq = t["z"] if t["z"].dtype == torch.bfloat16 else t["z"].to(torch.bfloat16)
        sc = 1.0 / (self.d // 8) ** 0.5
        ms_at = timer(lambda: p.attention(zq, zq, zq, 8, sc, "softmax"), max(3, steps))
        ao, al = p.attention(zq, zq, zq, 8, sc, "softmax")
        dd = torch.ones_like(ao)
        ms_atb = timer(lambda: p.attention_backward(dd, ao, al, zq, zq, zq, 8, sc, "softmax"), 3)
        ms_ap = timer(lambda: p.attention(zq, zq, zq, 1, 1.0, "product"), max(3, steps))
        del ao, al, dd
        # cyclic self-join on a batch of small graphs (a separate synthetic workload): plan, forward,
        # backward; the walk's algorithmic bytes are the records (16 B) + the B and C key rows once +
        # the A rows and output rows once
        from paper_2605_24207_b300 import workloads as WL
        gh, ga, gb, gc, gs, gd = WL.graph_batch(11, 50_000, 32, 64)
        dv = t["src"].device
        th, ts, td = (torch.from_numpy(x).to(dv) for x in (gh, gs, gd))
        tA, tB, tC = (torch.from_numpy(x).to(dv) for x in (ga, gb, gc))
        tri_holder = {}

        def tri_plan():
            tri_holder["T"] = None
            tri_holder["T"] = R.TrianglePlan(th, ts, td)
        ms_tp = timer(tri_plan, 3)
        T3 = tri_holder["T"]
        ms_tf = timer(lambda: T3.forward(tA, tB, tC), max(3, steps))
        to = T3.forward(tA, tB, tC)
        ms_tb = timer(lambda: T3.backward(torch.ones_like(to), tA, tB, tC), 3)
        tri_bytes = 16 * T3.n_records + 4 * 64 * (3 * gh.size + T3.n_out)
        tri = {"edges": int(gs.size), "records": T3.n_records, "n_out": T3.n_out, "plan_ms": ms_tp,
               "forward_ms": ms_tf, "backward_ms": ms_tb, "forward_algorithmic_bytes": tri_bytes,
               "forward_gbs": tri_bytes / (ms_tf * 1e-3) / 1e9,
               "what": "relnn_triangle_*: 50,000 ring graphs of 32 nodes (3 forward edges per node, each "
                       "reversed with p 0.5), d = 64 f32; plan = join with H, two edge sorts, per-edge "
                       "sorted-list intersection into records"}
        del T3, tri_holder, to
        # algorithmic bytes of the softmax forward: 3 index arrays per tuple, q / k / v rows once,
        # the output rows and their log-sum-exp once
        n_h = t["h"].numel()
        at_bytes = 12 * self.matched + 3 * n_h * self.d * 2 + self.n_out * (self.d + 8) * 4
        return {"warm_forward_tuples_per_s": self.matched / (ms_f * 1e-3), "warm_forward_ms": ms_f,
                "warm_forward_kernels_ms": {"seg_sum": k_fs, "agg_gemm": k_f},
                "warm_forward_roofline": {"bound": "hbm", "algorithmic_bytes": f_bytes,
                                          "achieved_gbs": f_bytes / (ms_f * 1e-3) / 1e9,
                                          "frac": f_bytes / (ms_f * 1e-3) / 1e9 / pk["hbm_gbs"],
                                          "what": "the whole warm forward (both kernels, fix-ups, launches) "
                                                  "against its compulsory bytes (no intermediate)"},
                "warm_backward_ms": ms_b,
                "warm_backward_kernels_ms_per_pass": {"seg_sum": k_bs, "agg_gemm": k_b},
                "warm_backward_roofline": {"bound": "hbm", "algorithmic_bytes": b_bytes,
                                           "achieved_gbs": b_bytes / (ms_b * 1e-3) / 1e9,
                                           "frac": b_bytes / (ms_b * 1e-3) / 1e9 / pk["hbm_gbs"],
                                           "what": "the whole warm backward (two passes of gather-sum + "
                                                   "GEMM, dOut preparation, fix-ups) against its compulsory "
                                                   "bytes"},
                "warm_fwd_bwd_tuples_per_s": self.matched / (ms_fb * 1e-3), "warm_fwd_bwd_ms": ms_fb,
                "per_tuple_form": {"warm_forward_ms": ms_pt, "fwd_tc_kernel_ms": k_pt,
                                   "tensor_tflops": pt_flop / (k_pt * 1e-3) / 1e12 if k_pt else None,
                                   "frac_of_bf16_burst": (pt_flop / (k_pt * 1e-3) / 1e12 / pk["bf16_tflops"]) if k_pt else None,
                                   "warm_backward_ms": ms_ptb, "bwd_tc_kernel_ms": k_ptb,
                                   "what": "RELNN_FLAG_PER_TUPLE: the Linear on every matched tuple (tcgen05), "
                                           "then the SUM walk; backward: two tcgen05 passes"},
                "pushdown_warm_forward": {"tuples_per_s": self.matched / (ms_pd * 1e-3), "ms": ms_pd,
                                          "what": "RELNN_FLAG_PUSHDOWN: P = Z W_src^T, Q = Z W_dst^T + b per H row "
                                                  "(tensor cores), then per-tuple f32 row gathers + SUM"},
                "stream_forward": {"tuples_per_s": self.matched / (ms_st * 1e-3), "ms": ms_st, "chunks": 4,
                                   "h2d_bytes": h2d, "h2d_copy_ms": ms_cp,
                                   "what": "relnn_stream_forward: E keys in pinned host memory, 4 chunks, each "
                                           "planned against the shared H side and evaluated while the next is "
                                           "copied; h2d_copy_ms is one plain pinned copy of the same key bytes"},
                "attention": {"softmax_forward_ms": ms_at, "softmax_forward_tuples_per_s": self.matched / (ms_at * 1e-3),
                              "softmax_backward_ms": ms_atb, "product_forward_ms": ms_ap,
                              "softmax_forward_algorithmic_bytes": at_bytes,
                              "softmax_forward_gbs": at_bytes / (ms_at * 1e-3) / 1e9,
                              "what": "relnn_attention_* on this join: HGT softmax head (8 heads of 16, bf16 "
                                      "q = k = v = z) and the product head; bytes = indices + q, k, v rows once "
                                      "+ output rows and log-sum-exp"},
                "triangle": tri,
                "max_warm_forward": {"tuples_per_s": self.matched / (ms_mx * 1e-3), "ms": ms_mx,
                                     "what": "RELNN_FLAG_MAX: the same fused forward with a MAX group-by (per-feature "
                                             "maximum and the position of its first tuple, kept for the backward)"},
                "torch_fp32_unfused": {"tuples_per_s": self.matched / (ms_torch * 1e-3), "ms_per_step": ms_torch,
                                       "what": "sort+searchsorted join, index_select, cat, F.linear f32 (TF32 off), "
                                               "unique + index_add_; same step (join + forward)"}}

    def torch_step(self):
        """The plain unfused FP32 form of the same step in torch ops (the comparator)."""
        import torch
        import torch.nn.functional as F
        t = self.t
        torch.backends.cuda.matmul.allow_tf32 = False
        h = t["h"]
        order = torch.argsort(h)
        sk = h[order]
        ps = torch.searchsorted(sk, t["src"]).clamp_(max=sk.numel() - 1)
        pd = torch.searchsorted(sk, t["dst"]).clamp_(max=sk.numel() - 1)
        keep = (sk[ps] == t["src"]) & (sk[pd] == t["dst"])
        hs, hd = order[ps[keep]], order[pd[keep]]
        z = t["z"].float()
        X = torch.cat([z.index_select(0, hs), z.index_select(0, hd)], dim=1)
        Y = F.linear(X, t["W"], t["b"])
        uk, inv = torch.unique(t["dst"][keep], return_inverse=True)
        out = torch.zeros((uk.numel(), Y.shape[1]), dtype=torch.float32, device=Y.device)
        out.index_add_(0, inv, Y)
        return out

    def cpu_rate(self, n_sample):
        from oracle import relnn_oracle as O
        br = self.rel.branches[0]
        n = min(n_sample, br.src.size)
        ob = _Br(br.src[:n], br.dst[:n], _bf16(br.W), br.b)
        z = _bf16(self.rel.z)
        t0 = time.perf_counter()
        _, _, sizes = O.rule_forward(self.rel.h_ids, z, [ob], agg=self.agg)
        dt = time.perf_counter() - t0
        return sizes[0] / dt, f"first {n} of {self.n_tuples} E rows with the full H ({sizes[0]} matched tuples, {dt:.1f} s)"


class C3:
    """Two stacked rules + SUM readout + MSE: one training step (content cached)."""
    name = "c3"

    def __init__(self, args):
        from paper_2605_24207_b300 import workloads as W
        self.n_tuples = args.n_tuples or 4_000_000
        self.n_keys = args.n_keys or 500_000
        self.args = args
        r1, W2, b2, groups, targets = W.config3(seed=0, n_tuples=self.n_tuples, n_keys=self.n_keys)
        br = r1.branches[0]
        self.host = dict(h=r1.h_ids, z=r1.z, src=br.src, dst=br.dst, W1=br.W, b1=br.b, W2=W2, b2=b2,
                         g_keys=r1.h_ids.copy(), g_groups=groups, t_keys=np.arange(8, dtype=np.int32),
                         targets=targets)

    def describe(self):
        return (f"two stacked rules (Linear 128->64 + ReLU, Linear 128->64) + SUM readout into 8 groups + "
                f"MSE; E {self.n_tuples} tuples over {self.n_keys} int32 keys (src Zipf 1.2), z f32[64]; "
                f"step = forward + backward (BF16 form, content cached across steps)")

    def to_device(self, dev):
        import torch
        from paper_2605_24207_b300 import programs
        self.t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in self.host.items()}
        t = self.t
        self.prog = programs.StackedReadout(t["h"], t["src"], t["dst"], t["g_keys"], t["g_groups"], t["t_keys"],
                                            t["targets"], 64, bf16=True)
        self.matched = self.prog.tuples

    def step(self):
        t = self.t
        return self.prog.step(t["z"], t["W1"], t["b1"], t["W2"], t["b2"])

    def kernels(self):
        from paper_2605_24207_b300 import relnn as R
        pr = self.prog
        m1, m2 = pr.p1.n_matched, pr.p2.n_matched
        n_h, n1, n2 = int(self.t["h"].numel()), pr.p1.n_out, pr.p2.n_out
        # rule 1 (ReLU) runs its forward per tuple on the tensor cores (2 x 128 x 64 FLOP per tuple,
        # keeping the ReLU mask); rule 2 (linear) its forward aggregate-first, and both backwards run
        # aggregate-first (rule 1 through the mask). HBM-bound work per step: the gather-sums (5
        # launches: rule 2's forward, two passes per backward) read per tuple a 4-byte index (+ a
        # 4-byte mask word and its index for rule 1's src pass), each gathered row once (bf16) and
        # write a bf16 pair (4 x 64 B) per H row; the GEMMs (5 launches) read those pairs and each
        # H row once and write each output / dz row once (f32, dz rows read back by the dst pass).
        sum_b = (4 * m2 + n1 * 64 * 2 + n2 * 256) + 2 * (4 * m2 + n2 * 64 * 2 + n1 * 256) + \
                2 * (4 * m1 + n1 * 64 * 2 + n_h * 256) + 8 * m1
        gemm_f = n2 * 256 + n2 * 128 + n2 * 256
        gemm_b = 2 * (n1 * 256 + n1 * 128 + n1 * 256) + 2 * (n_h * 256 + n_h * 128 + n_h * 256)
        return {R.PROF_FWD_TC: ("fwd_tc_kernel (rule 1)", 2.0 * 128 * 64 * m1, "tensor"),
                R.PROF_AGG_SUM: ("seg_sum kernels (rule 2 forward; both backwards)", float(sum_b), "hbm"),
                R.PROF_AGG_FWD: ("agg_gemm_kernel forward (rule 2)", float(gemm_f), "hbm"),
                R.PROF_AGG_BWD: ("agg_gemm_kernel backward (both rules)", float(gemm_b), "hbm"),
                R.PROF_BWD_TC: ("bwd_tc_kernel (per-tuple backward, if taken)", 2.0 * 2.0 * 128 * 64 * m1, "tensor"),
                R.PROF_FWD_FP32: ("fwd_identity_agg_kernel (readout gather-sum)", float(n2 * 64 * 4 + n2 * 4), "hbm")}

    def e2e_setup(self):
        import torch
        keys = ("z", "W1", "b1", "W2", "b2")
        self.hp = {k: self.t[k].cpu().pin_memory() for k in keys}
        self.dv = {k: torch.empty_like(self.t[k]) for k in keys}
        self.loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
        return sum(v.numel() * v.element_size() for v in self.hp.values()), 4

    def e2e_step(self):
        for k in self.hp:
            self.dv[k].copy_(self.hp[k], non_blocking=True)
        d = self.dv
        loss, g = self.prog.step(d["z"], d["W1"], d["b1"], d["W2"], d["b2"])
        self.loss_host.copy_(loss, non_blocking=True)
        return loss

    def extras(self, timer, steps):
        ms_t = timer(self.torch_step, 3)
        return {"torch_fp32_unfused": {"tuples_per_s": self.matched / (ms_t * 1e-3), "ms_per_step": ms_t,
                                       "what": "index_select + cat + F.linear f32 (TF32 off) + ReLU + index_add_ "
                                               "per rule, index_add_ readout, MSE, torch.autograd backward; join "
                                               "indices cached like the library's plans"}}

    def torch_step(self):
        import torch
        import torch.nn.functional as F
        torch.backends.cuda.matmul.allow_tf32 = False
        t = self.t
        if not hasattr(self, "_idx"):
            def join(keys, src, dst):
                order = torch.argsort(keys)
                sk = keys[order]
                ps = torch.searchsorted(sk, src).clamp_(max=sk.numel() - 1)
                pd = torch.searchsorted(sk, dst).clamp_(max=sk.numel() - 1)
                keep = (sk[ps] == src) & (sk[pd] == dst)
                uk, inv = torch.unique(dst[keep], return_inverse=True)
                return order[ps[keep]], order[pd[keep]], uk, inv
            hs1, hd1, k1, inv1 = join(t["h"], t["src"], t["dst"])
            hs2, hd2, k2, inv2 = join(k1, t["src"], t["dst"])
            sk = k2
            pg = torch.searchsorted(sk, t["g_keys"]).clamp_(max=sk.numel() - 1)
            keep = sk[pg] == t["g_keys"]
            go, ginv = torch.unique(t["g_groups"][keep], return_inverse=True)
            self._idx = (hs1, hd1, k1, inv1, hs2, hd2, k2, inv2, pg[keep], ginv, go)
        hs1, hd1, k1, inv1, hs2, hd2, k2, inv2, gsrc, ginv, go = self._idx
        z = t["z"].clone().requires_grad_(True)
        W1 = t["W1"].clone().requires_grad_(True)
        b1 = t["b1"].clone().requires_grad_(True)
        W2 = t["W2"].clone().requires_grad_(True)
        b2 = t["b2"].clone().requires_grad_(True)
        Y1 = F.relu(F.linear(torch.cat([z.index_select(0, hs1), z.index_select(0, hd1)], 1), W1, b1))
        h1 = torch.zeros((k1.numel(), 64), device=z.device).index_add(0, inv1, Y1)
        Y2 = F.linear(torch.cat([h1.index_select(0, hs2), h1.index_select(0, hd2)], 1), W2, b2)
        h2 = torch.zeros((k2.numel(), 64), device=z.device).index_add(0, inv2, Y2)
        ho = torch.zeros((go.numel(), 64), device=z.device).index_add(0, ginv, h2.index_select(0, gsrc))
        loss = ((ho - t["targets"][go.long()]) ** 2).mean()
        loss.backward()
        return loss

    def cpu_rate(self, n_sample):
        from oracle import relnn_oracle as O
        from paper_2605_24207_b300 import workloads as W
        # a bounded sample of the same workload: the same recipe at 1/40 of the tuples and keys
        nt, nk = max(1000, self.n_tuples // 40), max(100, self.n_keys // 40)
        r1, W2, b2, groups, targets = W.config3(seed=0, n_tuples=nt, n_keys=nk)
        br = r1.branches[0]
        a = (r1.h_ids, r1.z, br.src, br.dst, br.W, br.b, W2, b2, r1.h_ids.copy(), groups,
             np.arange(8, dtype=np.int32), targets)
        t0 = time.perf_counter()
        f = O.stacked_forward(*a)
        O.stacked_backward(*a, fwd=f)
        dt = time.perf_counter() - t0
        e1 = O.join(br.src, br.dst, r1.h_ids)[0].size
        e2 = O.join(br.src, br.dst, f["k1"])[0].size
        return (e1 + e2) / dt, f"same recipe at {nt} tuples / {nk} keys ({e1 + e2} rule tuples, {dt:.1f} s)"


class C4:
    """Union of three branches into one output (plan + forward)."""
    name = "c4"

    def __init__(self, args):
        from paper_2605_24207_b300 import workloads as W
        self.rel = W.config4(seed=0)
        self.sizes = [b.src.size for b in self.rel.branches]

    def describe(self):
        return ("union replicator over 3 relations (2M/1M/0.5M tuples, shared 300k int32 keys, src uniform, "
                "dst Zipf 1.0), z f32[64], r f32[64] per tuple, BF16 Linear 192->96 per branch, SUM by dst; "
                "step = plan + forward, Kahan summation")

    def to_device(self, dev):
        import torch
        from paper_2605_24207_b300 import relnn as R
        rel = self.rel
        self.t = dict(h=torch.from_numpy(rel.h_ids).to(dev), z=torch.from_numpy(rel.z).to(dev))
        self.brs = [(torch.from_numpy(b.src).to(dev), torch.from_numpy(b.dst).to(dev)) for b in rel.branches]
        self.W = [torch.from_numpy(b.W).to(dev) for b in rel.branches]
        self.b = [torch.from_numpy(b.b).to(dev) for b in rel.branches]
        self.r = [torch.from_numpy(b.r).to(dev) for b in rel.branches]
        self.flags = R.FLAG_BF16 | R.FLAG_KAHAN
        p = R.RulePlan(self.t["h"], self.brs, 64, 96, flags=self.flags, d_r=64)
        self.matched, self.n_out = p.n_matched, p.n_out
        self.n_h = int(rel.h_ids.size)
        self.plan0 = p
        self.out = torch.empty((self.n_out, 96), dtype=torch.float32, device=dev)

    def tune(self):
        """The autotuner's tile choice of the per-tuple form (the rule has a per-tuple embedding),
        timed on the first branch, applied before anything is timed."""
        from paper_2605_24207_b300 import autotune as A
        import torch
        c = A.tune_rule(64, 96, int(self.sizes[0]), rel=self.rel, z_dtype=torch.float32, kahan=True,
                        backward=False, cache=None, reps=3)
        self.flags = (self.flags & ~A.R.FLAG_TILE128) | A.apply(c)
        return c

    def step(self):
        from paper_2605_24207_b300 import relnn as R
        p = R.RulePlan(self.t["h"], self.brs, 64, 96, flags=self.flags, d_r=64)
        p.forward(self.t["z"], self.W, self.b, self.r, out=self.out)
        p.release()  # stream-ordered free, as in the single-rule step
        return None

    def kernels(self):
        from paper_2605_24207_b300 import relnn as R
        # HBM-bound (about 115 FLOP per byte): algorithmic bytes of the three launches = per tuple its
        # r row (64 x f32) and its four 4-byte indices, each H row once (f32[64]) and each output row
        # once (f32[96])
        by = self.matched * (64 * 4 + 16) + self.n_h * 64 * 4 + self.n_out * 96 * 4
        return {R.PROF_FWD_TC: ("fwd_tc_kernel", float(by), "hbm")}

    def e2e_setup(self):
        import torch
        self.hp = [v.cpu().pin_memory() for v in [self.t["h"], self.t["z"]] + [x for s, d in self.brs for x in (s, d)] + self.r]
        self.dv = [torch.empty_like(v, device="cuda") for v in self.hp]
        self.out_host = torch.empty((self.n_out, 96), dtype=torch.float32).pin_memory()
        return sum(v.numel() * v.element_size() for v in self.hp), self.out_host.numel() * 4

    def e2e_step(self):
        from paper_2605_24207_b300 import relnn as R
        for a, b in zip(self.dv, self.hp):
            a.copy_(b, non_blocking=True)
        h, z = self.dv[0], self.dv[1]
        brs = [(self.dv[2 + 2 * i], self.dv[3 + 2 * i]) for i in range(3)]
        r = self.dv[8:11]
        p = R.RulePlan(h, brs, 64, 96, flags=self.flags, d_r=64)
        o = p.forward(z, self.W, self.b, r, out=self.out)
        self.out_host.copy_(o, non_blocking=True)
        return p

    def extras(self, timer, steps):
        """Error per output relation against the FP64 oracle on sampled keys, Kahan on and off."""
        from oracle import relnn_oracle as O
        from paper_2605_24207_b300 import relnn as R
        res = {}
        keys = self.plan0.out_keys().cpu().numpy()
        rng = np.random.default_rng(0)
        # the hubs (largest segments) plus a uniform sample of the other keys
        deg = np.zeros(keys.size, np.int64)
        pos = {k: i for i, k in enumerate(keys.tolist())}
        for b in self.rel.branches:
            idx = np.searchsorted(keys, b.dst)
            ok = (idx < keys.size) & (keys[np.minimum(idx, keys.size - 1)] == b.dst)
            np.add.at(deg, idx[ok], 1)
        pick = np.unique(np.concatenate([np.argsort(-deg)[:20], rng.choice(keys.size, 200, replace=False)]))
        sel = set(keys[pick].tolist())
        brs = []
        for b in self.rel.branches:
            m = np.isin(b.dst, keys[pick])
            brs.append(_Br(b.src[m], b.dst[m], _bf16(b.W), b.b, _bf16(b.r[m])))
        ok, oo, _ = O.rule_forward(self.rel.h_ids, _bf16(self.rel.z), brs)
        for kahan in (False, True):
            fl = R.FLAG_BF16 | (R.FLAG_KAHAN if kahan else 0)
            p = R.RulePlan(self.t["h"], self.brs, 64, 96, flags=fl, d_r=64)
            out = p.forward(self.t["z"], self.W, self.b, self.r).cpu().numpy()[pick]
            err = float(np.linalg.norm(out - oo) / np.linalg.norm(oo))
            ms = timer(lambda: p.forward(self.t["z"], self.W, self.b, self.r, out=self.out), max(3, steps))
            res["kahan" if kahan else "plain"] = {"rel_frob_err_vs_fp64": err, "warm_forward_ms": ms,
                                                  "warm_forward_tuples_per_s": self.matched / (ms * 1e-3)}
        res["sampled_keys"] = int(pick.size)
        return {"union_error_and_kahan": res}

    def cpu_rate(self, n_sample):
        from oracle import relnn_oracle as O
        brs, n = [], 0
        for b in self.rel.branches:
            k = min(b.src.size, max(1, n_sample // 6))
            brs.append(_Br(b.src[:k], b.dst[:k], _bf16(b.W), b.b, _bf16(b.r[:k])))
        t0 = time.perf_counter()
        _, _, sizes = O.rule_forward(self.rel.h_ids, _bf16(self.rel.z), brs)
        dt = time.perf_counter() - t0
        return sum(sizes) / dt, f"first {n_sample // 6} E rows of each branch with the full H ({sum(sizes)} tuples, {dt:.1f} s)"


class C1B:
    """4,096 independent instances of the small FP32 rule (E 2,000 tuples over 500 int32 keys, z f32[16],
    Linear 32 -> 16) evaluated together: instance i's keys are offset by i * 1024 so the key spaces are
    disjoint, and one plan + one FP32-form fused launch covers all of them (one shared Linear)."""
    name = "c1b"

    def __init__(self, args):
        from paper_2605_24207_b300 import workloads as W
        self.B = args.instances
        hs, zs, ss, ds = [], [], [], []
        for i in range(self.B):
            r = W.config1(seed=i)
            br = r.branches[0]
            off = np.int32(i * 1024)
            hs.append(r.h_ids + off)
            zs.append(r.z)
            ss.append(br.src + off)
            ds.append(br.dst + off)
            if i == 0:
                self.Wn, self.bn = br.W, br.b
        self.h, self.z = np.concatenate(hs), np.concatenate(zs)
        self.src, self.dst = np.concatenate(ss), np.concatenate(ds)

    def describe(self):
        return (f"{self.B} independent instances of the FP32 rule (E 2,000 tuples over 500 int32 keys, z f32[16], "
                f"Linear 32->16 shared) in one plan + one FP32-form launch; step = plan + forward")

    def to_device(self, dev):
        import torch
        from paper_2605_24207_b300 import relnn as R
        self.t = dict(h=torch.from_numpy(self.h).to(dev), z=torch.from_numpy(self.z).to(dev),
                      src=torch.from_numpy(self.src).to(dev), dst=torch.from_numpy(self.dst).to(dev),
                      W=torch.from_numpy(self.Wn).to(dev), b=torch.from_numpy(self.bn).to(dev))
        p = R.RulePlan(self.t["h"], [(self.t["src"], self.t["dst"])], 16, 16)
        self.matched, self.n_out = p.n_matched, p.n_out
        self.out = torch.empty((self.n_out, 16), dtype=torch.float32, device=dev)
        # virtual rows of the aggregate-first forward: one per output row, or per 32 tuples of one
        _, cnt = np.unique(self.dst, return_counts=True)
        self.n_vrows = int(((cnt + 31) // 32).sum())

    def step(self):
        from paper_2605_24207_b300 import relnn as R
        t = self.t
        p = R.RulePlan(t["h"], [(t["src"], t["dst"])], 16, 16)
        p.forward(t["z"], [t["W"]], [t["b"]], out=self.out)
        p.release()  # stream-ordered free, as in the single-rule step
        return None

    def kernels(self):
        from paper_2605_24207_b300 import relnn as R
        # the FP32 form aggregate-first (the rule is linear, its H keys unique): per matched tuple its
        # 4-byte src row index, per virtual row its 16-byte descriptor and 4-byte dst row index, each
        # H row once (f32[16]) and each output row once (f32[16]); its FLOPs (2 x 32 x 16 per virtual
        # row, 16 per tuple) are a small share of the FMA probe's rate, so the bound is HBM
        n_h = int(self.t["h"].numel())
        work = 4 * self.matched + 20 * self.n_vrows + 64 * n_h + 64 * self.n_out
        return {R.PROF_FWD_FP32: ("fwd_fp32_agg_kernel (FP32 form, aggregate-first)", float(work), "hbm")}

    def e2e_setup(self):
        import torch
        self.hp = {k: v.cpu().pin_memory() for k, v in self.t.items()}
        self.dv = {k: torch.empty_like(v) for k, v in self.t.items()}
        self.out_host = torch.empty((self.n_out, 16), dtype=torch.float32).pin_memory()
        return sum(v.numel() * v.element_size() for v in self.hp.values()), self.out_host.numel() * 4

    def e2e_step(self):
        from paper_2605_24207_b300 import relnn as R
        for k in self.hp:
            self.dv[k].copy_(self.hp[k], non_blocking=True)
        dv = self.dv
        p = R.RulePlan(dv["h"], [(dv["src"], dv["dst"])], 16, 16)
        o = p.forward(dv["z"], [dv["W"]], [dv["b"]], out=self.out)
        self.out_host.copy_(o, non_blocking=True)
        return p

    def extras(self, timer, steps):
        return {}

    def cpu_rate(self, n_sample):
        from oracle import relnn_oracle as O
        from paper_2605_24207_b300 import workloads as W
        n_inst = max(1, min(self.B, n_sample // 2000))
        t0 = time.perf_counter()
        tot = 0
        for i in range(n_inst):
            r = W.config1(seed=i)
            br = r.branches[0]
            _, _, sz = O.rule_forward(r.h_ids, r.z, [_Br(br.src, br.dst, self.Wn, self.bn)])
            tot += sz[0]
        dt = time.perf_counter() - t0
        return tot / dt, f"{n_inst} of the {self.B} instances ({tot} tuples, {dt:.1f} s)"


WORKLOADS = {"c2": C2, "c3": C3, "c4": C4, "c1b": C1B}


# ===================================================================================== serving
def _torch_query(h, z, src, dst, Wt, bt):
    """Plain unfused FP32 form of one query (the serving comparator)."""
    import torch
    import torch.nn.functional as F
    order = torch.argsort(h)
    sk = h[order]
    ps = torch.searchsorted(sk, src).clamp_(max=sk.numel() - 1)
    pd = torch.searchsorted(sk, dst).clamp_(max=sk.numel() - 1)
    keep = (sk[ps] == src) & (sk[pd] == dst)
    zf = z.float()
    X = torch.cat([zf.index_select(0, order[ps[keep]]), zf.index_select(0, order[pd[keep]])], dim=1)
    Y = F.linear(X, Wt, bt)
    uk, inv = torch.unique(dst[keep], return_inverse=True)
    return uk, torch.zeros((uk.numel(), Y.shape[1]), device=Y.device).index_add_(0, inv, Y)


def serving_stats(nq: int, n_cmp: int, local: int = 0, with_cpu: bool = True, workers: int = 2) -> dict:
    """A stream of rule queries (T ~ logU[1k, 1M], K = T/8, z bf16[64], shared Linear 128 -> 64)
    arriving as a Poisson process at 2,000 queries/s, served by relnn_server_* with memory-admitted
    continuous batching; latency = arrival -> results ready. Paced run (clocks sampled), saturation
    run (arrivals as fast as admission allows), and the unfused FP32 torch form on the first n_cmp
    queries of the same trace."""
    import threading

    import torch
    from paper_2605_24207_b300 import autotune
    from paper_2605_24207_b300 import relnn as R
    from paper_2605_24207_b300 import workloads as W

    torch.backends.cuda.matmul.allow_tf32 = False
    arrivals, sizes = W.serving_trace(0, nq, 2000.0)
    grid = np.unique(np.round(np.exp(np.linspace(np.log(1000), np.log(1_000_000), 24))).astype(np.int64))
    qsize = grid[np.argmin(np.abs(np.log(grid)[None, :] - np.log(sizes)[:, None]), axis=1)]
    pool = {}
    for g in grid.tolist():
        keys, src, dst, z = W.serving_query(0, g, g, 64)
        pool[g] = (torch.from_numpy(keys).cuda(), torch.from_numpy(z).cuda().to(torch.bfloat16),
                   torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    rng = np.random.default_rng(7)
    Wt = torch.from_numpy((rng.standard_normal((64, 128)) / np.sqrt(128)).astype(np.float32)).cuda()
    bt = torch.from_numpy((rng.standard_normal(64) / np.sqrt(128)).astype(np.float32)).cuda()
    thr = autotune.tune_tile128_below(64, 64)
    tuples = int(qsize.sum())

    def serve(paced: bool, n: int):
        srv = R.Server(Wt, bt, 64, flags=R.FLAG_BF16, max_queue=4096, max_batch_tuples=2_000_000,
                       max_batch_queries=64, tile128_below=thr, n_workers=workers)
        # warm-up: every size class alone, then a burst of 96 queries of mixed sizes at once (batched
        # path, memory pool at its working set, clocks up), none of it timed
        for g in grid.tolist():
            t = srv.submit(*pool[g])
            while srv.poll(t, 100_000) is None:
                pass
            srv.release(t)
        burst = [srv.submit(*pool[int(g)]) for g in np.resize(grid, 96)]
        for t in burst:
            while srv.poll(t, 100_000) is None:
                pass
            srv.release(t)
        tickets, t_sub = [None] * n, [0.0] * n
        t0 = time.perf_counter()

        def submitter():
            for i in range(n):
                if paced:
                    wait = t0 + arrivals[i] - time.perf_counter()
                    if wait > 0:
                        time.sleep(wait)
                while True:
                    try:
                        tickets[i] = srv.submit(*pool[int(qsize[i])])
                        t_sub[i] = time.perf_counter()
                        break
                    except R.RelnnError as e:
                        if e.status != 4:
                            raise
                        time.sleep(50e-6)

        th = threading.Thread(target=submitter)
        th.start()
        lat, batch_q = [], []
        for i in range(n):
            while tickets[i] is None:
                time.sleep(20e-6)
            r = None
            while r is None:
                r = srv.poll(tickets[i], 200_000)
            arr = (t0 + arrivals[i]) if paced else t0
            lat.append((t_sub[i] - arr) * 1e3 + r[2] * 1e-3)
            batch_q.append(r[3])
            srv.release(tickets[i])
        th.join()
        wall = time.perf_counter() - t0
        srv.close()
        return np.array(lat), wall, float(np.mean(batch_q))

    clk = Clocks(local)
    te0 = time.time()
    lat, wall, mean_batch = serve(True, nq)
    te1 = time.time()
    clocks = clk.stop(te0, te1)
    lat_s, wall_s, mean_batch_s = serve(False, nq)

    # comparator: the unfused FP32 form, one query at a time in arrival order, same trace prefix
    n_cmp = min(nq, n_cmp)
    for g in grid[:3].tolist():
        _torch_query(*pool[g], Wt, bt)
    torch.cuda.synchronize()
    lat_t = []
    t0 = time.perf_counter()
    for i in range(n_cmp):
        wait = t0 + arrivals[i] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        h, z, s_, d_ = pool[int(qsize[i])]
        _torch_query(h, z, s_, d_, Wt, bt)
        torch.cuda.synchronize()
        lat_t.append((time.perf_counter() - (t0 + arrivals[i])) * 1e3)
    lat_t = np.array(lat_t)

    cpu = None
    if with_cpu:
        # CPU oracle on one query of median size
        from oracle import relnn_oracle as O
        gm = int(np.median(qsize))
        keys, src, dst, z = W.serving_query(0, gm, gm, 64)
        t1 = time.perf_counter()
        _, _, sz = O.rule_forward(keys, _bf16(z), [_Br(src, dst, _bf16(Wt.cpu().numpy()), bt.cpu().numpy())])
        cpu = {"value": sz[0] / (time.perf_counter() - t1), "unit": UNIT, "cores": cores(), "kind": "oracle",
               "sample": f"one query of {gm} tuples"}

    pct = lambda a, q: float(np.percentile(a, q))
    return {"value": tuples / wall_s, "unit": UNIT, "queries": nq, "tuples": tuples,
            "config": {"workload": f"serving stream of {nq} rule queries, T ~ logU[1k,1M] (24 size classes), "
                                   f"K = T/8, int32 keys, z bf16[64], shared Linear 128->64, Poisson arrivals "
                                   f"2000/s; value = saturation tuples/s", "tile128_below": thr, "workers": workers},
            "serving": {"paced_p50_ms": pct(lat, 50), "paced_p99_ms": pct(lat, 99),
                        "paced_queries_per_s": nq / wall, "mean_queries_per_batch": mean_batch,
                        "saturation_queries_per_s": nq / wall_s, "saturation_tuples_per_s": tuples / wall_s,
                        "saturation_mean_queries_per_batch": mean_batch_s,
                        "saturation_p50_ms": pct(lat_s, 50), "saturation_p99_ms": pct(lat_s, 99),
                        "first_n_paced_p50_ms": pct(lat[:n_cmp], 50), "first_n_paced_p99_ms": pct(lat[:n_cmp], 99),
                        "torch_fp32_unfused_first_n_p50_ms": pct(lat_t, 50),
                        "torch_fp32_unfused_first_n_p99_ms": pct(lat_t, 99), "first_n": n_cmp},
            "clocks": clocks, "cpu_baseline": cpu}


def run_serving(args):
    """--config c5: the serving stream on its own (one JSON line)."""
    st = serving_stats(args.n_queries, args.cmp_queries, workers=args.workers)
    nq = st["queries"]
    line = {"metric": METRIC, "value": st["value"], "unit": UNIT, "n_gpus": 1, "steps": nq, "warmup": 4,
            "ms_per_step": 1e3 * st["tuples"] / st["value"] / nq, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic (seeded serving trace; no dataset)",
            "config": st["config"], "serving": st["serving"], "cpu_baseline": st["cpu_baseline"],
            "clocks": st["clocks"], "roofline": None, "e2e": None}
    print(json.dumps(line), flush=True)


# ===================================================================================== arms
def reduce_max(x: float, device) -> float:
    """Maximum of x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(step_ms_local: float, units_local: int, device):
    """Whole-job throughput of replicas: every rank processed `units_local` per step; the job's step
    time is the slowest rank's. Returns (units per second over all ranks, job step ms)."""
    import torch.distributed as dist
    world = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    t = reduce_max(step_ms_local, device)
    return world * units_local / (t * 1e-3), t


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands on the host cores (rank 0 only)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    wl = WORKLOADS[args.config](args)
    sample = max(1000, args.cpu_sample // 4)
    for _ in range(args.warmup):
        wl.cpu_rate(sample)
    rates, desc = [], ""
    t_tot = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rate, desc = wl.cpu_rate(sample)
        t_tot += time.perf_counter() - t0
        rates.append(rate)
    value = float(statistics.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded relations; no dataset)",
            "config": {"workload": wl.describe() + " -- FP64 CPU oracle on a bounded sample per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores(), "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def choose_peak(bound: str, pk: dict, pk_src: str, region_s: float, clocks: dict, fp32: dict | None):
    """Roofline denominator of a kernel: (peak, unit, source, the other bf16 peak or None). A bf16
    contraction timed in a region shorter than a second with the SM clock at its maximum is compared
    with the burst GEMM peak, otherwise with the sustained (power-capped) one."""
    if bound == "hbm":
        return pk["hbm_gbs"], "GB/s", f"{pk_src} HBM copy bandwidth", None
    if bound == "alu":
        if fp32 and fp32.get("tflops"):
            return fp32["tflops"], "TFLOP/s", "f32 FMA probe (relnn_peak_fma_f32) measured in this run", None
        return 148 * 128 * 2 * 2.032, "TFLOP/s", "derived f32 peak (148 SM x 128 FMA/clk x 2.032 GHz)", None
    burst, sust = pk["bf16_tflops"], pk["bf16_tflops_sustained"]
    sm, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    at_max = bool(sm and mx and sm >= 0.95 * mx)
    if region_s < 1.0 and at_max:
        return burst, "TFLOP/s", f"{pk_src} bf16 burst (timed region {region_s:.3f} s at the maximum SM clock)", sust
    return sust, "TFLOP/s", f"{pk_src} bf16 sustained", burst


def run_relnn(args):
    import torch
    import torch.distributed as dist
    from paper_2605_24207_b300 import relnn as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, dev)

    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pk, pk_src = peaks()

    def timer(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def measure(wl, steps, warmup):
        """Device time per step (CUDA events on the launching stream, max over ranks), launches and
        the clocks sampled during the timed region; then the library kernels' CUDA-event times over
        the same number of steps run again with every profiled launch bracketed by events (those
        events stay out of the region the step time comes from)."""
        clk = Clocks(local)
        for _ in range(warmup):
            wl.step()
        torch.cuda.synchronize()
        barrier()
        R.profile_enable(False)
        n0 = R.launch_count()
        torch.cuda.synchronize()
        barrier()
        tw0, te0 = time.perf_counter(), time.time()
        e0.record(stream)
        keep = None
        for _ in range(steps):
            keep = wl.step()
        e1.record(stream)
        torch.cuda.synchronize()
        tw, te1 = time.perf_counter() - tw0, time.time()
        barrier()
        launches = R.launch_count() - n0
        clocks = clk.stop(te0, te1)
        ms = max_over_ranks(e0.elapsed_time(e1) / steps)
        # the kernels' durations: the same steps again, each profiled launch between two events
        R.profile_reset()
        R.profile_enable(True)
        for _ in range(steps):
            keep = wl.step()
        torch.cuda.synchronize()
        R.profile_enable(False)
        ks = {kid: R.profile_read(kid) for kid in wl.kernels()}
        plan_ms, plan_n = R.profile_read(R.PROF_PLAN)
        del keep
        return dict(ms=ms, clocks=clocks, launches=launches, wall=tw, region_s=te1 - te0, ks=ks,
                    plan_ms=plan_ms / plan_n if plan_n else None)

    def roofline(wl, m, steps, fp32, traffic=None):
        """Roofline of the step's dominant library kernel (the largest device time), and the same
        figures for every kernel of the step."""
        table = wl.kernels()
        rows = {}
        for kid, (name, work, bound) in table.items():
            k_ms, k_n = m["ks"][kid]
            if k_n == 0:
                continue
            peak, unit, src, other = choose_peak(bound, pk, pk_src, m["region_s"], m["clocks"], fp32)
            per_step = k_ms / steps
            achieved = work / (per_step * 1e-3) / (1e9 if unit == "GB/s" else 1e12)
            r = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                 "kernel": name, "kernel_ms": k_ms / k_n, "kernel_launches_per_step": k_n / steps,
                 "kernel_ms_per_step": per_step, "peak_source": src}
            if other is not None:
                r["frac_other_bf16_peak"] = achieved / other
                r["other_bf16_peak"] = other
            if traffic and traffic.get(kid) is not None:
                r["traffic"] = traffic[kid]
            rows[kid] = r
        if not rows:
            return None, []
        dom = max(rows, key=lambda k: rows[k]["kernel_ms_per_step"])
        main = dict(rows[dom])
        main["traffic"] = traffic.get(dom) if traffic else None
        return main, [rows[k] for k in sorted(rows, key=lambda k: -rows[k]["kernel_ms_per_step"])]

    # FP32 CUDA-core peak (the FP32 form's roofline denominator), clocks sampled around it
    fp32 = None
    if rank == 0:
        clk = Clocks(local)
        R.peak_fma_f32(1 << 14)
        te0 = time.time()
        tf, fms = R.peak_fma_f32(1 << 20)
        te1 = time.time()
        fp32 = {"tflops": tf, "ms": fms, "clocks": clk.stop(te0, te1),
                "what": "relnn_peak_fma_f32: 296 blocks x 1024 threads x 8 independent FMA chains x 2^20 steps"}

    wl = WORKLOADS[args.config](args)
    wl.to_device(dev)
    tuned = wl.tune() if hasattr(wl, "tune") and not args.no_tune else None

    # ------------------------------------------------------------ timed region (device inputs)
    m = measure(wl, args.steps, args.warmup)
    value, t_step = job_throughput(m["ms"], wl.matched, dev)
    traffic = getattr(wl, "ncu_traffic", lambda: None)()
    rl, rl_all = roofline(wl, m, args.steps, fp32, traffic)

    extras = {} if args.no_extras else wl.extras(timer, args.steps)
    extras["plan_ms"] = m["plan_ms"]
    extras["kernels"] = rl_all

    # ------------------------------------------------------------ end to end (host buffers)
    h2d, d2h = wl.e2e_setup()
    e2e_steps = max(3, args.steps // 2)
    if hasattr(wl, "e2e_begin"):
        wl.e2e_begin(stream, 2)
    for _ in range(2):
        wl.e2e_step()
    if hasattr(wl, "e2e_end"):
        wl.e2e_end(stream)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    if hasattr(wl, "e2e_begin"):
        wl.e2e_begin(stream, e2e_steps)
    for _ in range(e2e_steps):
        wl.e2e_step()
    if hasattr(wl, "e2e_end"):
        wl.e2e_end(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, desc = wl.cpu_rate(args.cpu_sample)
        cpu = {"value": rate, "unit": UNIT, "cores": cores(), "kind": "oracle", "sample": desc}
    describe, matched = wl.describe(), wl.matched
    del wl
    torch.cuda.empty_cache()

    # ------------------------------------------------------------ the other configurations
    subs = {}
    if rank == 0 and args.config == "c2" and not args.no_subrecords:
        for name, steps in (("c3", 40), ("c4", 40), ("c1b", 40)):
            sa = argparse.Namespace(**vars(args))
            sa.n_tuples = sa.n_keys = None
            sw = WORKLOADS[name](sa)
            sw.to_device(dev)
            from paper_2605_24207_b300 import autotune as A
            A.apply(None)  # library defaults, then this configuration's own tuning
            s_tuned = sw.tune() if hasattr(sw, "tune") and not args.no_tune else None
            sm = measure(sw, steps, 3)
            srl, srl_all = roofline(sw, sm, steps, fp32)
            rec = {"value": sw.matched / (sm["ms"] * 1e-3), "unit": UNIT, "ms_per_step": sm["ms"], "steps": steps,
                   "warmup": 3, "config": {"workload": sw.describe(), "matched_tuples_per_step": sw.matched},
                   "roofline": srl, "kernels": srl_all, "clocks": sm["clocks"], "gpu_launches": sm["launches"],
                   "plan_ms": sm["plan_ms"]}
            if s_tuned:
                rec["tuned"] = s_tuned
            rec.update(sw.extras(timer, steps))
            subs[name] = rec
            del sw
            torch.cuda.empty_cache()
        if not args.no_serving:
            st = serving_stats(args.sub_queries, args.sub_cmp_queries, local, with_cpu=False, workers=args.workers)
            st["config"]["workload"] += (f" (shortened to the first {args.sub_queries} queries of the trace; the "
                                         f"torch comparator on the first {args.sub_cmp_queries})")
            subs["c5"] = st

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic (seeded Zipf/uniform relations; no dataset)",
            "config": {"workload": describe, "matched_tuples_per_step": matched,
                       "l2": "inputs larger than L2 (no flush needed)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": rl, "cpu_baseline": cpu,
            "e2e": {"value": world * matched / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": m["launches"], "clocks": m["clocks"], "wall_s_timed": m["wall"],
            "fp32_peak": fp32,
        }
        if tuned:
            line["tuned"] = dict(tuned, what="autotune.tune_rule on this relation (plan + forward): the "
                                             "configuration timed here; ms / default_ms are the tuner's "
                                             "forward times with it and with the library defaults, plan_ms / "
                                             "default_plan_ms the plan times")
        line.update(extras)
        if subs:
            line["subrecords"] = subs
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "c5":
        run_serving(args)
    else:
        run_relnn(args)


if __name__ == "__main__":
    main()
