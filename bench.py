#!/usr/bin/env python
"""Benchmark of the SIC step on GB300: segment-updates/s.

One step = one pass of the whole hot path over the workload: one launch of
the step kernel (fused gather-kick-drift-deposit over every segment, then the
field solve by the block that finishes last).  The default workload is the
two-stream configuration (512 sheets x 16384 tracers = 8,388,608 segments,
Nx = 1024), the largest single-simulation configuration of the paper-shaped
set.  L2 (129 MB) is flushed before every timed step by reading a 256 MB
buffer (a read leaves no dirty lines for the timed step to write back),
because the tracer state (100 MB read + 100 MB written per step) would
otherwise partly stay resident between steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  ``--impl reference`` times the FP64 oracle on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SIC segment-updates/s"
UNIT = "segment-updates/s"
ALGO_BYTES_PER_SEGMENT = 20          # read x, v, charge (4+4+4), write x, v (4+4)
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


def workload(name):
    from paper_1506_07207_gb300 import inputs
    makers = {
        "two_stream": inputs.two_stream_config,
        "landau_nonlinear": inputs.landau_nonlinear,
        "landau_linear": inputs.landau_linear,
        "langmuir": inputs.langmuir,
    }
    return makers[name]()


def describe(p, name):
    return {"workload": f"{name}: {p.n_sheets} sheets x {int(p.counts[0])} tracers "
                        f"({p.n_segments} segments), Nx={p.nx}, L={p.L:.6g}, dt={p.dt}",
            "segments": p.n_segments, "nx": p.nx, "sheets": p.n_sheets,
            "l2": "flushed before every timed step (256 MB read)"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBps", "hbm"):
                if key in d:
                    return float(d[key]), "measured (MEASURED_PEAKS.json)"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback (no MEASURED_PEAKS.json)"


def kernel_traffic(segments):
    """ncu DRAM bytes of the fused kernel, if the committed capture matches the source."""
    path = os.path.join(ROOT, "profiles", "traffic_push_deposit.json")
    src = os.path.join(ROOT, "paper_1506_07207_gb300", "csrc", "sic_kernels.cu")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if d.get("source_sha256") != sha:
            return None
        return float(d["dram_bytes_per_segment"]) * segments
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and self.uuid not in parts[1]:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_baseline(p, steps):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.run_problem(p, n_steps=steps)
    el = time.perf_counter() - t0
    return {"value": p.n_segments * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} of {p.n_steps} steps of the same workload, FP64 C oracle, "
                      f"single thread (includes one initial deposit)",
            "seconds": el}


def run_reference(args, rank):
    if rank != 0:
        return 0
    p = workload(args.workload)
    import oracle
    oracle.build()
    oracle.run_problem(p, n_steps=args.warmup)
    t0 = time.perf_counter()
    oracle.run_problem(p, n_steps=args.steps)
    el = time.perf_counter() - t0
    v = p.n_segments * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": describe(p, args.workload),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps (after {args.warmup} warm-up) of the "
                                       f"workload, FP64 C oracle, single thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sic", choices=["sic", "reference"])
    ap.add_argument("--workload", default="two_stream")
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--e2e-runs", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1506_07207_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_1506_07207_gb300.sic import Sim, sic_launch_count

    p = workload(args.workload)
    S = p.n_segments
    stream = torch.cuda.Stream()
    sim = Sim.from_problem(p, history_len=64, stream=stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    flush.fill_(1.0)

    def one_step(ev=None):
        with torch.cuda.stream(stream):
            flush.sum()
        if ev:
            ev[0].record(stream)
        sim.sic_step(1)
        if ev:
            ev[1].record(stream)

    for _ in range(args.warmup):
        one_step()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sic_launch_count()
    with Clocks(uuid) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            one_step(evs[k])
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
    launches = sic_launch_count() - launches0
    step_ms = [e[0].elapsed_time(e[1]) for e in evs]
    k1_ms = step_ms  # one kernel per step
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * S * args.steps / (total_ms / 1e3)
    sim.sic_sync()

    # end to end through the C ABI: host arrays in, a full run, state out
    e2e = None
    if rank == 0 and not args.no_e2e:
        x, v, w = p.x, p.v, p.w
        e2e_steps = args.e2e_steps
        times = []
        for _ in range(args.e2e_runs):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = Sim.sic_create(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, x, v, w,
                                qm=p.qm, half_step_init=p.half_step_init, history_len=64,
                                stream=stream.cuda_stream)
            s2.sic_step(e2e_steps)
            xs, vs = s2.sic_get_state()
            times.append(time.perf_counter() - t0)
            s2.sic_destroy()
        n_alloc = sum(-(-int(c) // 32) * 32 for c in p.counts)
        e2e = {"value": S * e2e_steps / min(times), "unit": UNIT,
               "h2d_bytes_per_step": 12 * n_alloc / e2e_steps,
               "d2h_bytes_per_step": 12 * n_alloc / e2e_steps,
               "runs": args.e2e_runs, "steps_per_run": e2e_steps,
               "note": "sic_create from float64 host arrays + sic_step(n) + sic_get_state; "
                       "bytes are the int64 positions and float32 velocities crossing the bus"}

    clocks = clk.summary()
    peak, peak_src = peaks()
    k1_avg_s = statistics.mean(k1_ms) / 1e3
    achieved = ALGO_BYTES_PER_SEGMENT * S / k1_avg_s / 1e9
    traffic = kernel_traffic(S)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 push/deposit, i64 charge, f64 field scale",
        "data": "synthetic", "config": describe(p, args.workload),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_step (fused gather-kick-drift-deposit + field epilogue)",
                     "algorithmic_bytes_per_launch": ALGO_BYTES_PER_SEGMENT * S,
                     "avg_launch_ms": k1_avg_s * 1e3, "peak_source": peak_src,
                     "kernels_per_step": 1},
        "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
        "wall_s_timed_region": t_wall,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, args.cpu_steps)
    sim.sic_destroy()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
