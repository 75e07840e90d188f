#!/usr/bin/env python
"""Benchmark of the SIC step on GB300: segment-updates/s and request latency.

Workload (default ``serving``): a seeded sample of the serving request mix --
Landau and two-stream runs with sheets M in [32, 1024], tracers per sheet N in
[512, 65536], cells Nx in [64, 2048], 200-2000 steps, powers of two uniform
in log2 (``inputs.serving_mix``, seed 0x5EC5).

* ``value``: segment-updates/s of all sampled requests held resident on the
  GPU as one persistent batch (one kernel launch per step for all of them);
  the state (several GB) is far larger than L2, so no flush is needed.  The
  dominant (only) kernel, the fused step, is timed per launch with CUDA
  events on the batch's stream for the roofline.
* ``serving``: the same requests replayed with Poisson arrivals (rate 0.7 x
  the measured batched capacity, and again at 2 x, where requests queue up)
  through the request server, batched (continuous batching) and plain (one
  simulation per launch sequence, first come first served): throughput and
  p50/p99 latency.
* ``e2e``: the batched server fed from host arrays (compact horizontal-sheet
  inputs), every request arriving at t = 0, end to end.
* ``mid_life``: the same resident batch after every request has run 600 of
  its own steps (or all of them) alone, refining as it goes: folded,
  filamented sheets and per-particle charges where refinement split them.
* ``late_states``: nonlinear Landau at t = 50 and two-stream at t = 60,
  refined as they stretch: folded sheets, most particles crossing cell
  edges (``--profile-case`` runs only the ncu case of these).
* ``single_sim``: the two-stream (512 x 16384 = 8,388,608 segments, Nx
  1024), nonlinear Landau (1024 x 4096, Nx 512), linear Landau (256 x 1024,
  Nx 128) and Langmuir (1 x 4096, Nx 64) configurations stepped alone:
  graphs of 8 steps with a 256 MB L2 flush before each, and single steps
  with a flush before each.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SIC segment-updates/s"
UNIT = "segment-updates/s"
# Algorithmic bytes per segment-update of the fused step (one streaming pass):
# read x and v, write x and v (4 + 4 + 4 + 4 in FP32), plus a 4-byte read of
# the tracer charge when charges differ inside a sheet.  Per-sheet charges
# (every horizontal-sheet request) come with the work item, not per tracer.
ALGO_BYTES_SHEET_CHARGE = 16
ALGO_BYTES_TRACER_CHARGE = 20
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
SEED = 0x5EC5


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


def kernel_traffic(segments):
    """DRAM bytes of one step-kernel launch over `segments` segments, scaled
    from an ncu capture of a smaller case (profiles/k_step_traffic.json), or
    None when the kernel source changed since that capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_step_traffic.json")
    src = os.path.join(ROOT, "paper_1506_07207_gb300", "csrc", "sic_kernels.cu")
    try:
        d = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if d.get("kernel_sha256") != sha:
            return None
        return float(d["dram_bytes_per_segment"]) * segments
    except Exception:
        return None


def algo_bytes(probs):
    """Algorithmic bytes of one fused step over these problems."""
    total = 0
    for p in probs:
        per_tracer = not p.is_horizontal and p.w_full is not None and any(
            np.ptp(p.w[b:b + n]) > 0 for b, n in zip(np.r_[0, np.cumsum(p.counts)[:-1]], p.counts))
        total += (ALGO_BYTES_TRACER_CHARGE if per_tracer else ALGO_BYTES_SHEET_CHARGE) * p.n_segments
    return total


def sample_requests(n, rate=None):
    from paper_1506_07207_gb300 import inputs
    return inputs.serving_mix(n_requests=n, seed=SEED, rate=rate)


def describe(reqs, probs):
    segs = [p.n_segments for p in probs]
    return {"workload": f"serving mix sample: {len(reqs)} seeded requests (seed 0x5EC5), Landau and "
                        f"two-stream, M 32-1024 sheets, N 512-65536 tracers, Nx 64-2048, 200-2000 steps",
            "requests": len(reqs), "segments_resident": int(sum(segs)),
            "segment_updates_total": int(sum(p.n_segments * p.n_steps for p in probs)),
            "l2": "resident state several GB, far above the 129 MB L2: no flush"}


def oracle_rate(probs, budget_s=12.0):
    """FP64 oracle on a bounded sample: a few steps of the first requests."""
    import oracle
    oracle.build()
    done_upd, el = 0, 0.0
    for p in probs:
        if p.n_segments > (1 << 24):     # bound host memory of the FP64 arrays
            continue
        steps = 4
        p.x, p.v, p.w
        t0 = time.perf_counter()
        oracle.run_problem(p, n_steps=steps)
        el += time.perf_counter() - t0
        done_upd += p.n_segments * steps
        if el > budget_s:
            break
    return done_upd / el, done_upd, el


def _oracle_request(params):
    """One sampled request, rebuilt from its recipe, 4 oracle steps (a worker)."""
    import oracle
    from paper_1506_07207_gb300 import inputs
    r = inputs.Request(index=params["index"], arrival=0.0, kind=params["kind"], params=params["params"])
    p = r.problem()
    p.x, p.v, p.w
    t0 = time.perf_counter()
    oracle.run_problem(p, n_steps=4)
    return p.n_segments * 4, time.perf_counter() - t0


def oracle_rate_all_cores(reqs, probs, budget_s=12.0):
    """The same oracle over the host's cores: independent requests in a pool of
    spawned processes (one per core), the requests the single-thread sample
    would take in about budget_s x cores seconds."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    todo = [dict(index=r.index, kind=r.kind, params=r.params) for r, p in zip(reqs, probs)
            if p.n_segments <= (1 << 24)]
    # about budget_s of wall time: estimate from the single-thread rate of the first ones
    est, pick = 0.0, []
    for t, p in zip(todo, [q for q in probs if q.n_segments <= (1 << 24)]):
        pick.append(t)
        est += p.n_segments * 4 / 8e7
        if est > budget_s * cores:
            break
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        out = pool.map(_oracle_request, pick, chunksize=1)
    wall = time.perf_counter() - t0
    upd = sum(u for u, _ in out)
    return upd / wall, upd, wall, cores, len(pick)


def run_reference(args, rank):
    """The FP64 oracle as it stands, on the host cores, on the same workload
    and config as the GPU arm.  Each counted step is one oracle step (kick,
    drift, deposit, field) of one sampled request: the request is run for 2
    steps and for 0 steps (the set-up: first deposit, field and the half kick
    back), and the difference is timed, so no set-up deposit is counted."""
    if rank != 0:
        return 0
    reqs = sample_requests(args.requests)
    probs = [r.problem() for r in reqs]
    import oracle
    oracle.build()
    config = dict(describe(reqs, probs), deposit=args.deposit)
    small = min(probs, key=lambda p: p.n_segments)
    for _ in range(args.warmup):
        oracle.run_problem(small, n_steps=1)
    per = 2
    upd, el = 0, 0.0
    t_all = time.perf_counter()
    probs = [p for p in probs if p.n_segments <= (1 << 24)]
    done = 0
    for k in range(args.steps):
        p = probs[k % len(probs)]
        p.x, p.v, p.w                    # expand the compact sheets before timing
        t0 = time.perf_counter()
        oracle.run_problem(p, n_steps=0, order=args.deposit)
        t1 = time.perf_counter()
        oracle.run_problem(p, n_steps=per, order=args.deposit)
        t2 = time.perf_counter()
        el += max((t2 - t1) - (t1 - t0), 1e-9)
        upd += p.n_segments * per
        done += 1
        if time.perf_counter() - t_all > 150:
            break
    v = upd / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, done),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per} oracle steps of each of {done} sampled requests (of at most 2^24 "
                                       f"segments, cycling through the first ones), the set-up (first deposit, "
                                       f"field, half kick) timed separately and subtracted; FP64 C oracle, "
                                       f"single thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def single_sim(torch, Sim, steps, warmup):
    """One simulation alone: the two-stream and nonlinear Landau
    configurations (the roofline applies), and the linear Landau and Langmuir
    ones (small: bound by launch and latency, absolute times only).  Two
    timings each: steps as a user runs them (sic_step of 8 steps, one CUDA
    graph, the L2 flushed before every group of 8), and one step per call with
    the L2 flushed before every step."""
    from paper_1506_07207_gb300 import inputs
    peak, _ = peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush.fill_(1.0)
    out = {}
    for name, p in (("two_stream", inputs.two_stream_config()), ("landau_nonlinear", inputs.landau_nonlinear()),
                    ("landau_linear", inputs.landau_linear()), ("langmuir", inputs.langmuir())):
        stream = torch.cuda.Stream()
        sim = Sim.from_problem(p, history_len=8, stream=stream.cuda_stream)
        for _ in range(max(warmup, 2)):
            sim.sic_step(8)

        def timed(k, reps):
            ev = []
            for _ in range(reps):
                with torch.cuda.stream(stream):
                    flush.sum()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sim.sic_step(k)
                b.record(stream)
                ev.append((a, b))
            torch.cuda.synchronize()
            return statistics.mean(a.elapsed_time(b) for a, b in ev) / 1e3 / k

        g8 = timed(8, max(3, steps // 4))
        one = timed(1, steps)
        sim.sic_destroy()
        gbs = algo_bytes([p]) / g8 / 1e9
        out[name] = {"workload": f"{name.replace('_', ' ')} {p.n_sheets} x {p.n_tracers // p.n_sheets} "
                                 f"({p.n_segments:,} segments), Nx {p.nx}, alone",
                     "value": p.n_segments / g8, "unit": UNIT, "ms_per_step": g8 * 1e3,
                     "achieved_gbs": gbs,
                     "roofline_frac": gbs / peak if name in ("two_stream", "landau_nonlinear") else None,
                     "ms_per_step_single_launch": one * 1e3,
                     "timing": "sic_step(8) (one graph of 8 steps) after a 256 MB L2 flush, per step; "
                               "single launch: sic_step(1) after a flush"}
    return out


def mid_life(torch, Sim, Batch, probs, presteps, steps, warmup, deposit):
    """The resident batch after every request has run `presteps` of its own
    steps (at most its length) alone, refining as its particles pass the
    refinement length (Sec. 2.6): folded, filamented sheets, more crossings
    and, for refined requests, per-particle charges (a second launch)."""
    stream = torch.cuda.Stream()
    sims = [Sim.from_problem(p, history_len=1, stream=stream.cuda_stream, order=deposit) for p in probs]
    t0 = time.perf_counter()
    for sim, p in zip(sims, probs):
        sim.sic_run(min(presteps, p.n_steps))
    t_pre = time.perf_counter() - t0
    batch = Batch(sims)
    S = batch.sic_batch_segments()
    for _ in range(warmup):
        batch.sic_batch_step(1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    steps0 = [s.sic_diagnostics()["step"] for s in sims]
    for a, b in evs:
        a.record(stream)
        batch.sic_batch_step(1)
        b.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    done = [s.sic_diagnostics()["step"] - k for s, k in zip(sims, steps0)]
    segs = [int(s.n_tracers - sum(1 for c in p.closed if not c)) for s, p in zip(sims, probs)]
    work = sum(n * d for n, d in zip(segs, done))
    refined = sum(1 for s, p in zip(sims, probs) if s.n_tracers > p.n_tracers)
    batch.sic_batch_destroy()
    for s in sims:
        s.sic_destroy()
    return {"presteps": presteps, "value": work / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "segments_resident": int(S), "requests_refined": refined,
            "held_during_timing": sum(1 for d in done if d < steps), "presteps_wall_s": round(t_pre, 1),
            "note": "every request advanced min(presteps, its length) steps alone first (sic_run, refining); "
                    "then the same resident batch timed; work counted at each simulation's own steps"}


def late_problem(name):
    """A late, folded state: nonlinear Landau run to t = 50 or two-stream to
    t = 60, refining at half a box (splitting to a quarter)."""
    from paper_1506_07207_gb300 import inputs
    p = inputs.landau_nonlinear() if name == "landau_nonlinear" else inputs.two_stream_config()
    p.refine_length = 0.5 * p.L
    p.refine_split = 0.25 * p.L
    return p, (1000 if name == "landau_nonlinear" else 1200)


def late_states(torch, Sim, groups=4):
    """Step time of late states (folded sheets: most particles cross cell
    edges), stepped as a user runs them (sic_run of 8 steps, refining when a
    particle passes the refinement length), the L2 flushed before each group."""
    peak, _ = peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    for name in ("landau_nonlinear", "two_stream"):
        p, pre = late_problem(name)
        stream = torch.cuda.Stream()
        sim = Sim.from_problem(p, history_len=8, stream=stream.cuda_stream)
        sim.sic_run(pre)
        sim.sic_run(1)
        ev = []
        for _ in range(groups):
            with torch.cuda.stream(stream):
                flush.sum()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.sic_run(8)
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        s = statistics.median(a.elapsed_time(b) for a, b in ev) / 1e3 / 8
        segs = sim.n_tracers
        t = sim.sic_diagnostics()["t"]
        sim.sic_destroy()
        out[name] = {"t": t, "segments": segs, "value": segs / s, "unit": UNIT, "ms_per_step": s * 1e3,
                     "roofline_frac": ALGO_BYTES_TRACER_CHARGE * segs / s / 1e9 / peak,
                     "timing": "sic_run(8) after a 256 MB L2 flush, per step (refinements included)"}
    return out


def profile_case(torch, Sim, name):
    """The case of the late-state ncu capture: the state of late_states, then
    two steps inside an NVTX range named "late"."""
    p, pre = late_problem(name)
    sim = Sim.from_problem(p, history_len=8)
    sim.sic_run(pre)
    sim.sic_run(1)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("late")
    sim.sic_step(2)
    sim.sic_sync()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_case": name, "step": sim.sic_diagnostics()["step"], "tracers": sim.n_tracers}))
    sim.sic_destroy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sic", choices=["sic", "reference"])
    ap.add_argument("--workload", default="serving", choices=["serving", "two_stream"],
                    help="serving: the request-mix sample; two_stream: the 8.4M-segment two-stream run alone")
    ap.add_argument("--deposit", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="0 box particles (Sec. 2.3), 1 piecewise linear (Sec. 2.5), 2 PIC NGP, 3 PIC CIC, 4 first-order weighting (Sec. 2.4)")
    ap.add_argument("--autotune", type=int, default=1, help="tune the batch schedule before timing (0: default)")
    ap.add_argument("--requests", type=int, default=512,
                    help="leading requests of the seeded 4096-request mix to serve (and hold resident for value)")
    ap.add_argument("--budget-gib", type=float, default=4.0, help="server device-memory budget")
    ap.add_argument("--max-active", type=int, default=32, help="server slots")
    ap.add_argument("--presteps", type=int, default=0,
                    help="advance the resident batch this many steps before the warm-up (evolved, filamented states)")
    ap.add_argument("--load", type=float, default=0.7, help="arrival rate / batched capacity")
    ap.add_argument("--overload", type=float, default=0.0,
                    help="a second replay at this load (0: none): requests queue up")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-single", action="store_true")
    ap.add_argument("--no-late", action="store_true")
    ap.add_argument("--profile-case", default=None, choices=["landau_nonlinear", "two_stream"],
                    help="only run the late-state case profiled with ncu (two steps in an NVTX range)")
    ap.add_argument("--mid-life", type=int, default=600,
                    help="also time the resident batch after this many steps of each request (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1506_07207_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_1506_07207_gb300 import inputs, ranks, serving
    from paper_1506_07207_gb300.sic import Batch, Sim, sic_launch_count
    if args.profile_case:
        if rank == 0:
            profile_case(torch, Sim, args.profile_case)
        if world > 1:
            dist.destroy_process_group()
        return 0

    legs = {}
    t_leg = time.perf_counter()
    serving_mode = args.workload == "serving"
    if serving_mode:
        reqs = sample_requests(args.requests)
        probs = [r.problem() for r in reqs]
        config = describe(reqs, probs)
    else:
        probs = [inputs.two_stream_config()]
        config = {"workload": "two-stream instability, 512 sheets x 16384 tracers (8,388,608 segments), "
                              "Nx 1024, one simulation", "segments_resident": probs[0].n_segments,
                  "l2": "256 MB read before every timed step (L2 flush)"}

    # ---- value: every sampled problem resident, one batch, one launch per step
    stream = torch.cuda.Stream()
    flush = None
    if not serving_mode:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        flush.fill_(1.0)
    sims = [Sim.from_problem(p, history_len=1, stream=stream.cuda_stream, order=args.deposit) for p in probs]
    if args.presteps > 0:
        # untimed: each simulation advanced on its own, refining where its
        # particles pass the refinement length (Sec. 2.6)
        for sim, p in zip(sims, probs):
            sim.sic_run(min(args.presteps, p.n_steps))
        config["presteps"] = args.presteps
    batch = Batch(sims)
    S = batch.sic_batch_segments()
    for _ in range(args.warmup):
        batch.sic_batch_step(1)
    schedule = None
    if args.autotune:
        d, st, mn = batch.sic_batch_autotune(3)   # untimed: 40 more warm-up steps
        schedule = {"claim_divisor": d, "staging": ["auto", "off", "on"][st], "claim_min": mn}
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
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
    steps0 = [s.sic_diagnostics()["step"] for s in sims]
    with Clocks(uuid) as clk:
        t_wall = time.perf_counter()
        for a, b in evs:
            if flush is not None:
                with torch.cuda.stream(stream):
                    flush.sum()
            a.record(stream)
            batch.sic_batch_step(1)
            b.record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
    launches = sic_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    # the work done: each simulation's own steps (one that holds for
    # refinement, or for an error, takes fewer), at its segments
    seg_each = [int(s.n_tracers - sum(1 for c in p.closed if not c)) for s, p in zip(sims, probs)]
    done_steps = [s.sic_diagnostics()["step"] - k for s, k in zip(sims, steps0)]
    work = sum(n * d for n, d in zip(seg_each, done_steps))
    held = sum(1 for d in done_steps if d < args.steps)
    total_ms, value = ranks.combine(sum(step_ms), work, world, dist, torch.device("cuda", local))
    batch.sic_batch_destroy()
    for s in sims:
        s.sic_destroy()
    del sims
    clocks = clk.summary()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 push/deposit, i64 fixed-point charge, exact integer field solve",
        "data": "synthetic", "config": dict(config, deposit=args.deposit), "schedule": schedule,
    }
    peak, peak_src = peaks()
    avg_s = statistics.mean(step_ms) / 1e3
    abytes = algo_bytes(probs) * work / max(1, S * args.steps)   # per launch, of the work done
    achieved = abytes / avg_s / 1e9
    traffic = kernel_traffic(S)
    line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": traffic,
                        "kernel": "k_step (fused gather-kick-drift-deposit + field epilogue), one launch "
                                  "per step over every resident simulation",
                        "algorithmic_bytes_per_launch": abytes,
                        "algorithmic_bytes_per_segment": abytes / S,
                        "traffic_frac": (traffic / avg_s / 1e9 / peak) if traffic else None,
                        "avg_launch_ms": avg_s * 1e3, "peak_source": peak_src}
    line["clocks"] = clocks
    line["gpu_launches"] = int(launches)
    line["held_during_timing"] = held
    legs["value"] = time.perf_counter() - t_leg
    line["wall_s_timed_region"] = t_wall

    budget = int(args.budget_gib * (1 << 30))
    if rank == 0 and serving_mode and not args.no_serving:
        works = [p.n_segments * p.n_steps for p in probs]

        def replay(load):
            rate = load * value / (sum(works) / len(works))
            arrivals = []
            t = 0.0
            rng = np.random.default_rng(SEED)
            for _ in probs:
                t += rng.exponential(1.0 / rate)
                arrivals.append(t)
            out = {}
            for mode in ("batched", "plain"):
                r = serving.run_trace(probs, arrivals, plain=(mode == "plain"), hbm_budget=budget,
                                      max_active=args.max_active, chunk_steps=32)
                out[mode] = {"throughput": r["throughput"], "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
                             "makespan_s": r["makespan_s"], "segment_updates": r["segment_updates"],
                             "peak_device_bytes": r["bytes_peak"], "device_busy_s": r["busy_s"],
                             "admission_waits_slots": r["waits_slots"],
                             "admission_waits_memory": r["waits_memory"], "refinements": r["refinements"],
                             "failed_requests": r["failed"]}
            out["arrival_rate_per_s"] = rate
            out["load"] = load
            out["requests"] = len(probs)
            out["hbm_budget_bytes"] = budget
            out["max_active"] = args.max_active
            return out

        t_leg = time.perf_counter()
        line["serving"] = replay(args.load)
        legs["serving"] = time.perf_counter() - t_leg
        if args.overload > 0:
            t_leg = time.perf_counter()
            line["serving"]["overload"] = replay(args.overload)
            legs["overload"] = time.perf_counter() - t_leg
    t_leg = time.perf_counter()
    if rank == 0 and not args.no_e2e:
        if serving_mode:
            arrivals0 = [0.0] * len(probs)
            r = serving.run_trace(probs, arrivals0, plain=False, hbm_budget=budget, max_active=args.max_active,
                                  chunk_steps=32, history=True)
            steps_total = sum(p.n_steps for p in probs)
            h2d = sum(8 * (p.x_template.size + 2 * p.n_sheets) for p in probs)
            d2h = sum(32 * p.n_steps + 96 for p in probs)
            bad = [(i, res["status"]) for i, res in enumerate(r["results"]) if res["status"] != 0]
            hist_ok = sum(1 for res, p in zip(r["results"], probs)
                          if "history" in res and res["history"].shape == (p.n_steps, 4))
            line["e2e"] = {"value": r["throughput"], "unit": UNIT, "failed_requests": bad[:16],
                           "histories_read": hist_ok,
                           "h2d_bytes_per_step": h2d / steps_total,
                           "d2h_bytes_per_step": d2h / steps_total,
                           "note": "request server fed from host arrays (position template, per-sheet "
                                   "velocity and weight), all requests at t = 0, each request's result and "
                                   "its per-step [W_E, KE, P, Q] history read back; per-step bytes averaged "
                                   "over all requests' steps",
                           "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "makespan_s": r["makespan_s"]}
        else:
            line["e2e"] = e2e_single(torch, Sim, probs[0])
    legs["e2e"] = time.perf_counter() - t_leg
    t_leg = time.perf_counter()
    if rank == 0 and serving_mode and args.mid_life > 0 and args.presteps == 0:
        line["mid_life"] = mid_life(torch, Sim, Batch, probs, args.mid_life, args.steps, args.warmup, args.deposit)
    legs["mid_life"] = time.perf_counter() - t_leg
    t_leg = time.perf_counter()
    if rank == 0 and serving_mode and not args.no_single:
        line["single_sim"] = single_sim(torch, Sim, args.steps, args.warmup)
    legs["single_sim"] = time.perf_counter() - t_leg
    t_leg = time.perf_counter()
    if rank == 0 and serving_mode and not args.no_late:
        line["late_states"] = late_states(torch, Sim)
    legs["late_states"] = time.perf_counter() - t_leg
    t_leg = time.perf_counter()
    if rank == 0 and not args.no_cpu_baseline:
        v, upd, el = oracle_rate(probs)
        va, upa, wall, cores, nreq = oracle_rate_all_cores(reqs, probs) if serving_mode else (v, upd, el, 1, 0)
        line["cpu_baseline"] = {"value": va, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"4 steps each of {nreq} sampled requests of at most 2^24 segments, "
                                          f"one per process in a pool of {cores} ({upa} segment-updates in "
                                          f"{wall:.1f} s wall), FP64 C oracle"}
        line["cpu_baseline_single_thread"] = {
            "value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"4 steps each of the sampled problems of at most 2^24 segments, in order, until 12 s "
                      f"({upd} segment-updates in {el:.1f} s), FP64 C oracle, single thread"}
    legs["cpu_baseline"] = time.perf_counter() - t_leg
    line["leg_wall_s"] = {k: round(v, 1) for k, v in legs.items()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def e2e_single(torch, Sim, p, n_steps=200):
    """sic_create from host arrays, n_steps steps, state read back: end to end."""
    x, v, w = p.x, p.v, p.w
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = Sim.sic_create(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, x, v, w, history_len=1)
    sim.sic_step(n_steps)
    xs, vs = sim.sic_get_state()
    el = time.perf_counter() - t0
    sim.sic_destroy()
    return {"value": p.n_segments * n_steps / el, "unit": UNIT,
            "h2d_bytes_per_step": 24 * p.n_tracers / n_steps, "d2h_bytes_per_step": 16 * p.n_tracers / n_steps,
            "note": f"sic_create from host float64 x, v, w (full arrays), {n_steps} steps, positions and "
                    f"velocities read back; bytes averaged over the steps"}


if __name__ == "__main__":
    sys.exit(main())
