"""Replay a request stream against the SIC request server.

``run_trace`` submits every request at its arrival time (seconds after the
start, on the server clock), drives the server's scheduling loop, and returns
the per-request latencies (finish minus arrival) and the throughput in
segment-updates per second.  ``plain=True`` runs the one-simulation-at-a-time
baseline through the same server.
"""
from __future__ import annotations

import time

import numpy as np

from .sic import Server


def run_trace(problems, arrivals, plain=False, hbm_budget=64 << 30, max_active=64, chunk_steps=32,
              stream=None, keep=False, history=False):
    """problems: list of ``inputs.Problem`` (horizontal sheets); arrivals: seconds, ascending.
    history: every request keeps its per-step diagnostics [W_E, KE, P, Q] and
    they are read back when it finishes (``results[i]["history"]``)."""
    from .sic import adopt_sim
    order = np.argsort(np.asarray(arrivals, dtype=np.float64), kind="stable")
    srv = Server(hbm_budget=hbm_budget, max_active=max_active, chunk_steps=chunk_steps, plain=plain,
                 stream=stream)
    t0 = srv.sic_server_clock()
    ids = {}
    results = {}
    nxt = 0
    n = len(problems)
    while len(results) < n:
        now = srv.sic_server_clock() - t0
        while nxt < n and arrivals[order[nxt]] <= now:
            i = int(order[nxt])
            p = problems[i]
            ids[srv.sic_server_submit_horizontal(p, keep=keep or history,
                                                 history_len=p.n_steps if history else 1)] = i
            nxt += 1
        pending = srv.sic_server_tick()
        for r in srv.sic_server_results():
            i = ids[r["id"]]
            if history and r["sim"]:
                sim = adopt_sim(r["sim"], problems[i].nx, problems[i].counts)
                r["history"] = sim.sic_history(problems[i].n_steps)
                if not keep:
                    sim.sic_destroy()
                    r["sim"] = None
            results[i] = r
        if pending == 0 and nxt < n:
            wait = arrivals[order[nxt]] - (srv.sic_server_clock() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
    stats = srv.sic_server_stats()
    srv.sic_server_destroy()
    lat = np.array([results[i]["t_done"] - t0 - arrivals[i] for i in range(n)])
    first = min(arrivals)
    last_done = max(results[i]["t_done"] for i in range(n)) - t0
    seg = sum(results[i]["segment_updates"] for i in range(n))
    return {
        "results": [results[i] for i in range(n)],
        "latency_s": lat,
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "segment_updates": int(seg),
        "makespan_s": float(last_done - first),
        "throughput": float(seg / max(last_done - first, 1e-9)),
        "bytes_peak": int(stats["bytes_peak"]),
        "ticks": int(stats["ticks"]),
        "busy_s": float(stats["busy_s"]),
        "failed": int(sum(1 for i in range(n) if results[i]["status"] != 0)),
        "waits_slots": int(stats["waits_slots"]),
        "waits_memory": int(stats["waits_memory"]),
        "refinements": int(stats["refinements"]),
    }
