"""Several ranks, emulated on the CPU with gloo (world size 2).

* The timing of a multi-GPU bench run: every rank gets the maximum over ranks
  of the timed regions and the same whole-job throughput (weak scaling).
* Sharding one simulation's sheets over ranks: each rank deposits its own
  sheets and one sum over ranks of the Nx-cell meshes gives the whole
  deposit (the single exchange the design needs per step).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1506_07207_gb300 import ranks
        total_ms, value = ranks.combine(100.0 + 50.0 * rank, 1.0e9, world, dist, torch.device("cpu"))
        import oracle
        from paper_1506_07207_gb300 import inputs
        p = inputs.tiny_problem(5, n_sheets=6, max_tracers=400, nx=32, L=2.0)
        bounds = np.r_[0, np.cumsum(p.counts)]
        mine = [s for s in range(len(p.counts)) if s % world == rank]
        idx = np.concatenate([np.arange(bounds[s], bounds[s + 1]) for s in mine])
        part = oracle.deposit(p.nx, p.L, p.counts[mine], p.closed[mine], p.winding[mine], p.x[idx], p.w[idx])
        t = torch.tensor(part, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        full = oracle.deposit(p.nx, p.L, p.counts, p.closed, p.winding, p.x, p.w)
        out[rank] = (total_ms, value, float(np.abs(t.numpy() - full).max() / np.abs(full).max()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_timing_and_sharded_deposit():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in (0, 1):
        total_ms, value, err = res[rank]
        assert total_ms == 150.0                       # the slower rank's time
        assert value == pytest.approx(2 * 1.0e9 / 0.150)
        assert err < 1e-13
