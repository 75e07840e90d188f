"""A simulation's sheets split over two ranks (two processes on the one GPU,
gloo between them): each rank deposits its own sheets through sic_deposit
with the shared fixed-point unit, and the all-reduced sum of the two int64
meshes equals the whole simulation's mesh bit for bit (the one exchange per
step of the sheet-sharded design).  The ranks' kernels never wait on one
another: the exchange is on the host."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1506_07207_gb300 import inputs, ranks
        from paper_1506_07207_gb300.sic import Sim
        p = inputs.tiny_problem(5, n_sheets=6, max_tracers=4000, nx=96, L=2.0)
        bounds = np.r_[0, np.cumsum(p.counts)]
        mine = [s for s in range(len(p.counts)) if s % world == rank]
        idx = np.concatenate([np.arange(bounds[s], bounds[s + 1]) for s in mine])
        args = (p.nx, p.L, p.dt, p.counts[mine], p.closed[mine], p.winding[mine], p.x[idx], p.v[idx], p.w[idx])
        probe = Sim.sic_create(*args, half_step_init=False)
        local_unit = probe.sic_diagnostics()["charge_unit"]
        probe.sic_destroy()
        unit = ranks.common_charge_unit(local_unit, world, dist, torch.device("cpu"))
        part = Sim.sic_create(*args, half_step_init=False, charge_unit=unit)
        mesh, _ = part.sic_deposit()
        part.sic_destroy()
        t = torch.from_numpy(mesh.astype(np.int64))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        res = dict(unit=unit, local=local_unit, summed=t.numpy().tolist())
        if rank == 0:
            whole = Sim.sic_create(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, p.w,
                                   half_step_init=False, charge_unit=unit)
            res["whole"] = whole.sic_deposit()[0].tolist()
            res["whole_auto_unit"] = Sim.sic_create(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, p.w,
                                                    half_step_init=False).sic_diagnostics()["charge_unit"]
            whole.sic_destroy()
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_sheet_shards_sum_to_the_whole_mesh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=300)
            assert pr.exitcode == 0
        res = dict(out)
    assert res[0]["unit"] == res[1]["unit"] == max(res[0]["local"], res[1]["local"])
    assert res[0]["unit"] == res[0]["whole_auto_unit"]     # the whole's own choice
    np.testing.assert_array_equal(res[0]["summed"], res[0]["whole"])
    np.testing.assert_array_equal(res[1]["summed"], res[0]["whole"])
