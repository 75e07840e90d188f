"""Host logic of a run over several GPUs of one node (one process per GPU).

The simulations are independent, so the ranks share no data: each steps its
own resident set, and the only exchange is the timing of the run, the
maximum over ranks of each rank's timed region, which sets the whole-job
throughput (weak scaling: the work per rank is fixed).

One simulation's sheets can also be split over ranks (every sheet is a
separate run of tracers, Sec. 2.2); then the ranks' integer meshes add up to
the whole deposit bit for bit once they share one fixed-point charge unit
(``common_charge_unit``), and one all-reduce of Nx int64 per step is the only
exchange.
"""
from __future__ import annotations


def combine(total_ms: float, units_per_rank: float, world: int, dist=None, device=None):
    """(max over ranks of total_ms, whole-job units per second).

    With world > 1 every rank must call this together (an all-reduce over the
    default process group; device is where the reduction tensor lives: the
    GPU for NCCL, the CPU for gloo)."""
    if world > 1:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * float(units_per_rank) / (total_ms / 1e3)


def common_charge_unit(local_unit: float, world: int, dist=None, device=None) -> float:
    """The fixed-point charge unit every rank can use: the largest of the
    ranks' own units (each the library's choice for its own largest weight,
    ``sic_diagnostics()["charge_unit"]``), so every rank's charges fit."""
    if world <= 1:
        return float(local_unit)
    import torch
    t = torch.tensor([float(local_unit)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
