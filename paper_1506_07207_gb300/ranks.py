"""Host logic of a run over several GPUs of one node (one process per GPU).

The simulations are independent, so the ranks share no data: each steps its
own resident set, and the only exchange is the timing of the run, the
maximum over ranks of each rank's timed region, which sets the whole-job
throughput (weak scaling: the work per rank is fixed).
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
