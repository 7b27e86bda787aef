"""Whole-job throughput of independent replicas (one process per GPU, no data-path collective).

Batches shard naturally (Eq. H_decomp), and every rank here runs its own replica of the
workload; the job's throughput is the units all ranks processed divided by the slowest rank's
time, the only cross-rank step being two scalar reductions (MAX of the time, SUM of the units).
The reductions run on whatever backend the process group has (NCCL with CUDA tensors under
torchrun on GPUs, gloo with CPU tensors in the tests).
"""
from __future__ import annotations


def aggregate(units: float, ms: float, device=None) -> tuple[float, float, float]:
    """(units per second of the whole job, the slowest rank's ms, the units of all ranks)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units) / (float(ms) / 1e3), float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    slowest, total = float(t.item()), float(u.item())
    return total / (slowest / 1e3), slowest, total
