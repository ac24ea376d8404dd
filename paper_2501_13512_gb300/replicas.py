"""Replica aggregation for runs on several GPUs.

The solves are independent (no data exchange), so N GPUs run N replicas; the
whole-job rate is the units all ranks completed divided by the slowest rank's
time (weak scaling). Only these two scalars cross ranks.
"""
from __future__ import annotations


def aggregate(elapsed_s: float, units: float, device=None):
    """Return (units_per_s, total_units, max_elapsed_s) over the process group
    (or for this process alone when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units / elapsed_s, float(units), float(elapsed_s)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(u.item()), float(t.item())
