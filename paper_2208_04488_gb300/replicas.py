"""Whole-job throughput of N independent replicas (one process per GPU).

The method's instances are independent, so `bench.py --gpus N` runs one
replica of the workload per rank with no data-path collective; the ranks only
agree on the result: the units all ranks processed divided by the slowest
rank's time (weak scaling). Host-side logic only, so it runs under any
torch.distributed backend (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations


def whole_job_rate(units: float, seconds: float, dist=None, device: str = "cpu"):
    """(units of all ranks / the slowest rank's seconds, slowest seconds).
    `dist` is torch.distributed when running with more than one rank, else None."""
    if dist is None:
        return units / seconds, seconds
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    t_max = float(t.item())
    return float(u.item()) / t_max, t_max
