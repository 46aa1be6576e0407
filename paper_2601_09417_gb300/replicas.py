"""Whole-job throughput of independent replicas (one process per GPU).

The fine-tuning step has no cross-GPU exchange in this build: with N processes
every rank runs its own replica of the workload, and the job's rate is the
units all ranks processed divided by the slowest rank's time (weak scaling).
"""

import torch
import torch.distributed as dist


def job_rate(local_total_ms, steps, device=None):
    """(max over ranks of the timed milliseconds, job steps/s = ranks x steps / that time).

    Without an initialised process group this is the single-process rate."""
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    total_ms = float(local_total_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps / (total_ms / 1e3)
