"""Multi-GPU execution of the renderer: replicas.

Every camera ray is independent and one GPU renders a whole workload, so N GPUs run N replicas (one
process per GPU, launched by torch.distributed.run): no ray data moves between ranks.  The only
collective is on the timing: the job's time is the slowest rank's, and the whole-job rate is the rays
all ranks traced divided by that time (weak scaling: every rank renders the full workload).
"""
from __future__ import annotations

import os


def dist_env():
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks of the default process group (the value itself when no
    group is initialised).  device: where the reduction tensor lives (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds: float, world_size: int) -> float:
    """Units per second of the whole job: every rank processes units_per_rank in at most `seconds`."""
    return world_size * units_per_rank / seconds
