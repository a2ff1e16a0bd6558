"""Multi-GPU runs as independent replicas.

The step has no exchange between GPUs when each GPU holds its own grid (or
its own pool of instances), so an N-GPU run is N replicas.  The only
cross-rank operations are timing ones: a barrier before and after the timed
region and the maximum of the elapsed times; the whole-job throughput is the
units of all ranks over that maximum ("weak" scaling).  These helpers work on
any torch.distributed backend (NCCL on GPUs, gloo in the CPU tests)."""
from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, device=None):
    """Maximum of a float over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_throughput(units_per_rank, elapsed_max, world_size):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world_size / elapsed_max
