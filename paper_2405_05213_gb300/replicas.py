"""Multi-GPU runs as independent replicas (no collective on the data path).

One process per GPU (torchrun), each propagating its own trajectory; the only
collectives are the timing barrier and the max-over-ranks of the elapsed time.
"""
from __future__ import annotations

import os


def dist_env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend):
    """Join the process group when launched with more than one rank."""
    ws, _, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return ws


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value, device=None):
    """The largest `value` over all ranks (the job's elapsed time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank, elapsed_s, world_size):
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    return world_size * units_per_rank / elapsed_s
