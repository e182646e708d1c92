"""Host-side multi-GPU logic: one process per GPU, independent systems.

The FLO-SIC step shards by independent units (systems of a batch, or whole
replicas of a workload): no data-path collective is needed, only a barrier
around the timed region and the maximum of the per-rank times.  Works with
NCCL on GPUs and with gloo on CPU (used by the tests).
"""
import datetime
import os

import torch
import torch.distributed as dist


def env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend, timeout_s=600):
    """Initialise the default process group from the environment (no-op for
    a single process)."""
    rank, world, _ = env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))
    return rank, world


def shard(n_units, rank, world):
    """Contiguous balanced split of range(n_units): the units of this rank.
    Every unit is owned by exactly one rank; sizes differ by at most one."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def max_over_ranks(value, device=None):
    """Maximum of a per-rank scalar (the step time of the slowest rank)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device_sync=None):
    """Barrier across ranks, then wait for this rank's device work."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
    if device_sync is not None:
        device_sync()
