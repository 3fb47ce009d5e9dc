"""Replica sharding over processes, one GPU each.

The path shards only across independent trajectories: replica r of the whole
job draws its noise from Philox key seed + r, so a process that runs replicas
[first, first + count) with seed' = seed + first reproduces exactly those
replicas of a single-process run. There is no collective on the data path;
torch.distributed (gloo, CPU tensors) is used only for the barrier around timed
regions, the max of per-rank times and gathering results on rank 0.
"""
from __future__ import annotations

import os

import numpy as np


def rank_env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_range(rank: int, world: int, total: int | None = None, per_rank: int | None = None):
    """First replica and count of `rank`: an even split of `total` (strong scaling, the
    first total % world ranks take one more) or `per_rank` each (weak scaling)."""
    if per_rank is not None:
        return rank * per_rank, per_rank
    base, extra = divmod(int(total), world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def init(world: int):
    """A gloo process group when world > 1 (None otherwise)."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("gloo", init_method="env://")
    return dist


def barrier(group):
    if group is not None:
        group.barrier()


def max_over_ranks(group, value: float) -> float:
    if group is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    group.all_reduce(t, op=group.ReduceOp.MAX)
    return float(t.item())


def gather_rows(group, rows: np.ndarray, world: int):
    """Concatenate each rank's rows (same trailing shape) on rank 0, in rank order; other
    ranks get None."""
    if group is None:
        return rows
    import torch
    t = torch.from_numpy(np.ascontiguousarray(rows, np.float64))
    n = torch.tensor([t.shape[0]], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    group.all_gather(sizes, n)
    width = int(np.prod(t.shape[1:])) if t.dim() > 1 else 1
    m = int(max(s.item() for s in sizes))
    pad = torch.zeros((m, width), dtype=torch.float64)
    pad[:t.shape[0]] = t.reshape(t.shape[0], width)
    bufs = [torch.zeros_like(pad) for _ in range(world)]
    group.all_gather(bufs, pad)
    if group.get_rank() != 0:
        return None
    out = np.concatenate([b[:int(s.item())].numpy() for b, s in zip(bufs, sizes)])
    return out.reshape((-1,) + tuple(t.shape[1:]))
