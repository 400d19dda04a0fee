"""Sharding of a batch of independent 2x2 problems over the ranks of one node.

The matrices of a batch are independent (Sec. 1: the annihilations of one
Kogbetliantz step), so ranks need no data exchange: each rank (one process per
GPU) decomposes a contiguous slice of the batch, or its own batch (weak
scaling).  The only collectives are for timing: a barrier and the maximum of
the per-rank times.  Everything here is host logic and runs under any
torch.distributed backend (gloo on the CPU in the tests, NCCL in the bench).
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def partition(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous slice [start, start + count) of n matrices for rank: the first
    n % world ranks get one more matrix; slices cover 0..n-1 exactly once."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad partition arguments")
    q, r = divmod(n, world)
    start = rank * q + min(rank, r)
    return start, q + (1 if rank < r else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (e.g. elapsed milliseconds) over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch
    import torch.distributed as dist
    if torch.cuda.is_available() and device is not None and torch.device(device).type == "cuda":
        torch.cuda.synchronize(device)
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
    if torch.cuda.is_available() and device is not None and torch.device(device).type == "cuda":
        torch.cuda.synchronize(device)


def run_sharded(A, fn, world: int, rank: int):
    """Apply fn (a batch -> result function, e.g. svd2.svd2) to this rank's slice
    of the split-layout batch A (columns are matrices).  Returns (start, count,
    result); no data leaves the rank."""
    start, count = partition(A.shape[1], world, rank)
    return start, count, fn(A[:, start:start + count])
