"""Multi-process (one process per GPU) helpers for batch-partitioned solves.

Chains are independent, so several GPUs only partition the problems: no data
moves between ranks while solving. The collectives here carry timings and the
gathered results to rank 0, and work on any torch.distributed backend (NCCL on
GPUs, gloo on CPUs).
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, rank: int, world: int):
    """Contiguous block [start, stop) of `n_items` for `rank` (sizes differ by at
    most one)."""
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_to_rank0(tensor):
    """Concatenation of every rank's 1-D tensor on rank 0 (None elsewhere);
    sizes may differ between ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return tensor
    world = dist.get_world_size()
    n = torch.tensor([tensor.numel()], dtype=torch.int64, device=tensor.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes)
    pad = torch.zeros(m, dtype=tensor.dtype, device=tensor.device)
    pad[:tensor.numel()] = tensor
    bufs = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad)
    if dist.get_rank() != 0:
        return None
    return torch.cat([b[:s] for b, s in zip(bufs, sizes)])
