"""Data parallelism over Lambda batches: one process per GPU, replicas.

Every Lambda point is an independent problem (a sampler's walkers are
independent too), so each rank loads the same catalog and injections and
evaluates its own slice of the Lambda batch: nothing on the data path needs a
collective.  torch.distributed is used only for the timing barrier, the max
over ranks and, when a caller wants every result on every rank, an all-gather
of the K output rows.
"""
from __future__ import annotations

import os

import numpy as np


def init_from_env():
    """(rank, local_rank, world) from torchrun's environment; initialises the process group for world > 1."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, local, world


def shard(K, rank, world):
    """Contiguous, balanced slice [start, stop) of K Lambda rows for this rank."""
    base, extra = divmod(int(K), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _device():
    import torch
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(x, world):
    """Largest value of a float across ranks (the slowest rank's time)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local, K, world):
    """All-gather the per-rank slices (shard order) of a length-K float64 array."""
    local = np.ascontiguousarray(local, dtype=np.float64)
    if world == 1:
        return local
    import torch
    import torch.distributed as dist
    sizes = [shard(K, r, world)[1] - shard(K, r, world)[0] for r in range(world)]
    width = max(sizes)
    buf = torch.zeros(width, dtype=torch.float64, device=_device())
    buf[:local.size] = torch.from_numpy(local).to(buf.device)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    return np.concatenate([p[:n].cpu().numpy() for p, n in zip(parts, sizes)])
