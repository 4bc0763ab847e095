"""Multi-process helpers: one process per GPU, systems sharded across ranks.

Model systems are independent (every chi2 is a separate sum, Eq. 5), so a
batch splits by system with no exchange of data between ranks: each rank
evaluates its share and, if the caller wants one array, the shares are
gathered at the end.  The only collectives are for bookkeeping (timing,
optional gather); they work with the gloo (CPU) and nccl (GPU) backends.
"""
from __future__ import annotations

import os
from typing import List, Tuple

import numpy as np


def env() -> Tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [start, stop) share of n systems for `rank`; shares differ
    by at most one system and cover [0, n) exactly once."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_by_work(work: np.ndarray, world: int) -> List[np.ndarray]:
    """Partition system indices over `world` ranks balancing total work
    (planet-observation evaluations), greedy longest-first; each rank's
    indices are returned sorted."""
    work = np.asarray(work, dtype=np.int64)
    order = np.argsort(-work, kind="stable")
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(work.size, dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += work[i]
    return [np.sort(np.nonzero(owner == r)[0]) for r in range(world)]


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a scalar over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_shards(local, counts: List[int]):
    """Concatenate every rank's 1-D result in rank order (all ranks receive
    the whole array).  counts[r] is rank r's length."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local
    width = max(counts) if counts else 0
    buf = torch.zeros(width, dtype=local.dtype, device=local.device)
    buf[:local.numel()] = local
    parts = [torch.empty_like(buf) for _ in counts]
    dist.all_gather(parts, buf)
    return torch.cat([p[:c] for p, c in zip(parts, counts)])
