"""Data-parallel sharding of chains over ranks (one process per GPU).

Chains are independent Monte Carlo units and every random number is keyed by
(seed, chain id, step), so a rank owning the contiguous chain-id range
[start, start + count) produces exactly the chains a single process would.
There is no collective on the sampling path; results are gathered once, at
the end (``gather_rows``).  Weak scaling: each rank keeps its own chains.
"""
from __future__ import annotations

import numpy as np


def shard(n_total: int, rank: int, world: int):
    """Contiguous range (start, count) of rank `rank`: the first n_total % world
    ranks hold one extra chain."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def gather_rows(local: np.ndarray, n_total: int, group=None) -> np.ndarray:
    """All-gather per-chain rows (first axis = local chains) into the full
    (n_total, ...) array ordered by chain id, through torch.distributed."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    local = np.ascontiguousarray(local, dtype=np.float64)
    row_shape = local.shape[1:]
    width = int(np.prod(row_shape)) if row_shape else 1
    cap = shard(n_total, 0, world)[1]                 # rank 0 holds the largest range
    buf = torch.zeros((cap, width), dtype=torch.float64)
    buf[: len(local)] = torch.from_numpy(local.reshape(len(local), width))
    out = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(out, buf, group=group)
    rows = [out[r][: shard(n_total, r, world)[1]].numpy() for r in range(world)]
    full = np.concatenate(rows, axis=0)
    return full.reshape((n_total,) + row_shape)
