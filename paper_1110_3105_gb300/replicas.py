"""Replica form of the multi-GPU solve (host-side bookkeeping only).

The factorization of A is small next to HBM (0.2-1 GB at the workloads'
sizes), so every rank builds or holds the whole compressed inverse and solves
its own contiguous slice of a batch of right-hand-side columns: the columns
are independent (Sec. 4.3: the inverse is applied column by column), so
nothing crosses ranks on the data path.  `column_range` assigns the slices;
`gather_columns` reassembles X on rank 0 for a caller that wants it in one
place (a collective outside the solve).
"""
from __future__ import annotations

import numpy as np


def column_range(total: int, world: int, rank: int) -> tuple:
    """Columns [c0, c1) of a `total`-column batch owned by `rank` of `world`:
    contiguous, in rank order, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad world/rank/total")
    base, extra = divmod(total, world)
    c0 = rank * base + min(rank, extra)
    return c0, c0 + base + (1 if rank < extra else 0)


def gather_columns(x_local, total: int, dist, world: int, rank: int):
    """Rank 0 receives the full N x total batch (numpy, column-major) from the
    ranks' slices (numpy or CPU torch, N x (c1 - c0)); other ranks get None.
    Uses torch.distributed's all_gather on column-padded CPU tensors (gloo)."""
    import torch
    x = torch.as_tensor(np.asarray(x_local))
    n = x.shape[0]
    width = max(column_range(total, world, r)[1] - column_range(total, world, r)[0] for r in range(world))
    pad = torch.zeros((width, n), dtype=x.dtype)
    pad[:x.shape[1]] = x.t()
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    if rank != 0:
        return None
    out = np.empty((n, total), dtype=np.asarray(x_local).dtype, order="F")
    for r in range(world):
        c0, c1 = column_range(total, world, r)
        out[:, c0:c1] = parts[r][:c1 - c0].t().numpy()
    return out
