"""Host-side multi-GPU helpers: independent columns are sharded across ranks
without any data-path collective; only the timing is reduced (max over
ranks). A single column is replicated (it would need halo exchanges)."""
from __future__ import annotations

import numpy as np


def shard_columns(column_offsets, rank: int, world: int):
    """Contiguous range of columns [c0, c1) for `rank`, balanced by particle
    count: each split is the column boundary nearest to r/world of the total."""
    offs = np.asarray(column_offsets, dtype=np.int64)
    ncol = offs.size - 1
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    total = offs[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        c = int(np.searchsorted(offs, target, side="left"))
        c = min(c, ncol)
        if c > 0 and abs(offs[c - 1] - target) <= abs(offs[c] - target):
            c -= 1
        c = max(c, bounds[-1])
        bounds.append(c)
    bounds.append(ncol)
    return bounds[rank], bounds[rank + 1]


def local_offsets(column_offsets, c0: int, c1: int):
    """Offsets of columns [c0, c1) relative to their first particle."""
    offs = np.asarray(column_offsets, dtype=np.int64)
    return (offs[c0:c1 + 1] - offs[c0]).astype(np.int32)


def shard_state(state: dict, column_offsets, rank: int, world: int, per_column=None):
    """This rank's share of a batch of independent columns: the particles of
    columns [c0, c1) from shard_columns, their offsets relative to the first
    of them and, if given, the per-column values (e.g. mu_s) of those
    columns. Returns dict(state=..., offsets=..., per_column=..., c0=, c1=)."""
    c0, c1 = shard_columns(column_offsets, rank, world)
    offs = np.asarray(column_offsets, dtype=np.int64)
    b, e = int(offs[c0]), int(offs[c1])
    return dict(state={k: v[b:e] for k, v in state.items()},
                offsets=local_offsets(column_offsets, c0, c1),
                per_column=None if per_column is None else np.asarray(per_column)[c0:c1],
                c0=c0, c1=c1)


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks of the default process group (identity
    when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
