"""Multi-GPU layout of independent solves: one process per GPU, each owning a
disjoint shard of the (k, omega, polarisation) points, no collective on the
data path.  The only communication is host-side bookkeeping after the
solves: the slowest rank's time (max) and, for sweeps, the gather of the
0th-order responses (48 bytes per point) in the original point order.
"""
from __future__ import annotations

import numpy as np


def shard(n, rank, world):
    """Indices of the points rank `rank` of `world` solves: a strided split,
    which keeps the kappa grids of every frequency spread over the ranks."""
    return list(range(rank, n, world))


def max_over_ranks(value, device=None):
    """The maximum of a host float over all ranks (timing of the slowest)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local_rows, n, rank, world):
    """Reassemble per-point rows (e.g. E_0, 3 complex per point) computed on
    the shards into the original order on every rank."""
    import torch.distributed as dist
    local_rows = np.asarray(local_rows)
    if world == 1:
        return local_rows
    parts = [None] * world
    dist.all_gather_object(parts, (rank, local_rows))
    out = np.zeros((n,) + local_rows.shape[1:], dtype=local_rows.dtype)
    for r, rows in parts:
        out[shard(n, r, world)] = rows
    return out
