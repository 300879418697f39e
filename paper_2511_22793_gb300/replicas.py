"""Host logic of the multi-GPU form: independent replicas sharded by query.

Rendering one transmitter position touches only the scene and that query
(Sec. 4.1 renders each query on its own), so N ranks split the queries, run
the whole path on their own GPU and exchange nothing on the data path.  Two
host steps remain and live here so that they can be exercised with CPU ranks:
the shard of queries each rank draws, and the whole-job figure (the units all
ranks processed over the slowest rank's time).
"""
from __future__ import annotations

import numpy as np


def rank_queries(all_queries: np.ndarray, per_rank: int, rank: int, world: int) -> np.ndarray:
    """Rows [rank*per_rank, (rank+1)*per_rank) of a query list of at least per_rank*world rows:
    disjoint across ranks, and rank 0 of a one-rank job gets the list's first rows."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("rank %d of %d, %d queries per rank" % (rank, world, per_rank))
    if all_queries.shape[0] < per_rank * world:
        raise ValueError("%d queries for %d ranks x %d" % (all_queries.shape[0], world, per_rank))
    return all_queries[rank * per_rank:(rank + 1) * per_rank]


def job_totals(units: int, elapsed_ms: float, device=None):
    """(units summed over ranks, elapsed time maxed over ranks).

    Without an initialised process group the local values come back.  `device` is where the
    reduction tensors live: the rank's GPU under NCCL, None (CPU) under gloo.
    """
    import torch
    import torch.distributed as tdist

    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return int(units), float(elapsed_ms)
    u = torch.tensor([int(units)], dtype=torch.int64, device=device)
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    tdist.all_reduce(u, op=tdist.ReduceOp.SUM)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return int(u.item()), float(t.item())


def throughput(total_units: int, max_ms: float) -> float:
    """Units per second of the whole job."""
    if max_ms <= 0.0:
        raise ValueError("elapsed time %r ms" % max_ms)
    return total_units / (max_ms * 1e-3)
