"""Multi-GPU sharding of the (source, frequency) problems.

Every problem is independent (its own forward and adjoint solves), so ranks split the sources and
run their problems alone; the only exchange is the sum of the gradient (or of J^H r) over all
problems: one all-reduce of 5 nz nx values per gradient, plus the misfit scalar.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_sources(n_sources: int, rank: int, world: int) -> np.ndarray:
    """Source indices of `rank`: round-robin, so every rank spans the whole surface."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    return np.arange(rank, n_sources, world, dtype=np.int64)


def shard_workload(w, rank: int, world: int):
    """A copy of workload `w` keeping only this rank's sources (all frequencies)."""
    import copy
    idx = shard_sources(w.n_src, rank, world)
    s = copy.copy(w)
    s.src_cells = np.asarray(w.src_cells)[idx]
    s.src_force = np.asarray(w.src_force)[idx]
    return s


def allreduce_sum(t: torch.Tensor) -> torch.Tensor:
    """In-place sum over ranks (a no-op without an initialised process group)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def reduce_gradient(g: torch.Tensor, phi: torch.Tensor | None = None):
    """Sum a rank's gradient (and misfit) over all ranks."""
    allreduce_sum(g)
    if phi is not None:
        allreduce_sum(phi)
    return g, phi
