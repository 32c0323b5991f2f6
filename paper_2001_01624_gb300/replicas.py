"""Work per rank when one GPU runs one process (replicas: no data-path
collective).

Each rank solves its own seeded inputs: the config-2 geomodel with seed =
rank, ensemble members rank * members .. rank * members + members - 1, the
serving stream of models seeded by rank.  Timings are reduced with the
maximum over ranks (the job ends with its slowest rank) and throughputs count
the units of all ranks over that time.  The reductions run on any
torch.distributed backend (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

from typing import List, Sequence


def geomodel_seed(rank: int) -> int:
    return rank


def member_indices(rank: int, members: int) -> List[int]:
    """Ensemble members of one rank (disjoint across ranks)."""
    return [rank * members + k for k in range(members)]


def serving_seed(rank: int) -> int:
    return rank


def max_over_ranks(dist, values: Sequence[float], device) -> List[float]:
    """Element-wise maximum over the ranks of the process group (values
    unchanged when there is no group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Units of all ranks (each processed units_per_rank) over the slowest rank's time."""
    return units_per_rank * world / seconds
