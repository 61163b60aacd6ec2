"""Multi-process runs: one process per GPU, each stepping its own lattice (replicas).

The time step shards naturally by domain decomposition, but each box in use has one GPU, so a
run over N GPUs runs N independent replicas of the workload (each with its own seed) and
reports weak-scaling throughput.  This module holds the host-side logic shared by bench.py and
its tests: rank discovery from the launcher's environment, per-rank seeds, and the aggregation
of per-rank timings (barrier, then the maximum over ranks).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class Rank:
    rank: int
    world: int
    local: int

    @property
    def is_root(self) -> bool:
        return self.rank == 0


def from_env(env=None) -> Rank:
    """RANK / WORLD_SIZE / LOCAL_RANK as set by torchrun (defaults: a single process)."""
    env = os.environ if env is None else env
    rank = int(env.get("RANK", "0"))
    world = int(env.get("WORLD_SIZE", "1"))
    local = int(env.get("LOCAL_RANK", str(rank)))
    if not (0 <= rank < world) or local < 0:
        raise ValueError(f"inconsistent rank {rank} / world {world} / local {local}")
    return Rank(rank, world, local)


def replica_seed(base_seed: int, r: Rank) -> int:
    """Each replica draws its own synthetic input."""
    return base_seed + r.rank


def aggregate(local_seconds: float, local_sites: int, dist=None, device=None):
    """Whole-job throughput of N replicas: the job ends when the slowest rank ends, so the
    time is the maximum over ranks and the work is the sum over ranks.  Returns
    (max_seconds, total_sites).  With dist=None (one process) the local values are returned."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(local_seconds), int(local_sites)
    import torch

    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    n = torch.tensor([float(local_sites)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())
