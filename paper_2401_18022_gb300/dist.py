"""Host-side multi-GPU logic (one process per GPU).

Every CUT's eta is independent, and so is every launch-power profile, so the
path shards without a data-path collective:
  * weak scaling (the benchmark): each rank evaluates its own full system for
    an independent seeded launch-power profile (``rank_powers``);
  * strong scaling: the CUTs of one system are split across ranks
    (``shard_cuts``) and the per-CUT results gathered once at the end
    (``gather_by_cut``), which is the only exchange the method has.
The timing reduction (max over ranks) is the only collective on the bench path.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def rank_powers(wl, rank: int, spread_db: float = 0.5, seed0: int = 100) -> np.ndarray:
    """Launch powers of rank `rank`: the workload's own for rank 0, an
    independent seeded +-spread_db dB perturbation of them otherwise."""
    if rank == 0:
        return np.asarray(wl.P_W, dtype=np.float64).copy()
    rng = np.random.default_rng(seed0 + rank)
    return np.asarray(wl.P_W, dtype=np.float64) * 10.0 ** (rng.uniform(-spread_db, spread_db, wl.n_ch) / 10.0)


def shard_cuts(n_ch: int, rank: int, world: int, weights: Sequence[float] = None) -> List[int]:
    """Contiguous shard of CUTs for `rank`, balanced by per-CUT work weights
    (pieces per CUT; uniform when omitted)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    w = np.ones(n_ch) if weights is None else np.asarray(weights, dtype=np.float64)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    bounds = [int(np.searchsorted(cum, cum[-1] * r / world, side="left")) for r in range(world + 1)]
    bounds[0], bounds[-1] = 0, n_ch
    return list(range(bounds[rank], bounds[rank + 1]))


def gather_by_cut(values: np.ndarray, cuts: Sequence[int], n_ch: int, group=None) -> np.ndarray:
    """All-gather per-CUT values from every rank into one array of n_ch."""
    import torch.distributed as dist
    payload = (list(map(int, cuts)), np.asarray(values, dtype=np.float64).tolist())
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, payload, group=group)
    out = np.full(n_ch, np.nan)
    for c, v in parts:
        out[np.asarray(c, dtype=int)] = v
    return out


def max_over_ranks(t: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    x = torch.tensor([float(t)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        x = x.cuda()
    dist.all_reduce(x, op=dist.ReduceOp.MAX, group=group)
    return float(x.item())
