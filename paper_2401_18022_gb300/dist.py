"""Host-side multi-GPU logic (one process per GPU).

Every CUT's eta is independent, and so is every launch-power profile:
  * weak scaling (the benchmark's default): each rank evaluates its own full
    system for an independent seeded launch-power profile (``rank_powers``),
    with no data-path collective;
  * strong scaling (Sec. III: a group of channels under test per GPU): the
    CUTs of one system are split across ranks (``shard_cuts``).  The forward
    needs one exchange, the gather of eta (``gather_by_cut``); the gradient
    (``grad_split``) adds one all-reduce of the per-channel dT/dP parts,
    because the chain rule of a CUT reaches every launch power.
The timing reduction (max over ranks) is the only other collective.
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


def gather_by_cut(values, cuts: Sequence[int], n_ch: int, group=None):
    """All-gather per-CUT values from every rank into one array of n_ch.

    Each rank writes its CUTs into a zero vector and one all-reduce (sum)
    assembles them; with disjoint shards every entry has exactly one
    contribution, so the sum is exact.  ``values`` may be a numpy array or a
    torch tensor (CUDA tensors stay on the device for NCCL); the result has
    the same kind."""
    import torch
    import torch.distributed as dist
    is_t = isinstance(values, torch.Tensor)
    dev = values.device if is_t else torch.device("cpu")
    if dist.get_backend(group) == "nccl" and dev.type != "cuda":
        dev = torch.device("cuda", torch.cuda.current_device())
    full = torch.zeros(n_ch, dtype=torch.float64, device=dev)
    idx = torch.as_tensor(list(map(int, cuts)), dtype=torch.long, device=dev)
    v = values.to(device=dev, dtype=torch.float64) if is_t else torch.as_tensor(np.asarray(values, dtype=np.float64), device=dev)
    full[idx] = v[:len(idx)]
    dist.all_reduce(full, op=dist.ReduceOp.SUM, group=group)
    return full if is_t else full.cpu().numpy()


def grad_split(eng, wl, P, rank: int, world: int, group=None, weights: Sequence[float] = None):
    """One throughput gradient split over `world` ranks by CUT shards.

    ``eng`` provides the two phases of isrs_gn_grad_shard_fwd/_bwd
    (``grad_shard_fwd(wl, cuts, P) -> eta of the shard's CUTs`` and
    ``grad_shard_bwd(eta_all, with_direct) -> {"dT_dP", "snr", "T"}``).
    Steps: this rank's CUT shard (balanced by ``weights``); the fused forward +
    adjoint over it; the gather of eta; this shard's part of dT/dP, rank 0
    adding the terms outside every eta; one all-reduce (sum) of the parts.
    With world == 1 no collective is issued.  Returns the full dT/dP, the
    SNR of every channel, T, eta of every channel and this rank's CUTs."""
    cuts = shard_cuts(wl.n_ch, rank, world, weights)
    eta_s = eng.grad_shard_fwd(wl, cuts, P)
    if world > 1:
        eta_all = gather_by_cut(eta_s, cuts, wl.n_ch, group)
    else:
        eta_all = eta_s
    out = eng.grad_shard_bwd(eta_all, with_direct=(rank == 0))
    g = out["dT_dP"]
    if world > 1:
        import torch
        import torch.distributed as dist
        is_t = isinstance(g, torch.Tensor)
        gt = g if is_t else torch.as_tensor(np.asarray(g, dtype=np.float64))
        if dist.get_backend(group) == "nccl" and gt.device.type != "cuda":
            gt = gt.cuda()
        dist.all_reduce(gt, op=dist.ReduceOp.SUM, group=group)
        g = gt if is_t else gt.cpu().numpy()
    return {"dT_dP": g, "snr": out["snr"], "T": out["T"], "eta": eta_all, "cuts": cuts}


def max_over_ranks(t: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    x = torch.tensor([float(t)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        x = x.cuda()
    dist.all_reduce(x, op=dist.ReduceOp.MAX, group=group)
    return float(x.item())
