"""Tile-shape autotuner for the persistent quadrature launches.

A work tile is a run of pieces of one CUT; its size (grid points per tile)
and the threads per block set the load balance and the occupancy of the
persistent kernels.  ``tune`` times each candidate on a sample of the
workload (one profile per channel plan) with CUDA events around the batched
call (graph replays after the first call), keeps the fastest, applies it to
the engine and caches it in a JSON file keyed by the workload signature and
the GPU name.
"""
from __future__ import annotations

import json
import os
from typing import Iterable, Optional, Tuple

import numpy as np

DEFAULT_CANDIDATES: Tuple[Tuple[int, int], ...] = tuple(
    (1 << e, t) for e in (17, 18, 19, 20, 21) for t in (128, 256))


def cache_path() -> str:
    return os.environ.get("ISRS_TILE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "isrs_gn", "tiles.json"))


def signature(bw, gpu_name: str) -> str:
    p0 = bw.plans[0]
    sizes = ",".join(str(p.n_ch) for p in bw.plans)
    return f"{gpu_name}|G{p0.G}|N{p0.n_edges}|cells{p0.cell_set}|plans{sizes}"


def _sample(bw):
    from .workloads import BatchedWorkload
    first = {}
    for p, k in enumerate(bw.plan_of_profile):
        first.setdefault(int(k), p)
    idx = sorted(first.values())
    return BatchedWorkload(plans=bw.plans, plan_of_profile=np.asarray([bw.plan_of_profile[p] for p in idx]),
                           P_W=[bw.P_W[p] for p in idx])


def tune(engine, bw, candidates: Optional[Iterable[Tuple[int, int]]] = None, reps: int = 2,
         use_cache: bool = True) -> dict:
    import torch
    name = torch.cuda.get_device_name(engine.device)
    key = signature(bw, name)
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except Exception:
            cache = {}
    if use_cache and key in cache:
        best = cache[key]
        engine.set_tile(best["points_per_item"], best["threads"])
        return {**best, "cached": True}
    sample = _sample(bw)
    P = torch.tensor(np.concatenate(sample.P_W), dtype=torch.float64, device=f"cuda:{engine.device}")
    st = torch.cuda.current_stream(P.device)
    results = []
    for pts, th in (candidates or DEFAULT_CANDIDATES):
        engine.set_tile(pts, th)
        engine.eta_batched(sample, P)                  # builds tiles and captures the graph
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            engine.eta_batched(sample, P)
            e1.record(st)
            torch.cuda.synchronize(P.device)
            ms.append(e0.elapsed_time(e1))
        results.append({"points_per_item": pts, "threads": th, "ms": float(np.median(ms))})
    best = min(results, key=lambda r: r["ms"])
    engine.set_tile(best["points_per_item"], best["threads"])
    out = {"points_per_item": best["points_per_item"], "threads": best["threads"], "ms": best["ms"],
           "candidates": results}
    if use_cache:
        cache[key] = out
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, path)
    return {**out, "cached": False}
