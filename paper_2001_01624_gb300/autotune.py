"""Autotuner for the batched basis smoothing's work-item shape.

The persistent batched smoothing (ms_basis_rebuild_batch, and the first phase
of ms_solve_batch) hands out (member, tile) items: `tile_cells` consecutive
cells of one member's iteration, taken by `ctas_per_sm` resident blocks per
SM.  Small tiles balance uneven members but pay a queue round trip per item;
large tiles cut the queue traffic but leave SMs idle while a member's last
tiles finish.  tune() times each candidate shape once on the caller's
members (re-smoothing from the block indicator, which changes no result:
every shape gives bitwise the same bases) and caches the fastest per device
in a JSON file; apply() sets the cached shape on a context.
"""
from __future__ import annotations

import json
import os
import time
from typing import Optional, Sequence

from . import binding as B

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
SHAPES = [(256, 4), (512, 4), (1024, 4), (2048, 4), (4096, 2), (1024, 2), (1024, 6), (2048, 6)]


def _device_key(device: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|sm{p.multi_processor_count}"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(ctx, systems: Sequence, bases: Sequence, device: int = 0, shapes=None, repeats: int = 2,
         path: Optional[str] = None, workload: str = "default") -> dict:
    """Time every shape on these members (best of `repeats`), keep the
    fastest, store it under (device, workload) in the cache, set it on ctx."""
    path = path or CACHE
    shapes = list(shapes or SHAPES)
    timings = []
    for tile, cps in shapes:
        B.ms_set_batch_tuning(ctx, tile, cps)
        B.ms_basis_rebuild_batch(ctx, systems, bases)          # warm-up (and scratch sizing)
        best = float("inf")
        for _ in range(repeats):
            t0 = time.perf_counter()
            B.ms_basis_rebuild_batch(ctx, systems, bases)      # returns after the smoothing
            best = min(best, time.perf_counter() - t0)
        timings.append({"tile_cells": tile, "ctas_per_sm": cps, "ms": best * 1e3})
    win = min(timings, key=lambda r: r["ms"])
    cache = _load(path)
    cache.setdefault(_device_key(device), {})[workload] = {"tile_cells": win["tile_cells"],
                                                            "ctas_per_sm": win["ctas_per_sm"],
                                                            "ms": win["ms"], "candidates": timings}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    B.ms_set_batch_tuning(ctx, win["tile_cells"], win["ctas_per_sm"])
    return cache[_device_key(device)][workload]


def apply(ctx, device: int = 0, path: Optional[str] = None, workload: str = "default") -> Optional[dict]:
    """Set the cached shape for this device on ctx; None (library defaults
    kept) when nothing is cached."""
    ent = _load(path or CACHE).get(_device_key(device), {}).get(workload)
    if ent:
        B.ms_set_batch_tuning(ctx, int(ent["tile_cells"]), int(ent["ctas_per_sm"]))
    return ent


def tuned(ctx, systems: Sequence, bases: Sequence, device: int = 0, path: Optional[str] = None,
          workload: str = "default") -> dict:
    """The cached shape for this device and workload, tuning once if absent."""
    ent = apply(ctx, device, path, workload)
    return ent if ent else tune(ctx, systems, bases, device, path=path, workload=workload)
