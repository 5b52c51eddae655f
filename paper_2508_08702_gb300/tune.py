"""Autotuner: lanes per walker, warps per block and the split size.

Each candidate is timed on the batch it will run (device time of a whole
step from CUDA events, after one warm-up step); the fastest wins.  Results
are cached per (GPU name, batch shape) in a JSON file when a path is given.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict, List, Optional, Sequence

from . import instances as I
from . import msp as M

DEFAULT_GRID = {"lanes": (4, 8, 16), "warps_per_block": (8,), "split_target": (0, 4096)}


def _key(instances: Sequence) -> str:
    import torch
    dims = sorted({(x.m, x.n) for x in instances})
    return f"{torch.cuda.get_device_name()}|{len(instances)}|{dims[0]}..{dims[-1]}"


def time_step(instances: Sequence, repeats: int = 1, **opts) -> float:
    """Device milliseconds of one whole step (reduce + split + enumerate)."""
    pk = I.pack(list(instances))
    ctx = M.Context(**opts)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    best = float("inf")
    for r in range(repeats + 1):
        ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
        ctx.msp_run_async()
        ctx.msp_wait()
        ph = ctx.msp_phase_ms()
        if r > 0:
            best = min(best, ph["reduce"] + ph["split"] + ph["enumerate"] + ph["collect"])
    ctx.close()
    return best


def tune(instances: Sequence, grid: Optional[Dict] = None, cache: Optional[str] = None,
         repeats: int = 1) -> Dict:
    """Returns {"opts": best option dict, "ms": its step time, "table": [...]}"""
    grid = grid or DEFAULT_GRID
    key = _key(instances)
    if cache and os.path.exists(cache):
        saved = json.load(open(cache))
        if key in saved:
            return saved[key]
    names = list(grid)
    table: List[Dict] = []
    for values in itertools.product(*(grid[n] for n in names)):
        opts = dict(zip(names, values))
        try:
            ms = time_step(instances, repeats=repeats, **opts)
        except M.MspError as e:   # e.g. a shape that does not fit this GPU
            ms = float("inf")
            opts["error"] = str(e)
        table.append({"opts": opts, "ms": ms})
    best = min(table, key=lambda r: r["ms"])
    out = {"opts": {k: v for k, v in best["opts"].items() if k != "error"}, "ms": best["ms"], "table": table}
    if cache:
        saved = json.load(open(cache)) if os.path.exists(cache) else {}
        saved[key] = out
        with open(cache, "w") as f:
            json.dump(saved, f, indent=1)
    return out
