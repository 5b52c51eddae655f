"""Autotuner of the enumeration launch: lanes per walker, warps per block,
blocks per SM and the split (how many subtree prefixes per instance, i.e.
how many top levels the splitter expands, and the deepest it may go).

Each candidate is timed on the batch it will run: the device time of a whole
step (reduce + split + enumerate + collect, CUDA events inside the library),
best of `repeats` steps after one warm-up step.  Two strategies:

* ``grid``: every point of the grid (exhaustive);
* ``descent``: coordinate descent -- start from the library defaults, try
  every value of one parameter with the others fixed, keep the best, go on
  to the next parameter, and sweep again until a sweep changes nothing (at
  most `sweeps` sweeps).  It times sum(len(values)) candidates per sweep
  instead of their product, cheap enough to run before a benchmark.

A candidate the library rejects (a shape that does not fit) counts as
infinitely slow.  Results are cached per (GPU name, batch shape) in a JSON
file when a path is given.  Lanes change the summation order of ||w||_1 and
with it the node counts; every other parameter leaves the nodes unchanged.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict, List, Optional, Sequence

from . import instances as I
from . import msp as M

DEFAULT_GRID = {
    "lanes": (8, 16),
    "warps_per_block": (4, 8),
    "blocks_per_sm": (0, 1, 2, 4),     # 0: as many as fit (occupancy)
    "split_target": (0, 256, 1024, 4096, 16384),
    "split_depth": (24, 12),
}
# starting point of the descent: the library's defaults
START = {"lanes": 0, "warps_per_block": 8, "blocks_per_sm": 0, "split_target": 0, "split_depth": 24}


def _key(instances: Sequence) -> str:
    import torch
    dims = sorted({(x.m, x.n) for x in instances})
    return f"{torch.cuda.get_device_name()}|{len(instances)}|{dims[0]}..{dims[-1]}"


def time_step(instances: Sequence, repeats: int = 1, **opts) -> float:
    """Device milliseconds of one whole step (reduce + split + enumerate +
    collect), best of `repeats` after one warm-up step."""
    pk = I.pack(list(instances))
    ctx = M.Context(**opts)
    best = float("inf")
    try:
        for r in range(repeats + 1):
            ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
            ctx.msp_run_async()
            ctx.msp_wait()
            ph = ctx.msp_phase_ms()
            if r > 0:
                best = min(best, ph["reduce"] + ph["split"] + ph["enumerate"] + ph["collect"])
    finally:
        ctx.close()
    return best


def _timed(instances, repeats, opts, table, seen):
    key = tuple(sorted(opts.items()))
    if key in seen:
        return seen[key]
    row = {"opts": dict(opts)}
    try:
        row["ms"] = time_step(instances, repeats=repeats, **opts)
    except M.MspError as e:   # e.g. a shape that does not fit this GPU
        row["ms"] = float("inf")
        row["opts"]["error"] = str(e)
    table.append(row)
    seen[key] = row["ms"]
    return row["ms"]


def _grid(instances, grid, repeats):
    names = list(grid)
    table: List[Dict] = []
    seen: Dict = {}
    for values in itertools.product(*(grid[n] for n in names)):
        _timed(instances, repeats, dict(zip(names, values)), table, seen)
    return table


def _descent(instances, grid, repeats, sweeps):
    table: List[Dict] = []
    seen: Dict = {}
    cur = {n: (START[n] if n in START and START[n] in grid[n] else grid[n][0]) for n in grid}
    best = _timed(instances, repeats, cur, table, seen)
    for _ in range(sweeps):
        changed = False
        for n in grid:
            for v in grid[n]:
                if v == cur[n]:
                    continue
                cand = dict(cur, **{n: v})
                ms = _timed(instances, repeats, cand, table, seen)
                if ms < best:
                    best, cur, changed = ms, cand, True
        if not changed:
            break
    return table


def tune(instances: Sequence, grid: Optional[Dict] = None, cache: Optional[str] = None,
         repeats: int = 1, strategy: str = "grid", sweeps: int = 2) -> Dict:
    """Returns {"opts": best option dict, "ms": its step time, "table": [...],
    "strategy": ...}."""
    grid = grid or DEFAULT_GRID
    key = _key(instances)
    if cache and os.path.exists(cache):
        saved = json.load(open(cache))
        if key in saved:
            return saved[key]
    if strategy == "grid":
        table = _grid(instances, grid, repeats)
    elif strategy == "descent":
        table = _descent(instances, grid, repeats, sweeps)
    else:
        raise ValueError(f"unknown strategy {strategy}")
    best = min(table, key=lambda r: r["ms"])
    out = {"opts": {k: v for k, v in best["opts"].items() if k != "error"}, "ms": best["ms"], "table": table,
           "strategy": strategy}
    if cache:
        saved = json.load(open(cache)) if os.path.exists(cache) else {}
        saved[key] = out
        with open(cache, "w") as f:
            json.dump(saved, f, indent=1)
    return out
