"""Tile-shape autotuner for the batched sweep.

A CTA of the batched sweep has 128 threads, one cell each, laid out as tile_x cells along x
times 128/tile_x rows, or (tile_x = 1) as 128 consecutive cells in storage order.  Narrow or
ragged rows waste lanes on x-tiles; linear tiles waste none but pay two integer divisions per
cell; wide x-tiles give the longest contiguous runs per plane.  The tuner groups domains into
size classes by nx, times the batched sweep of each class for every candidate (CUDA events on
the batch's stream, after warm-up), and keeps the fastest per class (highest cell updates
per second).
Results do not depend on the tile shape, only the speed does.
"""
from __future__ import annotations

import json
import os

from . import capi

CANDIDATES = (1, 32, 64, 128)


def size_class(prm) -> str:
    """Class key of a domain: nx bucket (<=32, <=64, <=128, <=512, larger) and tube / box."""
    for b in (32, 64, 128, 512):
        if prm.nx <= b:
            nb = b
            break
    else:
        nb = 4096
    shape = "tube" if prm.ny * prm.nz <= 64 else "box"
    return f"nx{nb}-{shape}"


def _time_batch(handles, tile_x, steps, stream):
    import torch
    b = capi.grlb_batch_create(handles, use_graph=1, schedule=capi.SCHED_TABLE_CONST)
    try:
        capi.grlb_batch_set_stream(b, stream.cuda_stream)
        capi.grlb_batch_set_tile_x(b, [tile_x] * len(handles))
        capi.grlb_batch_step(b, 4)  # warm-up (also captures the graph)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        capi.grlb_batch_step(b, steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3
    finally:
        capi.grlb_batch_destroy(b)


def tune(cases, steps: int = 20, candidates=CANDIDATES, stream=None) -> dict:
    """Measure every candidate tile width per size class of `cases` (inputs.Case list).
    Returns {class: {"tile_x": best, "mlups": {width: MLUP/s}}}."""
    import torch
    stream = stream or torch.cuda.Stream()
    classes: dict[str, list] = {}
    for c in cases:
        classes.setdefault(size_class(c.params), []).append(c)
    table = {}
    for key, members in classes.items():
        doms = []
        for c in members:
            d = capi.Domain(c.params, stream=stream.cuda_stream)
            d.init(c.rho, c.u, c.p)
            doms.append(d)
        cells = sum(c.params.ncells for c in members)
        res = {}
        for tx in candidates:
            if tx > 32 and all(c.params.nx <= tx // 2 for c in members):
                continue  # the tile would leave more than half its lanes idle everywhere
            dt = _time_batch([d.h for d in doms], tx, steps, stream)
            res[tx] = cells * steps / dt / 1e6
        for d in doms:
            d.close()
        best = max(res, key=res.get)
        table[key] = {"tile_x": int(best), "mlups": {str(k): v for k, v in res.items()}}
    return table


def plan(cases, table: dict) -> list:
    """Per-domain tile widths for `cases` from a tuning table (0 = library default)."""
    return [int(table.get(size_class(c.params), {}).get("tile_x", 0)) for c in cases]


def save(table: dict, path: str):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump(table, f, indent=1)


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)
