"""Autotuner of the rasteriser configuration: tile shape (16x16, 32x8, 8x32)
x compositing variant (warps per tile 1/2/4/8, i.e. 8/4/2/1 pixels per
thread, and 1 or 2 instances staged per thread per round = Gaussians per
batch).  Each candidate is timed on the workload itself: full eager
iterations (projection, binning, compositing, loss, backward, x-step) with
CUDA events; the fastest is applied and cached per workload signature."""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence

import torch

from . import dogs as D

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, ".autotune_cache.json")

TILES = ((16, 16), (32, 8), (8, 32))
WARPS = (1, 2, 4, 8)
STAGES = (1, 2)


def signature(tr) -> str:
    c = tr.view_sets[0][0]
    return f"K{tr.split.K}_n{tr.split.n_copies}_V{len(tr.view_sets[0])}_{c.width}x{c.height}_d{tr.x.deg}"


def _time_steps(tr, steps: int) -> float:
    for _ in range(1):
        tr.step(consensus=False, graph=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        tr.step(consensus=False, graph=False)
    e1.record()
    torch.cuda.synchronize()
    if tr.overflowed():
        return float("inf")
    return e0.elapsed_time(e1) / steps


def tune(tr, tiles: Sequence = TILES, warps: Sequence[int] = WARPS, stages: Sequence[int] = STAGES,
         steps: int = 3, use_cache: bool = True) -> Dict:
    key = signature(tr)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except ValueError:
            cache = {}
    if use_cache and key in cache:
        best = cache[key]
        tr.set_tile(tuple(best["tile"]))
        tr.set_variant(best["warps"], best["stage"])
        D.set_raster_variant(best["warps"], best["stage"])
        return dict(best, cached=True)
    results = []
    for tile in tiles:
        tr.set_tile(tile)
        for w in warps:
            for s in stages:
                tr.set_variant(w, s)
                ms = _time_steps(tr, steps)
                results.append({"tile": list(tile), "warps": w, "stage": s, "ms": round(ms, 4)})
    best = min(results, key=lambda r: r["ms"])
    tr.set_tile(tuple(best["tile"]))
    tr.set_variant(best["warps"], best["stage"])
    D.set_raster_variant(best["warps"], best["stage"])
    out = dict(best, candidates=results, cached=False)
    if use_cache:
        cache[key] = {k: best[k] for k in ("tile", "warps", "stage", "ms")}
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return out
