"""Autotuner of the rasteriser configuration: tile shape (16x16, 32x8, 8x32)
x compositing variant of the forward and of the backward, each (warps per
tile 1/2/4/8, i.e. 8/4/2/1 pixels per thread, and 1 or 2 instances staged
per thread per round = Gaussians per batch).

For every tile shape the forward and the backward variants are chosen
separately from their own kernel times (CUDA events around the two calls,
on the workload itself); the tile shapes are then compared by full eager
iterations (projection, binning, compositing, loss, backward, x-step) with
their chosen variants.  Last, where the x-step runs in two parts, the way
its part for the groups without a kept record runs (streamed beside the
compositing adjoint, or a grid after the projection) is chosen by replays
of captured iterations: the streamed form pays where the adjoint is long
enough to hide it.  The fastest is applied and cached per workload
signature."""
from __future__ import annotations

import json
import os
from typing import Dict, Sequence, Tuple

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


def _kernel_times(tr, steps: int) -> Tuple[float, float]:
    """Mean forward and backward compositing times (ms) over the pool
    entries, the model left unchanged."""
    vb = tr.vb
    fw = bw = 0.0
    for i in range(steps + 1):
        p = i % len(tr.view_sets)
        vb.dev_cams.copy_(tr.cam_pool[p])
        D.dg_project(tr.x, vb)
        D.dg_bin_sort(vb)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        D.dg_rasterize_fwd(vb, tr.bg)
        ev[1].record()
        tr._loss(tr.targets[p])
        ev[2].record()
        D.dg_rasterize_bwd_records(vb, bg=tr.bg)
        ev[3].record()
        torch.cuda.synchronize()
        if i > 0:
            fw += ev[0].elapsed_time(ev[1]) / steps
            bw += ev[2].elapsed_time(ev[3]) / steps
    if tr.overflowed():
        return float("inf"), float("inf")
    return fw, bw


def _time_graph_steps(tr, steps: int, consensus: bool = False) -> float:
    """Mean time (ms) of replayed iterations with or without a consensus,
    the graphs of every pool entry captured afresh before the timing (and
    dropped afterwards)."""
    tr.graphs.clear()
    tr.prepare_graphs((consensus,))
    tr.step(consensus=consensus)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        tr.step(consensus=consensus)
    e1.record()
    torch.cuda.synchronize()
    tr.graphs.clear()
    if tr.overflowed():
        return float("inf")
    return e0.elapsed_time(e1) / steps


def _apply(tr, best: Dict) -> None:
    tr.set_tile(tuple(best["tile"]))
    v = list(best["fwd"]) + list(best["bwd"])
    tr.set_variant(*v)
    D.set_raster_variant(*v)
    if best.get("idle_mode") is not None:
        tr.idle_mode = best["idle_mode"]
        tr.graphs.clear()


def tune(tr, tiles: Sequence = TILES, warps: Sequence[int] = WARPS, stages: Sequence[int] = STAGES,
         steps: int = 3, use_cache: bool = True, idle_modes: Sequence[str] = ("stream", "grid"),
         consensus: bool = False) -> Dict:
    """Tile shape, then forward and backward variants, then (with the x-step
    split) the side stream's form, timed by graph replays of iterations with
    `consensus` as the run takes them, each form twice in alternation and
    its best kept."""
    key = signature(tr)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except ValueError:
            cache = {}
    if use_cache and key in cache and "fwd" in cache[key]:
        best = cache[key]
        _apply(tr, best)
        return dict(best, cached=True)
    results = []
    for tile in tiles:
        tr.set_tile(tile)
        per = {}
        for w in warps:
            for s in stages:
                tr.set_variant(w, s)
                per[(w, s)] = _kernel_times(tr, steps)
        bf = min(per, key=lambda v: per[v][0])
        bb = min(per, key=lambda v: per[v][1])
        tr.set_variant(*bf, *bb)
        ms = _time_steps(tr, steps)
        results.append({"tile": list(tile), "fwd": list(bf), "bwd": list(bb), "ms": round(ms, 4),
                        "fwd_ms": round(per[bf][0], 4), "bwd_ms": round(per[bb][1], 4),
                        "variants": {f"{w},{s}": [round(per[(w, s)][0], 4), round(per[(w, s)][1], 4)]
                                     for (w, s) in per}})
    best = min(results, key=lambda r: r["ms"])
    _apply(tr, best)
    idle = None
    if tr._split_xstep() and len(idle_modes) > 1:
        idle = {}
        for _ in range(2):
            for mode in idle_modes:
                tr.idle_mode = mode
                t = round(_time_graph_steps(tr, 4 * steps, consensus), 4)
                idle[mode] = min(idle.get(mode, t), t)
        best = dict(best, idle_mode=min(idle, key=idle.get))
        _apply(tr, best)
    out = dict(best, candidates=results, idle_modes=idle, cached=False)
    if use_cache:
        cache[key] = {k: best[k] for k in ("tile", "fwd", "bwd", "ms", "idle_mode") if k in best}
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return out
