"""Shared test helpers: input curation by the oracle's decision margins.

Floating-point decisions of the rasteriser (the tile rectangle, the radius,
the 1/255 skip, the T < 1e-4 stop, the 0.99 clamp, the colour clamp) can
differ between FP64 and FP32 when a value sits right at its threshold.
Parity is only asserted where every decision has margin; the oracle reports
the margins and these helpers drop or re-draw the inputs that lack it.
"""
from __future__ import annotations

import json
import os

import numpy as np

from paper_2405_13943_b300 import synth as S


def curate_gaussians(O, g: S.Gaussians, cams, tile_w, tile_h, thr=1e-4) -> S.Gaussians:
    """Drop Gaussians whose projection decisions lack margin in any view."""
    x = O.params_from(g)
    keep = np.ones(g.n, bool)
    for c in cams:
        p = O.project(x, g.sh_degree, c, tile_w, tile_h)
        keep &= p["margin"] >= thr
    return g.subset(np.nonzero(keep)[0])


def pixel_mask(views, thr=1e-4, grad=False):
    """Per view, True where every value decision of the pixel (and with
    grad=True also the 0.99 clamp, which only decides gradients) has relative
    margin >= thr."""
    if grad:
        return [(v["margin"] >= thr) & (v["margin_grad"] >= thr) for v in views]
    return [v["margin"] >= thr for v in views]


def smooth_weights(seed, cams):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1.0, 1.0, (3, c.height, c.width)) for c in cams]


def report(name: str, **values) -> None:
    """Append one JSON line of observed parity figures (excluded and flipped
    pixel counts and the like) to the file named by DOGS_PARITY_REPORT, when
    that variable is set; budgets in the tests are set just above them."""
    path = os.environ.get("DOGS_PARITY_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps({"check": name, **values}) + "\n")
