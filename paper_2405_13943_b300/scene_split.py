"""Scene splitting into K overlapping blocks (Sec. 3.2 "Scene Splitting",
Alg. 1) on top of the library's host entry points dg_scene_split and
dg_scene_assign.

split_scene cuts the ground positions of the initial point cloud by the
recursive bipartition of Alg. 1, expands each cell's tight box by the scale
factor s (1.4 in the paper's experiments) and lets every point covered by a
block's expanded box join that block; points in two or more blocks are the
shared Gaussians of the consensus.  split_views groups the training cameras
by the same expanded boxes, using their centres' ground positions; a camera
outside every box joins the nearest block so that no view is lost.
"""
from __future__ import annotations

import copy
from typing import List, Sequence, Tuple

import numpy as np

from . import _lib as L
from . import synth as S


def _xy(points) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(points, np.float64)[:, :2])
    if p.ndim != 2 or p.shape[1] != 2:
        raise ValueError("positions must be (n, 2) or (n, 3)")
    return p


def split_cells(points, K: int) -> Tuple[np.ndarray, np.ndarray]:
    """Alg. 1 on the ground positions of `points` ((n, 2) or (n, 3)): the
    cell of every point (int32) and each cell's tight box (K, 4) as
    xmin, xmax, ymin, ymax."""
    xy = _xy(points)
    n = xy.shape[0]
    cell = np.empty(n, np.int32)
    boxes = np.empty((K, 4), np.float64)
    L.check(L.lib().dg_scene_split(xy.ctypes.data, n, int(K), cell.ctypes.data, boxes.ctypes.data),
            "dg_scene_split")
    return cell, boxes


def assign(points, boxes: np.ndarray, s: float, own=None, nearest: bool = False) -> np.ndarray:
    """Membership (n, K) bool in the boxes expanded by s (see dg_scene_assign)."""
    xy = _xy(points)
    boxes = np.ascontiguousarray(boxes, np.float64)
    K = boxes.shape[0]
    n = xy.shape[0]
    mask = np.empty(n, np.uint64)
    own_arr = None if own is None else np.ascontiguousarray(own, np.int32)
    L.check(L.lib().dg_scene_assign(xy.ctypes.data, n, boxes.ctypes.data, K, float(s),
                                    None if own_arr is None else own_arr.ctypes.data, int(bool(nearest)),
                                    mask.ctypes.data), "dg_scene_assign")
    bits = np.uint64(1) << np.arange(K, dtype=np.uint64)
    return (mask[:, None] & bits[None, :]) != 0


def split_scene(points, K: int, s: float = 1.4) -> Tuple[S.BlockSplit, np.ndarray]:
    """Blocks of the initial point cloud: (BlockSplit, order) as the copy
    layout the trainer takes, `order` mapping its global ids to point
    indices.  The BlockSplit's cells are the unexpanded tight boxes."""
    cell, boxes = split_cells(points, K)
    member = assign(points, boxes, s, own=cell)
    return S.split_layout(_xy(points), member, boxes, float("nan"))


def split_views(cams: Sequence[S.Camera], boxes: np.ndarray, s: float = 1.4) -> List[List[S.Camera]]:
    """Training cameras of every block: those whose centre lies in the
    block's expanded box (the nearest block for a centre outside all of
    them).  Returns K lists of copies tagged with their block."""
    K = boxes.shape[0]
    if len(cams) == 0:
        return [[] for _ in range(K)]
    pos = np.stack([np.asarray(c.campos, np.float64)[:2] for c in cams])
    member = assign(pos, boxes, s, nearest=True)
    out: List[List[S.Camera]] = [[] for _ in range(K)]
    for i, c in enumerate(cams):
        for k in np.nonzero(member[i])[0]:
            v = copy.copy(c)
            v.block = int(k)
            out[k].append(v)
    return out


def make_blocks(z: S.Gaussians, cams: Sequence[S.Camera], K: int, s: float = 1.4,
                views_per_step: int = 1, pool: int = 1):
    """A K-block problem from an initial model and its training cameras:
    (split, z renumbered to the split's global ids, view_sets) with
    view_sets[p] holding views_per_step views of every block (cycling
    through the block's cameras), grouped by ascending block as the batch
    plan wants them.  A block that received no camera gets no views."""
    split, order = split_scene(z.means, K, s)
    per = split_views(cams, split.cells, s)
    view_sets = []
    for p in range(pool):
        vs = []
        for k in range(K):
            for j in range(views_per_step if per[k] else 0):
                vs.append(per[k][(p * views_per_step + j) % len(per[k])])
        view_sets.append(vs)
    return split, z.subset(order), view_sets
