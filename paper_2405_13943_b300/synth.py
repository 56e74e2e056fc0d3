"""Seeded synthetic inputs for the DOGS hot path.

This module is the only code shared by the CUDA path and the FP64 oracle.  It
draws random numbers and builds scene geometry (points, camera poses, block
membership); it contains none of the method's arithmetic: no projection, no
compositing, no loss, no ADMM update.  Everything is returned in a neutral
layout of float32 numpy arrays that both sides convert to their own layout.

Neutral layout of a Gaussian set (n Gaussians, SH degree D, K=(D+1)^2 coefs):
  means   (n, 3)   world position
  quats   (n, 4)   (w, x, y, z), not normalised
  log_scales (n, 3)
  opacity_logits (n,)
  sh      (n, K, 3)  coefficient k = l*l + l + m, channel last

The workloads follow the synthetic stand-ins for the paper's aerial datasets
(Mill19, UrbanScene3D, MatrixCity are not available): a cube scene for the
small single-view case, and a city height-field law for the large ones.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Real spherical-harmonic DC basis value 1/(2*sqrt(pi)); used only to turn a
# wanted flat colour into a DC coefficient when drawing inputs.
_Y00 = 0.28209479177387814


@dataclasses.dataclass
class Gaussians:
    means: np.ndarray
    quats: np.ndarray
    log_scales: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def sh_degree(self) -> int:
        return int(round(math.sqrt(self.sh.shape[1]))) - 1

    def subset(self, idx) -> "Gaussians":
        idx = np.asarray(idx)
        return Gaussians(self.means[idx].copy(), self.quats[idx].copy(),
                         self.log_scales[idx].copy(),
                         self.opacity_logits[idx].copy(), self.sh[idx].copy())

    def copy(self) -> "Gaussians":
        return self.subset(np.arange(self.n))

    @staticmethod
    def concat(parts: Sequence["Gaussians"]) -> "Gaussians":
        return Gaussians(np.concatenate([p.means for p in parts]),
                         np.concatenate([p.quats for p in parts]),
                         np.concatenate([p.log_scales for p in parts]),
                         np.concatenate([p.opacity_logits for p in parts]),
                         np.concatenate([p.sh for p in parts]))


@dataclasses.dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    A world point p maps to camera coordinates R @ p + t.  Pixel (px, py)
    covers [px, px+1) x [py, py+1).
    """
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray          # (3, 3) float32
    t: np.ndarray          # (3,) float32
    campos: np.ndarray     # (3,) float32
    near: float = 0.2
    block: int = 0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4)).astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


# --------------------------------------------------------------------------
# Cube scene: the small single-view workload (4,096 Gaussians, 128x128).
# --------------------------------------------------------------------------
def cube_scene(n: int = 4096, seed: int = 1001, sh_degree: int = 0,
               log_scale_mu: float = -3.0, log_scale_sigma: float = 0.3,
               extent: float = 1.0) -> Gaussians:
    """Means U[-extent, extent]^3, log-scales N(mu, sigma^2), random unit
    quaternions, opacity logits N(0,1).  For degree 0 the rendered colour is
    U(0,1), so the DC coefficient is (c - 0.5)/Y00; higher degrees get
    N(0, 0.05^2) coefficients."""
    rng = _rng(seed)
    means = rng.uniform(-extent, extent, (n, 3)).astype(np.float32)
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3)).astype(np.float32)
    quats = random_unit_quats(rng, n)
    ologit = rng.standard_normal(n).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32)
    colour = rng.uniform(0.0, 1.0, (n, 3))
    sh[:, 0, :] = ((colour - 0.5) / _Y00).astype(np.float32)
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, K - 1, 3)).astype(np.float32)
    return Gaussians(means, quats, log_scales, ologit, sh)


def cube_camera(width: int = 128, height: int = 128, f: float = 120.0,
                distance: float = 4.0, near: float = 0.2) -> Camera:
    """Camera at (0, 0, -distance) looking along +z: world_to_cam = [I | (0,0,d)]."""
    R = np.eye(3, dtype=np.float32)
    t = np.array([0.0, 0.0, distance], np.float32)
    return Camera(width, height, f, f, width / 2.0, height / 2.0, R, t,
                  np.array([0.0, 0.0, -distance], np.float32), near)


# --------------------------------------------------------------------------
# City height-field law: the large aerial workloads.
# --------------------------------------------------------------------------
@dataclasses.dataclass
class CityLayout:
    size: float            # side of the square area (m)
    lot: float             # lot side (m)
    heights: np.ndarray    # (L, L) building height per lot, 0 = open ground
    setback: float         # building inset from the lot border (m)


def city_layout(seed: int, size: float = 1000.0, lot: float = 20.0,
                hmax: float = 60.0, open_frac: float = 0.25,
                setback: float = 3.0) -> CityLayout:
    rng = _rng(seed)
    L = int(round(size / lot))
    h = rng.uniform(0.0, hmax, (L, L))
    h[rng.uniform(size=(L, L)) < open_frac] = 0.0
    return CityLayout(size, lot, h.astype(np.float64), setback)


def city_points(layout: CityLayout, n: int, rng: np.random.Generator,
                jitter_frac: float = 0.02) -> np.ndarray:
    """n points sampled area-proportionally on ground, roofs and walls of the
    layout, then jittered by N(0, (jitter_frac * lot)^2)."""
    L = layout.heights.shape[0]
    lot, sb = layout.lot, layout.setback
    fw = lot - 2 * sb                       # building footprint side
    h = layout.heights
    built = h > 0
    n_built = int(built.sum())
    # surface areas
    a_ground = layout.size ** 2 - n_built * fw * fw
    a_roof = n_built * fw * fw
    a_wall = float((4 * fw * h[built]).sum())
    areas = np.array([a_ground, a_roof, a_wall])
    kind = rng.choice(3, size=n, p=areas / areas.sum())
    pts = np.empty((n, 3), np.float64)
    bi, bj = np.nonzero(built)
    # ground: uniform over the area, rejecting points inside footprints
    ng = int((kind == 0).sum())
    g = np.empty((0, 2))
    while g.shape[0] < ng:
        c = rng.uniform(0, layout.size, (int((ng - g.shape[0]) * 1.6) + 16, 2))
        li = np.minimum((c // lot).astype(int), L - 1)
        loc = c - li * lot
        inside = built[li[:, 0], li[:, 1]] & (loc[:, 0] > sb) & (loc[:, 0] < lot - sb) \
            & (loc[:, 1] > sb) & (loc[:, 1] < lot - sb)
        g = np.concatenate([g, c[~inside]])
    pts[kind == 0, :2] = g[:ng]
    pts[kind == 0, 2] = 0.0
    # roofs: pick a building uniformly (equal roof areas), uniform on its roof
    nr = int((kind == 1).sum())
    b = rng.integers(0, n_built, nr)
    pts[kind == 1, 0] = bi[b] * lot + sb + rng.uniform(0, fw, nr)
    pts[kind == 1, 1] = bj[b] * lot + sb + rng.uniform(0, fw, nr)
    pts[kind == 1, 2] = h[bi[b], bj[b]]
    # walls: pick a building proportionally to its height, then a side
    nw = int((kind == 2).sum())
    hw = h[bi, bj]
    b = rng.choice(n_built, size=nw, p=hw / hw.sum())
    side = rng.integers(0, 4, nw)
    u = rng.uniform(0, fw, nw)
    x0 = bi[b] * lot + sb
    y0 = bj[b] * lot + sb
    wx = np.where(side == 0, x0 + u, np.where(side == 1, x0 + u, np.where(side == 2, x0, x0 + fw)))
    wy = np.where(side == 0, y0, np.where(side == 1, y0 + fw, np.where(side == 2, y0 + u, y0 + u)))
    pts[kind == 2, 0] = wx
    pts[kind == 2, 1] = wy
    pts[kind == 2, 2] = rng.uniform(0, 1, nw) * hw[b]
    pts += rng.normal(0.0, jitter_frac * lot, pts.shape)
    return pts.astype(np.float32)


def city_scene(n: int, seed: int, sh_degree: int = 3, layout_seed: Optional[int] = None,
               log_scale_mu: float = -1.0, log_scale_sigma: float = 0.5) -> Gaussians:
    """Gaussians on the city law: SH DC coefficients U(0,1), the rest
    N(0, 0.05^2); log-scales N(-1, 0.5^2) in metres; opacity logits N(0,1).
    The layout (buildings) depends on layout_seed so that a ground-truth set
    from another seed shares the same city."""
    layout = city_layout(seed if layout_seed is None else layout_seed)
    rng = _rng(seed + 7919)
    means = city_points(layout, n, rng)
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3)).astype(np.float32)
    quats = random_unit_quats(rng, n)
    ologit = rng.standard_normal(n).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh = np.empty((n, K, 3), np.float32)
    sh[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, K - 1, 3))
    return Gaussians(means, quats, log_scales, ologit, sh)


def look_camera(pos, yaw: float, pitch: float, width: int, height: int,
                f: float, near: float = 1.0, block: int = 0) -> Camera:
    """Camera at pos (z up world), heading yaw (rad, from +x towards +y) and
    pitched down by `pitch` (rad; pi/2 looks straight down)."""
    cp, sp = math.cos(pitch), math.sin(pitch)
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    fwd = np.array([cp * cy_, cp * sy_, -sp])
    right = np.array([sy_, -cy_, 0.0])
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd]).astype(np.float64)
    pos = np.asarray(pos, np.float64)
    t = -(R @ pos)
    return Camera(width, height, f, f, width / 2.0, height / 2.0,
                  R.astype(np.float32), t.astype(np.float32),
                  pos.astype(np.float32), near, block)


def focal_for_hfov(width: int, hfov_deg: float) -> float:
    return (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)


def grid_cameras(seed: int, n_side: int = 10, size: float = 1000.0,
                 altitude: float = 120.0, width: int = 1920, height: int = 1080,
                 hfov_deg: float = 60.0) -> List[Camera]:
    """Cameras on an n_side x n_side grid at `altitude`, pitch U(45, 90) deg,
    random yaw."""
    rng = _rng(seed)
    f = focal_for_hfov(width, hfov_deg)
    cams = []
    step = size / n_side
    for i in range(n_side):
        for j in range(n_side):
            pos = ((i + 0.5) * step, (j + 0.5) * step, altitude)
            cams.append(look_camera(pos, rng.uniform(0, 2 * math.pi),
                                    math.radians(rng.uniform(45, 90)),
                                    width, height, f))
    return cams


# --------------------------------------------------------------------------
# Block decomposition with shared boundary Gaussians.
# --------------------------------------------------------------------------
@dataclasses.dataclass
class BlockSplit:
    """K block-local models over one global set.

    copy_gid     (Nc,)  global id of every local copy; block k owns copies
                        [blk_off[k], blk_off[k+1]); inside a block shared
                        copies come first, each part sorted by global id
    blk_off      (K+1,)
    blk_nshared  (K,)   number of shared copies at the start of each block
    g_off, g_copies     CSR over globals: the copies of global i are
                        g_copies[g_off[i]:g_off[i+1]] (ascending block)
    n_shared_globals    globals [0, n_shared_globals) are the shared ones
    cells        (K, 4) xmin, xmax, ymin, ymax of each block's ground cell
    band         width of the sharing band (m)
    """
    copy_gid: np.ndarray
    blk_off: np.ndarray
    blk_nshared: np.ndarray
    g_off: np.ndarray
    g_copies: np.ndarray
    n_shared_globals: int
    cells: np.ndarray
    band: float

    @property
    def K(self) -> int:
        return int(self.blk_off.shape[0] - 1)

    @property
    def n_copies(self) -> int:
        return int(self.copy_gid.shape[0])

    @property
    def n_globals(self) -> int:
        return int(self.g_off.shape[0] - 1)

    def copy_shared(self) -> np.ndarray:
        f = np.zeros(self.n_copies, np.uint8)
        for k in range(self.K):
            f[self.blk_off[k]:self.blk_off[k] + self.blk_nshared[k]] = 1
        return f


def _quantile_splits(v: np.ndarray, loads: Sequence[float]) -> np.ndarray:
    c = np.cumsum(np.asarray(loads, np.float64))
    c = c[:-1] / c[-1]
    return np.quantile(v, c) if len(c) else np.zeros(0)


def grid_split(xy: np.ndarray, cols: int, rows: int, loads: Sequence[float],
               shared_frac: float) -> tuple:
    """Split ground positions xy (n,2) into cols x rows cells.

    Columns are cut at x quantiles matching the summed loads of their cells;
    each column is then cut at y quantiles of its own points.  Returns
    (cells (K,4), membership (n,K) bool, band) where a point belongs to its
    own cell and, if it lies within `band` of an interior cell border, to
    every cell whose box expanded by `band` contains it.  `band` is picked so
    that `shared_frac` of the points end up in two or more cells."""
    K = cols * rows
    loads = np.asarray(loads, np.float64).reshape(cols, rows)
    x, y = xy[:, 0].astype(np.float64), xy[:, 1].astype(np.float64)
    lo_x, hi_x = x.min() - 1.0, x.max() + 1.0
    lo_y, hi_y = y.min() - 1.0, y.max() + 1.0
    xs = np.concatenate([[lo_x], _quantile_splits(x, loads.sum(1)), [hi_x]])
    cells = np.zeros((K, 4))
    own = np.zeros(x.shape[0], np.int64)
    for c in range(cols):
        in_col = (x >= xs[c]) & (x < xs[c + 1]) if c < cols - 1 else (x >= xs[c])
        ys = np.concatenate([[lo_y], _quantile_splits(y[in_col], loads[c]), [hi_y]])
        for r in range(rows):
            k = c * rows + r
            cells[k] = (xs[c], xs[c + 1], ys[r], ys[r + 1])
            sel = in_col & (y >= ys[r]) & ((y < ys[r + 1]) if r < rows - 1 else True)
            own[sel] = k
    # distance of each point to the nearest interior border of its own cell
    cx0, cx1, cy0, cy1 = (cells[own, i] for i in range(4))
    d = np.full(x.shape[0], np.inf)
    for edge, val, coord in ((cx0, lo_x, x), (cx1, hi_x, x), (cy0, lo_y, y), (cy1, hi_y, y)):
        interior = np.abs(edge - val) > 1e-9
        dd = np.abs(coord - edge)
        d = np.where(interior, np.minimum(d, dd), d)
    band = float(np.quantile(d[np.isfinite(d)], shared_frac)) if shared_frac > 0 else 0.0
    member = np.zeros((x.shape[0], K), bool)
    for k in range(K):
        x0, x1, y0, y1 = cells[k]
        member[:, k] = (x >= x0 - band) & (x < x1 + band) & (y >= y0 - band) & (y < y1 + band)
    member[np.arange(x.shape[0]), own] = True
    return cells, member, band


def block_split(xy: np.ndarray, cols: int, rows: int, loads: Sequence[float],
                shared_frac: float) -> tuple:
    """Build the copy layout for a grid split.  Returns (BlockSplit, order)
    where `order` maps new global ids to the caller's point indices: shared
    globals are numbered first (by position along the first block that holds
    them), then unshared globals block by block."""
    cells, member, band = grid_split(xy, cols, rows, loads, shared_frac)
    return split_layout(xy, member, cells, band)


def morton2d(xy: np.ndarray) -> np.ndarray:
    """Z-order (Morton) code of ground positions: x and y quantised to 16
    bits each over their bounding box, bits interleaved (x in the even
    bits)."""
    xy = np.asarray(xy, np.float64)
    if xy.shape[0] == 0:
        return np.zeros(0, np.uint64)
    lo, hi = xy.min(0), xy.max(0)
    q = np.clip((xy - lo) / np.maximum(hi - lo, 1e-30) * 65535.0, 0, 65535).astype(np.uint64)

    def spread(v):
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x33333333)
        return (v | (v << np.uint64(1))) & np.uint64(0x55555555)
    return spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1))


def split_layout(xy: np.ndarray, member: np.ndarray, cells: np.ndarray, band: float) -> tuple:
    """Copy layout of a membership (n, K) bool (every point in at least one
    block).  Returns (BlockSplit, order), `order` mapping new global ids to
    the caller's point indices: shared globals first (by first block, then
    Z-order of the ground position), then unshared globals block by block
    in Z-order.  The Z-order keeps the copies one view sees in compact
    index ranges, so that projection loads and record gathers coalesce."""
    K = member.shape[1]
    n = xy.shape[0]
    if not member.any(1).all():
        raise ValueError("every point needs a block")
    cnt = member.sum(1)
    shared = cnt >= 2
    first_blk = np.argmax(member, axis=1)
    # renumber: shared first (sorted by first block, then Z-order), unshared by block
    key_sh = np.argsort((first_blk.astype(np.uint64) << np.uint64(32)) | morton2d(xy), kind="stable")
    sh_pts = key_sh[shared[key_sh]]
    un_pts = key_sh[~shared[key_sh]]
    un_pts = un_pts[np.argsort(first_blk[un_pts], kind="stable")]
    order = np.concatenate([sh_pts, un_pts])
    member_g = member[order]
    ns = int(shared.sum())
    gid_all = np.arange(n)
    copy_gid, blk_off, blk_nsh = [], [0], []
    for k in range(K):
        m = member_g[:, k]
        g_sh = gid_all[:ns][m[:ns]]
        g_un = gid_all[ns:][m[ns:]]
        copy_gid.append(g_sh)
        copy_gid.append(g_un)
        blk_nsh.append(g_sh.shape[0])
        blk_off.append(blk_off[-1] + g_sh.shape[0] + g_un.shape[0])
    copy_gid = np.concatenate(copy_gid).astype(np.int32)
    # CSR over globals, copies in ascending block order
    ordc = np.argsort(copy_gid, kind="stable")
    counts = np.bincount(copy_gid, minlength=n)
    g_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    split = BlockSplit(copy_gid, np.asarray(blk_off, np.int64), np.asarray(blk_nsh, np.int64),
                       g_off, ordc.astype(np.int32), ns, cells, band)
    return split, order


def dirichlet_loads(seed: int, K: int, conc: float = 2.0) -> np.ndarray:
    return _rng(seed).dirichlet(np.full(K, conc))


def block_views(split: BlockSplit, seed: int, per_block: int, width: int, height: int,
                pitch_deg: float = 45.0, altitude: float = 120.0,
                hfov_deg: float = 60.0, jitter: float = 0.3,
                ground: float = 0.0) -> List[Camera]:
    """`per_block` aerial views per block at a fixed pitch, each looking at a
    point drawn inside the block's cell (central `1 - 2*jitter` part), random
    yaw; views are returned grouped by block."""
    rng = _rng(seed)
    f = focal_for_hfov(width, hfov_deg)
    p = math.radians(pitch_deg)
    cams = []
    for k in range(split.K):
        x0, x1, y0, y1 = split.cells[k]
        for _ in range(per_block):
            tx = x0 + (x1 - x0) * rng.uniform(jitter, 1 - jitter)
            ty = y0 + (y1 - y0) * rng.uniform(jitter, 1 - jitter)
            yaw = rng.uniform(0, 2 * math.pi)
            dist = altitude / math.tan(p)
            pos = (tx - dist * math.cos(yaw), ty - dist * math.sin(yaw), ground + altitude)
            cams.append(look_camera(pos, yaw, p, width, height, f, near=1.0, block=k))
    return cams


def street_views(split: BlockSplit, seed: int, per_block: int, width: int, height: int, lot: float = 20.0,
                 eye: float = 1.7, pitch_deg: tuple = (0.0, 10.0), hfov_deg: float = 90.0,
                 jitter: float = 0.2) -> List[Camera]:
    """`per_block` street-level views per block: the camera stands at eye
    height on a street of the city law (the gaps between building lots run
    along the lot borders, x or y a multiple of `lot`) inside the block's
    cell, looks along the street in one of its two directions, pitched down
    by U(pitch_deg); views are returned grouped by block."""
    rng = _rng(seed)
    f = focal_for_hfov(width, hfov_deg)
    cams = []
    for k in range(split.K):
        x0, x1, y0, y1 = split.cells[k]
        for _ in range(per_block):
            tx = x0 + (x1 - x0) * rng.uniform(jitter, 1 - jitter)
            ty = y0 + (y1 - y0) * rng.uniform(jitter, 1 - jitter)
            if rng.uniform() < 0.5:             # a street along y, at a lot border in x
                pos = (round(tx / lot) * lot, ty, eye)
                yaw = math.pi / 2 if rng.uniform() < 0.5 else -math.pi / 2
            else:                                # a street along x
                pos = (tx, round(ty / lot) * lot, eye)
                yaw = 0.0 if rng.uniform() < 0.5 else math.pi
            p = math.radians(rng.uniform(*pitch_deg))
            cams.append(look_camera(pos, yaw, p, width, height, f, near=0.5, block=k))
    return cams


def random_pose_cameras(seed: int, n: int, resolutions: Sequence[tuple],
                        probs: Sequence[float], size: float = 1000.0,
                        alt: tuple = (50.0, 150.0), pitch_deg: tuple = (30.0, 90.0),
                        hfov_deg: float = 60.0) -> List[Camera]:
    """Serving requests: poses uniform over the scene, altitude U(alt),
    yaw U(0, 2pi), pitch U(pitch_deg); resolution drawn from `resolutions`."""
    rng = _rng(seed)
    cams = []
    ridx = rng.choice(len(resolutions), size=n, p=np.asarray(probs) / np.sum(probs))
    for i in range(n):
        w, h = resolutions[ridx[i]]
        pos = (rng.uniform(0, size), rng.uniform(0, size), rng.uniform(*alt))
        cams.append(look_camera(pos, rng.uniform(0, 2 * math.pi),
                                math.radians(rng.uniform(*pitch_deg)), w, h,
                                focal_for_hfov(w, hfov_deg), near=1.0))
    return cams


def poisson_arrivals(seed: int, rate: float, duration: float) -> np.ndarray:
    rng = _rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        out.append(t)
    return np.asarray(out)


def random_image(seed: int, height: int, width: int) -> np.ndarray:
    """(3, H, W) float32 target image, U(0,1)."""
    return _rng(seed).uniform(0.0, 1.0, (3, height, width)).astype(np.float32)


def random_like(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    return (_rng(seed).standard_normal(shape) * scale).astype(np.float32)


# --------------------------------------------------------------------------
# The DOGS block workloads (K uneven blocks over one aerial city scene).
# --------------------------------------------------------------------------
@dataclasses.dataclass
class DogsWorkload:
    split: BlockSplit
    z0: Gaussians                  # global model, numbered as in split
    views: List[List[Camera]]      # pool entries; each holds per_block views per block, grouped by block
    gt: Gaussians                  # ground-truth set of the same law (targets are rendered from it)


def dogs_workload(n_global: int, cols: int, rows: int, shared_frac: float, seed: int,
                  views_per_step: int = 1, pool: int = 4, width: int = 1920, height: int = 1080,
                  pitch_deg: float = 45.0, altitude: float = 120.0, sh_degree: int = 3,
                  loads: Optional[Sequence[float]] = None, cameras: str = "aerial",
                  log_scale_mu: float = -1.0) -> DogsWorkload:
    """City-law scene of n_global Gaussians split on a cols x rows ground
    grid at load quantiles (Dirichlet(2) from the seed unless given), with
    shared_frac of the Gaussians on interior borders shared by 2-4 blocks;
    `pool` steps' worth of views, views_per_step per block each:
      cameras="aerial"  block_views at pitch_deg and altitude;
      cameras="grid"    (one block) views drawn from a 10 x 10 grid of
                        cameras at `altitude`, pitch U(45, 90) deg;
      cameras="street"  street_views at eye height along the streets."""
    K = cols * rows
    z = city_scene(n_global, seed, sh_degree=sh_degree, log_scale_mu=log_scale_mu)
    if loads is None:
        loads = dirichlet_loads(seed + 3, K)
    split, order = block_split(z.means[:, :2], cols, rows, loads, shared_frac)
    z = z.subset(order)
    per = views_per_step * pool
    if cameras == "aerial":
        allv = block_views(split, seed + 2, per, width, height, pitch_deg, altitude)
    elif cameras == "street":
        allv = street_views(split, seed + 2, per, width, height)
    elif cameras == "grid":
        if K != 1:
            raise ValueError("grid cameras serve a single block")
        grid = grid_cameras(seed + 2, 10, altitude=altitude, width=width, height=height)
        pick = _rng(seed + 5).choice(len(grid), size=per, replace=per > len(grid))
        allv = [grid[i] for i in pick]
    else:
        raise ValueError(f"unknown camera law {cameras!r}")
    views = []
    for p in range(pool):
        vs = []
        for k in range(K):
            vs.extend(allv[k * per + p * views_per_step: k * per + (p + 1) * views_per_step])
        views.append(vs)
    gt = city_scene(n_global, seed + 1, sh_degree=sh_degree, layout_seed=seed, log_scale_mu=log_scale_mu)
    return DogsWorkload(split, z, views, gt)
