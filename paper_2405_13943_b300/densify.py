"""Densification under consensus (Sec. 4: densified at the intervals and
until the iteration of 3DGS, with its adaptive density control; Sec. 5: small
Gaussians pruned).

The trainer accumulates the statistic every iteration (dg_densify_stats in
the captured iteration).  At a densification iteration, right after its
consensus, `densify(trainer, cfg)`:
  1. decides per global Gaussian of z from the summed statistics of all its
     copies (dg_densify_decide) and writes the densified global set in place
     order (dg_densify_emit, split children from seeded normals);
  2. gives every new Gaussian its parent's sharing set (the blocks that held
     the parent) and builds the copy layout: by default on the device in the
     old layout's order, each Gaussian's outputs in its place
     (dg_densify_layout: a few linear passes; shared globals stay first and
     each block's copies keep their order), or with layout="resort" on the
     host with the initial split's numbering rule (shared globals first,
     Z-order of the new positions; dg_layout, as synth.split_layout);
  3. moves the state (dg_gather_rows): z from the emitted set; for every new
     copy whose Gaussian is its parent itself and whose parent had a copy in
     the same block, that copy's x, Adam moments and scaled dual; other
     copies start from their Gaussian's z with zero moments and duals (as
     3DGS zeroes the optimiser state of new points);
  4. rebuilds the anchors, the batch plan and the capacity; captured graphs
     are dropped.
"""
from __future__ import annotations

import time
from dataclasses import dataclass
from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import dogs as D
from . import synth as S


@dataclass
class DensifyConfig:
    interval: int = 200             # densify every `interval` iterations (a multiple of the consensus interval)
    start: int = 500                # first densification iteration
    until: int = 30000              # no densification from this iteration on
    grad_threshold: float = 2e-4    # mean screen-gradient norm (normalised device units)
    percent_dense: float = 0.01     # clone / split boundary on the largest scale, as a fraction of the extent
    min_opacity: float = 0.005      # prune below this opacity
    extent: Optional[float] = None  # scene extent; None: from the camera centres (scene_extent)
    seed: int = 0                   # seed of the split normals (advanced per densification)
    opacity_reset: int = 3000       # cap every opacity at reset_cap every this many iterations (0: never)
    reset_cap: float = 0.01
    layout: str = "inplace"         # "inplace": device, old order kept; "resort": host, initial numbering rule

    def due(self, t: int) -> bool:
        return self.start <= t < self.until and t % self.interval == 0

    def reset_due(self, t: int) -> bool:
        return self.opacity_reset > 0 and 0 < t < self.until and t % self.opacity_reset == 0


def reset_opacity(tr, cfg: DensifyConfig) -> None:
    """The opacity reset of the density control on z and on every copy (their
    moments' opacity lanes restart from zero), after a consensus; the anchors
    z - u are rebuilt."""
    D.dg_reset_opacity(tr.z, cfg.reset_cap)
    D.dg_reset_opacity(tr.x, cfg.reset_cap, tr.m, tr.v)
    D.dg_admm_anchor(tr.z, tr.u, tr.gid, tr.shared, tr.anchor)


def scene_extent(cams: Sequence[S.Camera]) -> float:
    """The extent 3DGS scales its split rule by: 1.1 times the largest
    distance of a camera centre from their mean."""
    c = np.stack([np.asarray(cam.campos, np.float64) for cam in cams])
    return float(1.1 * np.linalg.norm(c - c.mean(0), axis=1).max())


def membership(split: S.BlockSplit) -> np.ndarray:
    """uint64 per global Gaussian: bit k set when block k holds it."""
    m = np.zeros(split.n_globals, np.uint64)
    for k in range(split.K):
        m[split.copy_gid[split.blk_off[k]:split.blk_off[k + 1]]] |= np.uint64(1) << np.uint64(k)
    return m


def parent_membership(old: S.BlockSplit, parent: np.ndarray) -> np.ndarray:
    """uint64 per new Gaussian: the blocks that hold its parent (old global
    parent[j]) in the old layout (dg_layout_membership, host C++)."""
    from . import _lib as L
    old_blk = np.ascontiguousarray(old.blk_off, np.int64)
    old_goff = np.ascontiguousarray(old.g_off, np.int64)
    old_gcp = np.ascontiguousarray(old.g_copies, np.int32)
    par = np.ascontiguousarray(parent, np.int32)
    out = np.empty(max(par.shape[0], 1), np.uint64)
    L.check(L.lib().dg_layout_membership(old_blk.ctypes.data, old_goff.ctypes.data, old_gcp.ctypes.data,
                                         old_goff.shape[0] - 1, old.K, par.ctypes.data, par.shape[0],
                                         out.ctypes.data), "dg_layout_membership")
    return out[:par.shape[0]]


def carried_copies(old: S.BlockSplit, new: S.BlockSplit, src_of_new_global: np.ndarray,
                   original: np.ndarray) -> np.ndarray:
    """For every copy of the new layout, the copy of the old layout whose
    state it takes over (-1: none): the parent Gaussian's copy in the same
    block, when the new Gaussian is its parent itself.  The parent's copies
    are looked up through the old sharing map (dg_layout_carry, host C++)."""
    from . import _lib as L
    old_blk = np.ascontiguousarray(old.blk_off, np.int64)
    old_goff = np.ascontiguousarray(old.g_off, np.int64)
    old_gcp = np.ascontiguousarray(old.g_copies, np.int32)
    new_blk = np.ascontiguousarray(new.blk_off, np.int64)
    new_goff = np.ascontiguousarray(new.g_off, np.int64)
    new_gcp = np.ascontiguousarray(new.g_copies, np.int32)
    parent = np.ascontiguousarray(src_of_new_global, np.int32)
    orig = np.ascontiguousarray(original, np.uint8)
    if parent.shape[0] != new_goff.shape[0] - 1 or orig.shape[0] != parent.shape[0]:
        raise ValueError("one parent and one flag per new global")
    carry = np.empty(max(new.n_copies, 1), np.int32)
    L.check(L.lib().dg_layout_carry(old_blk.ctypes.data, old_goff.ctypes.data, old_gcp.ctypes.data,
                                    old_goff.shape[0] - 1, old.K, new_blk.ctypes.data, new_goff.ctypes.data,
                                    new_gcp.ctypes.data, parent.ctypes.data, orig.ctypes.data, parent.shape[0],
                                    carry.ctypes.data), "dg_layout_carry")
    return carry[:new.n_copies]


def densify(tr, cfg: DensifyConfig, extent: float, step_seed: int) -> Dict:
    """One densification of DogsTrainer `tr` (after a consensus).  Returns
    counts of the decisions and the sizes before and after."""
    dev = tr.z.data.device
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    z = tr.z
    codes, offsets = D.dg_densify_decide(z, tr.g_off, tr.g_copies, tr.dstats, cfg.grad_threshold,
                                         cfg.percent_dense, extent, cfg.min_opacity)
    n_out = int(offsets[-1].item()) & 0xFFFFFFFF
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(cfg.seed) * 1000003 + int(step_seed))
    normals = torch.randn(max(z.n, 1) * 6, device=dev, generator=gen, dtype=torch.float32)
    z_tmp, src, orig = D.dg_densify_emit(z, codes, offsets, normals, n_out)
    if cfg.layout == "inplace":
        c = D.dg_histogram_i32(codes, 0, 4)
        return _densify_inplace(tr, z, codes, offsets, z_tmp, n_out, c, t0)
    c = np.bincount(codes.cpu().numpy(), minlength=4)
    if cfg.layout != "resort":
        raise ValueError(f"unknown densification layout {cfg.layout!r}")
    src_h = src.cpu().numpy().astype(np.int64)
    orig_h = orig.cpu().numpy().astype(bool)
    t1 = time.perf_counter()
    # the new layout: every Gaussian in its parent's blocks
    old = tr.split
    member = parent_membership(old, src_h)
    xy = z_tmp.data[:4 * z_tmp.ld].view(z_tmp.ld, 4)[:n_out, :2].double().cpu().numpy()
    new_split, order = native_layout(xy, member, old.cells, old.band, K=old.K)
    t2 = time.perf_counter()
    order_t = torch.from_numpy(order.astype(np.int32)).to(dev)
    z_new = D.GaussianBuffer(n_out, z.deg, dev)
    D.dg_gather_rows(z_tmp, order_t, z_new)
    src_new = src_h[order]
    orig_new = orig_h[order]
    carry = torch.from_numpy(carried_copies(old, new_split, src_new, orig_new)).to(dev)
    gid_new = torch.from_numpy(new_split.copy_gid.astype(np.int32)).to(dev)
    n_c = new_split.n_copies
    x_new = D.GaussianBuffer(n_c, z.deg, dev)
    D.dg_gather_rows(z_new, gid_new, x_new)           # every copy from its Gaussian ...
    D.dg_gather_rows(tr.x, carry, x_new)              # ... the carried ones from their old copy
    bufs = {}
    for name in ("m", "v", "u"):
        b = D.GaussianBuffer(n_c, z.deg, dev)         # zeros where nothing is carried
        D.dg_gather_rows(getattr(tr, name), carry, b)
        bufs[name] = b
    del z_tmp
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    tr.install_split(new_split, z_new, x_new, bufs["m"], bufs["v"], bufs["u"])
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    return {"before": int(z.n), "after": int(n_out), "keep": int(c[D.L.DG_DENSIFY_KEEP]),
            "prune": int(c[D.L.DG_DENSIFY_PRUNE]), "clone": int(c[D.L.DG_DENSIFY_CLONE]),
            "split": int(c[D.L.DG_DENSIFY_SPLIT]), "copies": int(n_c),
            "carried_copies": int((carry >= 0).sum().item()),
            "seconds": {"decide_emit": round(t1 - t0, 3), "layout": round(t2 - t1, 3), "state": round(t3 - t2, 3),
                        "install": round(t4 - t3, 3)}}


def _densify_inplace(tr, z, codes, offsets, z_new, n_out: int, c, t0: float) -> Dict:
    """Steps 2-4 with the layout built on the device in the old order: z_new
    (the emitted set) is already in the new numbering."""
    dev = z.data.device
    old = tr.split
    torch.cuda.synchronize()
    t_de = time.perf_counter()
    new_g_off, new_g_cp, new_gid, carry, copy_off = D.dg_densify_layout(codes, offsets, tr.g_off, tr.g_copies,
                                                                        tr.gid)
    # the new block offsets: the copy offsets at the old block starts and shared ends (a few scalars)
    at = lambda i: int(copy_off[int(i)].item()) & 0xFFFFFFFF
    bo = np.array([at(b) for b in old.blk_off], np.int64)
    sh_end = np.array([at(old.blk_off[k] + old.blk_nshared[k]) for k in range(old.K)], np.int64)
    n_shared = int(offsets[int(old.n_shared_globals)].item()) & 0xFFFFFFFF
    new_split = S.BlockSplit(new_gid.cpu().numpy(), bo, sh_end - bo[:-1], new_g_off.cpu().numpy(),
                             new_g_cp.cpu().numpy(), n_shared, old.cells, old.band)
    t1 = time.perf_counter()
    n_c = new_split.n_copies
    x_new = D.GaussianBuffer(n_c, z.deg, dev)
    D.dg_gather_rows(z_new, new_gid, x_new)           # every copy from its Gaussian ...
    D.dg_gather_rows(tr.x, carry, x_new)              # ... the carried ones from their old copy
    bufs = {}
    for name in ("m", "v", "u"):
        b = D.GaussianBuffer(n_c, z.deg, dev)         # zeros where nothing is carried
        D.dg_gather_rows(getattr(tr, name), carry, b)
        bufs[name] = b
    carried = int(n_c - D.dg_histogram_i32(carry, -1, 1)[0])
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    tr.install_split(new_split, z_new, x_new, bufs["m"], bufs["v"], bufs["u"],
                     device_maps={"gid": new_gid, "g_off": new_g_off, "g_copies": new_g_cp})
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    return {"before": int(z.n), "after": int(n_out), "keep": int(c[D.L.DG_DENSIFY_KEEP]),
            "prune": int(c[D.L.DG_DENSIFY_PRUNE]), "clone": int(c[D.L.DG_DENSIFY_CLONE]),
            "split": int(c[D.L.DG_DENSIFY_SPLIT]), "copies": int(n_c), "carried_copies": carried,
            "layout": "inplace",
            "seconds": {"decide_emit": round(t_de - t0, 3), "layout": round(t1 - t_de, 3),
                        "state": round(t3 - t1, 3), "install": round(t4 - t3, 3)}}


def native_layout(xy: np.ndarray, member: np.ndarray, cells: np.ndarray, band: float, K: Optional[int] = None):
    """synth.split_layout's layout, computed by the library's host code
    (dg_layout, linear passes): (BlockSplit, order).  member: (n, K) bool,
    or uint64 bit masks with K given."""
    from . import _lib as L
    if member.dtype == np.uint64:
        bits, n = np.ascontiguousarray(member), member.shape[0]
    else:
        n, K = member.shape
        packed = np.packbits(member, axis=1, bitorder="little")
        pad = np.zeros((n, 8), np.uint8)
        pad[:, :packed.shape[1]] = packed
        bits = pad.view(np.uint64).reshape(n)
    xy = np.ascontiguousarray(xy[:, :2], np.float64)
    nc = int(L.lib().dg_layout_copies(bits.ctypes.data, n))
    if nc < 0:
        raise ValueError("bad membership")
    order = np.empty(max(n, 1), np.int32)
    copy_gid = np.empty(max(nc, 1), np.int32)
    blk_off = np.empty(K + 1, np.int64)
    blk_nsh = np.empty(K, np.int64)
    g_off = np.empty(n + 1, np.int64)
    g_cp = np.empty(max(nc, 1), np.int32)
    ns = np.zeros(1, np.int64)
    L.check(L.lib().dg_layout(xy.ctypes.data, bits.ctypes.data, n, K, order.ctypes.data, copy_gid.ctypes.data,
                              blk_off.ctypes.data, blk_nsh.ctypes.data, g_off.ctypes.data, g_cp.ctypes.data,
                              ns.ctypes.data), "dg_layout")
    split = S.BlockSplit(copy_gid[:nc], blk_off, blk_nsh, g_off, g_cp[:nc], int(ns[0]), cells, band)
    return split, order[:n].astype(np.int64)
