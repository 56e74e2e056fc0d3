"""Batched DOGS training on one GPU (Sec. 3.2, Alg. 2).

All K block-local models live in one set of device buffers; one iteration is
one launch per hot step over every block at once: dg_project, dg_bin_sort,
dg_rasterize_fwd, the Eq. 3 loss, dg_rasterize_bwd, the Adam + penalty
x-step (Eq. 8a / 12a) and, every `intv` iterations, the consensus
(Eq. 8b-c / 12b-c).  Iterations can be captured in CUDA graphs (one per pool
entry of views) and replayed.  SequentialTrainer is the plain per-block form:
K independent single-block models run one after another, the consensus
gathering their copies into one buffer and scattering the duals back.
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from . import dogs as D
from . import densify as DZ
from . import synth as S
from .admm import AdaptivePenalty

DEFAULT_LR = (1.6e-4, 1e-3, 5e-3, 2.5e-3, 1.25e-4, 5e-2)


def gather_copies(z: D.GaussianBuffer, gid: torch.Tensor, ld: Optional[int] = None) -> D.GaussianBuffer:
    """Copies x_c = z[gid[c]] in the library layout (setup-time data movement)."""
    n = gid.numel()
    out = D.GaussianBuffer(n, z.deg, z.data.device, ld)
    g = gid.long()
    for f in range(3):
        src = z.data[4 * f * z.ld:4 * (f + 1) * z.ld].view(z.ld, 4)
        out.data[4 * f * out.ld:4 * (f + 1) * out.ld].view(out.ld, 4)[:n] = src[g]
    P = 3 * D.sh_coefs(z.deg)
    src = z.data[12 * z.ld:].view(P, z.ld)
    out.data[12 * out.ld:].view(P, out.ld)[:, :n] = src[:, g]
    return out


class DogsTrainer:
    def __init__(self, split: S.BlockSplit, z0: D.GaussianBuffer, view_sets: Sequence[Sequence[S.Camera]],
                 targets: Sequence[torch.Tensor], rho=(1e-3,) * 5, lr=DEFAULT_LR, tile=(16, 16),
                 loss="dssim", w_l1=0.8, w_ssim=0.2, bg=(0.0, 0.0, 0.0), alpha=1.0, intv=100,
                 capacity: Optional[int] = None, device="cuda", adaptive: Optional[AdaptivePenalty] = None,
                 fused: bool = True, overlap: bool = True, densify: Optional["DZ.DensifyConfig"] = None,
                 deterministic: bool = False):
        self.device = device
        self.fused = fused
        # deterministic: the compositing adjoint sums each record's gradient
        # over its tiles in a fixed order (dg_rasterize_bwd_slots) instead of
        # by atomics, so a run repeats bit for bit (fused x-step, one view
        # per block)
        self.deterministic = deterministic
        # with the fused x-step: the groups of copies that no view sees are
        # stepped on a side stream right after the projection, alongside
        # binning, compositing and the loss (dg_xstep_part 1), the rest after
        # the compositing adjoint (part 2)
        self.overlap = overlap
        self.side = torch.cuda.Stream(device=device) if overlap and str(device).startswith("cuda") else None
        self._idle_queued = False
        # CTAs per SM of the side-stream part (a grid-stride loop), or 0 for
        # one CTA per group of copies.  Measured on the 6M-Gaussian step:
        # one per group 9.15 ms, 3 per SM 9.43, 2 per SM 10.03, 1 per SM
        # 11.93 (the compositing kernels leave few registers free, so a
        # small grid only drags the step), the one-part x-step 9.24
        self.idle_ctas_per_sm = 0
        # how that part runs: "stream" -- dg_xstep_stream, one persistent CTA
        # per SM (idle_ctas_per_sm: 0 = one) moving the groups through shared
        # memory, launched with the compositing adjoint, beside which it fits;
        # "stream_early" -- the same right after the projection; "grid" --
        # dg_xstep_part 1 right after the projection
        self.idle_mode = "stream"
        # the fused part 2 over the list of groups with a kept record that
        # the side stream builds first (dg_xstep_groups, dg_xstep_listed), so
        # that the CTAs past it, which find nothing to step, come after those
        # that step; False: one CTA per group, each finding out for itself
        # (dg_xstep_part 2)
        self.listed_part2 = True
        self._lists_ready = None
        self.n_sm = torch.cuda.get_device_properties(device).multi_processor_count if self.side is not None else 0
        self.adaptive = adaptive
        if adaptive is not None:
            adaptive.rho = [float(r) for r in rho]
        self.rho, self.lr, self.bg, self.alpha, self.intv = list(rho), list(lr), bg, alpha, intv
        # with the adaptive penalty, rho lives on the device: Eq. 10 runs there
        # right after each consensus (dg_admm_adapt, dg_admm_rescale) inside
        # the captured graph, and the kernels read rho when they run
        self.rho_dev = self.factor_dev = None
        if adaptive is not None:
            self.rho_dev = torch.tensor([float(r) for r in rho], dtype=torch.float32, device=device)
            self.factor_dev = torch.ones(5, dtype=torch.float32, device=device)
        self.adapt_on_device = adaptive is not None
        self.loss_kind, self.w_l1, self.w_ssim = loss, w_l1, w_ssim
        self.view_sets = [list(v) for v in view_sets]
        self.tile = tuple(tile)
        # densification under consensus (densify.DensifyConfig), statistics per copy
        self.densify_cfg = densify
        if densify is not None and (densify.interval % intv != 0 or densify.opacity_reset % intv != 0):
            raise ValueError("the densification and opacity-reset intervals must be multiples of the "
                             "consensus interval")
        self.extent = None
        if densify is not None:
            self.extent = densify.extent if densify.extent is not None else \
                DZ.scene_extent([c for vs in self.view_sets for c in vs])
        self.densify_log: List[Dict] = []
        # the layout the run starts from: a checkpoint of a later (densified)
        # layout of the same run can be resumed on a trainer built on it
        from .checkpoint import split_fingerprint
        self.split_origin = split_fingerprint(split)
        gid = torch.from_numpy(split.copy_gid.astype(np.int32)).to(device)
        x = gather_copies(z0, gid)
        self.install_split(split, z0, x, x.like(), x.like(), x.like(), capacity=capacity)
        self.targets = list(targets)
        # Adam's step counter lives on the device and each iteration advances
        # it there, so replays queued back to back each see their own count
        self.dev_step = torch.zeros(1, dtype=torch.int32, device=device)
        self.residuals = torch.zeros(10, dtype=torch.float64, device=device)
        self.t = 0
        self.graphs = {}
        self.host_targets = None

    # ---- the block layout and the state on it --------------------------------------
    def install_split(self, split: S.BlockSplit, z: D.GaussianBuffer, x: D.GaussianBuffer, m: D.GaussianBuffer,
                      v: D.GaussianBuffer, u: D.GaussianBuffer, capacity: Optional[int] = None,
                      calibrate: bool = True, device_maps: Optional[Dict[str, torch.Tensor]] = None) -> None:
        """Take a block layout with its global model, copies, Adam moments and
        scaled duals: the sharing map, the anchors z - u, the batch plan for
        the view sets and (after a first install, unless the caller fills the
        buffers afterwards and calibrates then) the instance capacity are
        rebuilt; captured graphs are dropped."""
        dev = self.device
        first = not hasattr(self, "split")
        variant = None if first else (self.vb.plan.raster_warps, self.vb.plan.raster_stage,
                                      self.vb.plan.raster_warps_bwd, self.vb.plan.raster_stage_bwd)
        self.split = split
        # globals held by several blocks numbered first: then, in an iteration
        # with a consensus, the x-step stores the unshared copies' values into
        # z itself and the consensus runs over the shared globals alone
        cnt = np.diff(split.g_off)
        ns = int(split.n_shared_globals)
        self._shared_first = bool((cnt[:ns] > 1).all() and (cnt[ns:] <= 1).all())
        self.n_shared_globals = ns
        if device_maps is not None:
            # the layout's arrays already on the device (as the split holds them): no upload
            self.gid, self.g_off, self.g_copies = device_maps["gid"], device_maps["g_off"], device_maps["g_copies"]
            self.shared = torch.zeros(split.n_copies, dtype=torch.uint8, device=dev)
            for k in range(split.K):
                b = int(split.blk_off[k])
                self.shared[b:b + int(split.blk_nshared[k])] = 1
        else:
            self.gid = torch.from_numpy(split.copy_gid.astype(np.int32)).to(dev)
            self.shared = torch.from_numpy(split.copy_shared()).to(dev)
            self.g_off = torch.from_numpy(split.g_off.astype(np.int64)).to(dev)
            self.g_copies = torch.from_numpy(split.g_copies.astype(np.int32)).to(dev)
        self.z, self.x, self.m, self.v, self.u = z, x, m, v, u
        self.grad, self.anchor = x.like(), x.like()
        self.xs_ws = D.xstep_stream_workspace(x) if self.side is not None else None
        D.dg_admm_anchor(self.z, self.u, self.gid, self.shared, self.anchor)
        self.dstats = (torch.zeros(2 * max(split.n_copies, 1), dtype=torch.float32, device=dev)
                       if self.densify_cfg is not None else None)
        self.vb = None
        if not first:
            torch.cuda.empty_cache()
        self.vb = D.ViewBatch(self.view_sets[0], split.blk_off, self.tile[0], self.tile[1], device=dev,
                              capacity=capacity, loss_ws=(self.loss_kind == "dssim"))
        if variant is not None:
            D.apply_variant(self.vb.plan, variant)
        self.cam_pool = [D.cams_to_device(D.plan_views(vs, split.blk_off, *self.tile)[0], dev)
                         for vs in self.view_sets]
        self.graphs = {}
        self._idle_queued, self._lists_ready = False, None
        if not first and calibrate:
            self.calibrate_capacity()

    # ---- rasteriser configuration (autotuner) ------------------------------------
    def set_tile(self, tile) -> None:
        """Re-plan the batch for another tile shape (new buffers, capacity
        recalibrated); captured graphs are dropped."""
        tile = tuple(tile)
        if tile == self.tile:
            return
        self.vb = None
        torch.cuda.empty_cache()
        self.tile = tile
        self.vb = D.ViewBatch(self.view_sets[0], self.split.blk_off, tile[0], tile[1], device=self.device,
                              loss_ws=(self.loss_kind == "dssim"))
        self.cam_pool = [D.cams_to_device(D.plan_views(vs, self.split.blk_off, *tile)[0], self.device)
                         for vs in self.view_sets]
        self.graphs.clear()
        self.calibrate_capacity()

    def set_variant(self, warps: int, stage: int, warps_bwd: int = 0, stage_bwd: int = 0) -> None:
        D.apply_variant(self.vb.plan, (warps, stage, warps_bwd, stage_bwd))
        self.graphs.clear()

    # ---- capacity -------------------------------------------------------------
    def calibrate_capacity(self, headroom=1.3) -> int:
        """Instance count of every pool entry (one synchronising pass each),
        then a capacity with headroom; buffers are re-allocated once."""
        mx = 0
        for p in range(len(self.view_sets)):
            self.vb.dev_cams.copy_(self.cam_pool[p])
            D.dg_project(self.x, self.vb)
            self.vb.status.zero_()
            D.dg_bin_sort(self.vb)
            torch.cuda.synchronize()
            mx = max(mx, int(self.vb.count.item()) & 0xFFFFFFFF)
        cap = int(mx * headroom) + 4096
        self.vb.set_capacity(cap)
        if self.deterministic:
            slots = 0
            for p in range(len(self.view_sets)):
                self.vb.dev_cams.copy_(self.cam_pool[p])
                D.dg_project(self.x, self.vb)
                r = self.vb.rect[:2 * self.vb.n_rec].cpu().numpy().view(np.uint32).reshape(-1, 2)
                w = (r[:, 1] & 0xFFFF).astype(np.int64) - (r[:, 0] & 0xFFFF)
                h = (r[:, 1] >> 16).astype(np.int64) - (r[:, 0] >> 16)
                slots = max(slots, int(np.where((w > 0) & (h > 0), w * h, 0).sum()))
            self.vb.enable_slots(int(slots * headroom) + 4096)
        self.graphs.clear()
        return mx

    # ---- one iteration ----------------------------------------------------------
    def _loss(self, target):
        if self.loss_kind == "dssim":
            D.dg_loss_dssim(self.vb, target, self.w_l1, self.w_ssim)
        else:
            D.dg_loss_l1(self.vb, target, self.w_l1)

    def enqueue(self, p: int, consensus: bool, target: Optional[torch.Tensor] = None,
                slot: Optional[int] = None) -> None:
        """All launches of one iteration for pool entry p on the current stream.
        The step counter for Adam's bias correction (dev_step) is advanced
        on the device first."""
        vb = self.vb
        vb.dev_cams.copy_(self.cam_pool[p], non_blocking=True)
        D.dg_step_advance(self.dev_step)
        D.dg_project(self.x, vb)
        zf = self._zfuse(consensus)
        if self._split_xstep() and self.idle_mode in ("grid", "stream_early"):
            self.idle_xstep(zf)
        D.dg_bin_sort(vb)
        D.dg_rasterize_fwd(vb, self.bg)
        self._loss(self.targets[p] if target is None else target)
        self.backward_step(zf)
        if self._stats_on():
            D.dg_densify_stats(vb, self.dstats)
        if consensus:
            D.dg_admm_consensus(self.x, self.u, self.z_shared() if zf else self.z, self.anchor, self.g_off,
                                self.g_copies, self.rho_arg(), self.alpha, self.residuals)
            if self.adaptive is not None and self.adapt_on_device:
                ad = self.adaptive
                D.dg_admm_adapt(self.residuals, self.rho_dev, self.factor_dev, self.dev_step, ad.mu, ad.tau_inc,
                                ad.tau_dec, ad.freeze_after)
                D.dg_admm_rescale(self.u, self.z, self.anchor, self.gid, self.shared, self.factor_dev)
        if self.host_targets is not None:
            self.host_loss[0 if slot is None else slot].copy_(vb.loss, non_blocking=True)

    # ---- targets in host memory ----------------------------------------------------
    def use_host_targets(self, host_targets: Sequence[torch.Tensor]) -> None:
        """Keep the pool's target images in pinned host memory (float32, or
        uint8 as training images come: then 1/4 of the bytes cross the link
        and a kernel widens them on the device).  Each step's target is
        copied in on a side stream one step ahead, into one of two device
        buffers, while the previous step computes; every step also
        copies its per-view losses back into one of two pinned host buffers
        (read them with loss_of(t) or last_loss(), which wait only for that
        step, so the host can read step t's losses while step t + 1 runs)."""
        self.host_targets = [t if t.is_pinned() else t.pin_memory() for t in host_targets]
        # 8-bit targets cross the link as bytes and widen to float on the copy stream
        self.stage_u8 = None
        if self.host_targets[0].dtype == torch.uint8:
            self.stage_u8 = [torch.empty(self.host_targets[0].shape, dtype=torch.uint8, device=self.device)
                             for _ in range(2)]
        self.stage = [torch.empty(self.host_targets[0].shape, dtype=torch.float32, device=self.device)
                      for _ in range(2)]
        self.host_loss = [torch.zeros(self.vb.loss.numel(), dtype=torch.float64).pin_memory() for _ in range(2)]
        self.loss_ready = [torch.cuda.Event() for _ in range(2)]
        self.loss_step = [-1, -1]
        self.copy_stream = torch.cuda.Stream()
        self.copied = [torch.cuda.Event() for _ in range(2)]
        self.used = [torch.cuda.Event() for _ in range(2)]
        self.slot_entry = [None, None]
        self.graphs.clear()
        self._prefetch(self.t % len(self.view_sets), self.t % 2)

    def _prefetch(self, p: int, slot: int) -> None:
        self.copy_stream.wait_event(self.used[slot])           # the step that last read this buffer
        with torch.cuda.stream(self.copy_stream):
            if self.stage_u8 is not None:
                self.stage_u8[slot].copy_(self.host_targets[p], non_blocking=True)
                D.dg_image_u8_to_f32(self.stage_u8[slot], self.stage[slot])
            else:
                self.stage[slot].copy_(self.host_targets[p], non_blocking=True)
        self.copied[slot].record(self.copy_stream)
        self.slot_entry[slot] = p

    def h2d_bytes_per_step(self) -> int:
        t = self.host_targets[0]
        return int(t.numel() * t.element_size())

    def loss_of(self, t: int) -> torch.Tensor:
        """The per-view losses of iteration t, one of the last two (waits for
        that iteration only)."""
        slot = t % 2
        if self.loss_step[slot] != t:
            raise ValueError(f"losses of iteration {t} are no longer (or not yet) on the host")
        self.loss_ready[slot].synchronize()
        return self.host_loss[slot].clone()

    def last_loss(self) -> torch.Tensor:
        """The per-view losses of the last step (waits for it)."""
        return self.loss_of(self.t - 1)

    def _split_xstep(self) -> bool:
        return self.side is not None and self.fused and D.one_view_per_block(self.vb.plan)

    def _zfuse(self, consensus: bool) -> bool:
        return bool(consensus) and self.fused and self._shared_first and D.one_view_per_block(self.vb.plan)

    def _zargs(self, zfuse: bool) -> dict:
        return dict(z_unshared=self.z, gid=self.gid) if zfuse else {}

    def z_shared(self) -> D.GaussianBuffer:
        """z restricted to the shared globals (a view of the same memory)."""
        return D.GaussianBuffer(self.n_shared_globals, self.z.deg, self.z.data.device, self.z.ld, self.z.data)

    def idle_xstep(self, zfuse: bool = False) -> None:
        """Part 1 of the split x-step (the groups of copies without a kept
        record) on the side stream, after the work queued so far on the
        current stream (the projection for "grid", everything up to the
        loss for "stream")."""
        cur = torch.cuda.current_stream()
        self.side.wait_stream(cur)
        with torch.cuda.stream(self.side):
            if self.idle_mode.startswith("stream") and self.listed_part2:
                D.dg_xstep_groups(self.vb, self.x, self.xs_ws)
                self._lists_ready = torch.cuda.Event()
                self._lists_ready.record(self.side)
                D.dg_xstep_listed(1, self.vb, self.x, self.m, self.v, self.anchor, self.shared, self.rho_arg(),
                                  self.lr, self.xs_ws, step=1, dev_step=self.dev_step,
                                  ctas=self.n_sm * self.idle_ctas_per_sm, **self._zargs(zfuse))
            elif self.idle_mode.startswith("stream"):
                D.dg_xstep_stream(self.vb, self.x, self.m, self.v, self.anchor, self.shared, self.rho_arg(), self.lr,
                                  self.xs_ws, step=1, dev_step=self.dev_step, ctas=self.n_sm * self.idle_ctas_per_sm,
                                  **self._zargs(zfuse))
            else:
                if self.listed_part2:
                    D.dg_xstep_groups(self.vb, self.x, self.xs_ws)
                    self._lists_ready = torch.cuda.Event()
                    self._lists_ready.record(self.side)
                D.dg_xstep_part(1, self.vb, self.x, self.m, self.v, self.anchor, self.shared, self.rho_arg(),
                                self.lr, step=1, dev_step=self.dev_step, ctas=self.n_sm * self.idle_ctas_per_sm,
                                **self._zargs(zfuse))
        self._idle_queued = True

    def backward_step(self, zfuse: bool = False) -> None:
        """Adjoint of the iteration's render and the x-step (Eq. 8a / 12a).
        With at most one view per block the projection adjoint and the step
        run fused (the gradient stays in registers); otherwise through the
        gradient buffer.  With the split x-step, its second part here and the
        side stream joined back.  zfuse: the x-step also stores the unshared
        copies into z (an iteration whose consensus then covers the shared
        globals only)."""
        vb = self.vb
        bwd_records = D.dg_rasterize_bwd_slots if self.deterministic else D.dg_rasterize_bwd_records
        if self.deterministic and not (self.fused and D.one_view_per_block(vb.plan)):
            raise ValueError("the deterministic backward runs with the fused x-step (one view per block)")
        if self.deterministic and getattr(vb, "part", None) is None:
            raise RuntimeError("deterministic mode: call calibrate_capacity() first (it sizes the slots)")
        if self._split_xstep() and self.idle_mode == "stream":
            self.idle_xstep(zfuse)                 # beside the compositing adjoint
        if self._split_xstep() and self._idle_queued:
            bwd_records(vb, bg=self.bg)
            if self._lists_ready is not None:      # the lists built on the side stream
                torch.cuda.current_stream().wait_event(self._lists_ready)
                D.dg_xstep_listed(2, vb, self.x, self.m, self.v, self.anchor, self.shared, self.rho_arg(), self.lr,
                                  self.xs_ws, step=1, dev_step=self.dev_step, **self._zargs(zfuse))
                self._lists_ready = None
            else:
                D.dg_xstep_part(2, vb, self.x, self.m, self.v, self.anchor, self.shared, self.rho_arg(), self.lr,
                                step=1, dev_step=self.dev_step, **self._zargs(zfuse))
            torch.cuda.current_stream().wait_stream(self.side)
            self._idle_queued = False
        elif self.fused and D.one_view_per_block(vb.plan):
            bwd_records(vb, bg=self.bg)
            D.dg_xstep_part(0, vb, self.x, self.m, self.v, self.anchor, self.shared, self.rho_arg(), self.lr,
                            step=1, dev_step=self.dev_step, **self._zargs(zfuse))
        else:
            D.dg_rasterize_bwd(vb, self.x, self.grad, bg=self.bg)
            D.dg_adam_admm_step(self.x, self.grad, self.m, self.v, self.anchor, self.shared, self.rho_arg(), self.lr,
                                step=1, dev_step=self.dev_step)

    def step(self, consensus: Optional[bool] = None, graph=True) -> None:
        """Iteration t (0-based) of Alg. 2: local steps, then the consensus
        when t mod intv == 0 (or as forced by `consensus`)."""
        p = self.t % len(self.view_sets)
        c = (self.t % self.intv == 0) if consensus is None else consensus
        slot, target = None, None
        if self.host_targets is not None:
            slot = self.t % 2
            if self.slot_entry[slot] != p:
                self._prefetch(p, slot)
            torch.cuda.current_stream().wait_event(self.copied[slot])
            target = self.stage[slot]
        ds = self._stats_on()
        if graph:
            key = (p, c, slot, ds)
            if key not in self.graphs:
                self.graphs[key] = self._capture(p, c, target, slot)
            self.graphs[key].replay()
        else:
            self.enqueue(p, c, target, slot)
        if slot is not None:
            self.used[slot].record(torch.cuda.current_stream())
            self.loss_ready[slot].record(torch.cuda.current_stream())
            self.loss_step[slot] = self.t
            nxt = self.t + 1
            self._prefetch(nxt % len(self.view_sets), nxt % 2)
        if c and self.adaptive is not None and not self.adapt_on_device and self.t < self.adaptive.freeze_after:
            self._adapt_penalty()
        if c and self.densify_cfg is not None and self.densify_cfg.due(self.t):
            self.densify_log.append(dict(DZ.densify(self, self.densify_cfg, self.extent, self.t), t=self.t))
        if c and self.densify_cfg is not None and self.densify_cfg.reset_due(self.t):
            DZ.reset_opacity(self, self.densify_cfg)
        self.t += 1

    def _stats_on(self) -> bool:
        """Whether this iteration adds to the densification statistic."""
        return self.densify_cfg is not None and self.t < self.densify_cfg.until

    def rho_arg(self):
        """rho as the kernels take it: the device array under the adaptive
        penalty (updated there by Eq. 10), else the host list."""
        return self.rho_dev if self.rho_dev is not None else self.rho

    def current_rho(self) -> List[float]:
        """The penalties in effect (read back from the device under the
        adaptive penalty; one synchronisation), also kept in self.rho and the
        AdaptivePenalty state."""
        if self.rho_dev is not None:
            self.rho = [float(r) for r in self.rho_dev.cpu().tolist()]
            if self.adaptive is not None:
                self.adaptive.rho = list(self.rho)
        return list(self.rho)

    def _adapt_penalty(self) -> None:
        """The host form of Eq. 10 (with adapt_on_device off): read the residuals (one synchronisation),
        update rho, rescale the scaled duals of the shared copies and rebuild
        the anchors z - u.  rho is a launch argument, so captured graphs are
        dropped when it changes (at most freeze_after / intv times)."""
        res = self.residuals.cpu().tolist()
        rho, factor = self.adaptive.update(res, self.t)
        if all(f == 1.0 for f in factor):
            return
        D.dg_admm_scale_duals(self.u, self.shared, factor)
        D.dg_admm_anchor(self.z, self.u, self.gid, self.shared, self.anchor)
        self.rho = rho
        if self.rho_dev is not None:
            self.rho_dev.copy_(torch.tensor(rho, dtype=torch.float32))
        self.graphs.clear()

    def _capture(self, p: int, c: bool, target: Optional[torch.Tensor] = None,
                 slot: Optional[int] = None) -> torch.cuda.CUDAGraph:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):       # warm the allocator-free launch path once
            torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.enqueue(p, c, target, slot)
        return g

    def prepare_graphs(self, consensus_values=(True,)) -> int:
        """Capture, ahead of time, the graph of every (pool entry, consensus
        or not, target slot) combination that later steps can replay, so no
        capture falls inside a timed loop.  Returns the number captured."""
        slots = [None] if self.host_targets is None else [0, 1]
        ds = self._stats_on()
        n = 0
        for p in range(len(self.view_sets)):
            for c in consensus_values:
                for slot in slots:
                    key = (p, bool(c), slot, ds)
                    if key not in self.graphs:
                        target = None if slot is None else self.stage[slot]
                        self.graphs[key] = self._capture(p, bool(c), target, slot)
                        n += 1
        return n

    def overflowed(self) -> bool:
        return bool(int(self.vb.status.item()) & L.DG_STATUS_CAPACITY)

    # ---- checkpoint / resume ------------------------------------------------------
    def refresh_anchor(self) -> None:
        """Anchors z - u of the shared copies from the current z and u (and
        the device step counter from t, after t was set from outside)."""
        D.dg_admm_anchor(self.z, self.u, self.gid, self.shared, self.anchor)
        self.dev_step.fill_(self.t)
        if self.rho_dev is not None:
            self.rho_dev.copy_(torch.tensor([float(r) for r in self.rho], dtype=torch.float32))
        torch.cuda.synchronize()

    def save_checkpoint(self, path: str) -> None:
        from . import checkpoint
        checkpoint.save(self, path)

    def load_checkpoint(self, path: str) -> dict:
        from . import checkpoint
        return checkpoint.load(self, path)


class SequentialTrainer:
    """The plain sequential per-block form: K single-block models, each with
    its own buffers and view batch, stepped one after another without graphs.
    The consensus gathers every block's copies into one buffer (what the
    paper's master receives), runs dg_admm_consensus and sends the duals and
    anchors back."""

    def __init__(self, split: S.BlockSplit, z0: D.GaussianBuffer, view_sets, targets, rho=(1e-3,) * 5,
                 lr=DEFAULT_LR, tile=(16, 16), loss="dssim", w_l1=0.8, w_ssim=0.2, bg=(0.0, 0.0, 0.0), alpha=1.0,
                 intv=100, capacity: Optional[int] = None, device="cuda"):
        self.split, self.device, self.K = split, device, split.K
        self.rho, self.lr, self.bg, self.alpha, self.intv = list(rho), list(lr), bg, alpha, intv
        self.loss_kind, self.w_l1, self.w_ssim = loss, w_l1, w_ssim
        self.z = z0
        self.gid = torch.from_numpy(split.copy_gid.astype(np.int32)).to(device)
        self.shared_all = torch.from_numpy(split.copy_shared()).to(device)
        self.g_off = torch.from_numpy(split.g_off.astype(np.int64)).to(device)
        self.g_copies = torch.from_numpy(split.g_copies.astype(np.int32)).to(device)
        self.blocks = []
        per = len(view_sets[0]) // self.K
        for k in range(self.K):
            b, e = int(split.blk_off[k]), int(split.blk_off[k + 1])
            gid = self.gid[b:e]
            x = gather_copies(z0, gid)
            blk = dict(b=b, e=e, x=x, grad=x.like(), m=x.like(), v=x.like(), u=x.like(), anchor=x.like(),
                       shared=self.shared_all[b:e].contiguous(), gid=gid.contiguous())
            D.dg_admm_anchor(z0, blk["u"], blk["gid"], blk["shared"], blk["anchor"])
            vsets = []
            for vs in view_sets:
                cams = []
                for c in vs[k * per:(k + 1) * per]:
                    cc = S.Camera(**{**c.__dict__, "block": 0})
                    cams.append(cc)
                vsets.append(cams)
            blk["vb"] = D.ViewBatch(vsets[0], [0, e - b], tile[0], tile[1], device=device, capacity=capacity,
                                    loss_ws=(loss == "dssim"))
            blk["cam_pool"] = [D.cams_to_device(D.plan_views(vs, [0, e - b], *tile)[0], device) for vs in vsets]
            blk["targets"] = []
            for t in targets:
                # the block's views are a contiguous slice of the batched image layout
                vb_all_pix = 3 * per * vsets[0][0].width * vsets[0][0].height
                blk["targets"].append(t[k * vb_all_pix:(k + 1) * vb_all_pix])
            self.blocks.append(blk)
        # gather buffers for the consensus (the master's copy of every block)
        n = split.n_copies
        self.x_all = D.GaussianBuffer(n, z0.deg, device)
        self.u_all, self.a_all = self.x_all.like(), self.x_all.like()
        self.t = 0
        self.residuals = torch.zeros(10, dtype=torch.float64, device=device)

    def calibrate_capacity(self, headroom=1.3):
        for blk in self.blocks:
            vb = blk["vb"]
            mx = 0
            for cp in blk["cam_pool"]:
                vb.dev_cams.copy_(cp)
                D.dg_project(blk["x"], vb)
                vb.status.zero_()
                D.dg_bin_sort(vb)
                torch.cuda.synchronize()
                mx = max(mx, int(vb.count.item()) & 0xFFFFFFFF)
            vb.set_capacity(int(mx * headroom) + 4096)

    def _copy_rows(self, dst: D.GaussianBuffer, src: D.GaussianBuffer, b: int, e: int, to_all: bool):
        for f in range(3):
            A = dst.data[4 * f * dst.ld:4 * (f + 1) * dst.ld].view(dst.ld, 4)
            B = src.data[4 * f * src.ld:4 * (f + 1) * src.ld].view(src.ld, 4)
            if to_all:
                A[b:e] = B[:e - b]
            else:
                A[:e - b] = B[b:e]
        P = 3 * D.sh_coefs(dst.deg)
        A = dst.data[12 * dst.ld:].view(P, dst.ld)
        B = src.data[12 * src.ld:].view(P, src.ld)
        if to_all:
            A[:, b:e] = B[:, :e - b]
        else:
            A[:, :e - b] = B[:, b:e]

    def step(self, consensus: Optional[bool] = None) -> None:
        p = self.t % len(self.blocks[0]["cam_pool"])
        c = (self.t % self.intv == 0) if consensus is None else consensus
        for blk in self.blocks:
            vb = blk["vb"]
            vb.dev_cams.copy_(blk["cam_pool"][p], non_blocking=True)
            D.dg_project(blk["x"], vb)
            D.dg_bin_sort(vb)
            D.dg_rasterize_fwd(vb, self.bg)
            if self.loss_kind == "dssim":
                D.dg_loss_dssim(vb, blk["targets"][p], self.w_l1, self.w_ssim)
            else:
                D.dg_loss_l1(vb, blk["targets"][p], self.w_l1)
            if D.one_view_per_block(vb.plan):      # the same fused adjoint + x-step as the batched form
                D.dg_rasterize_bwd_records(vb, bg=self.bg)
                D.dg_xstep_from_records(vb, blk["x"], blk["m"], blk["v"], blk["anchor"], blk["shared"], self.rho,
                                        self.lr, step=self.t + 1)
            else:
                D.dg_rasterize_bwd(vb, blk["x"], blk["grad"], bg=self.bg)
                D.dg_adam_admm_step(blk["x"], blk["grad"], blk["m"], blk["v"], blk["anchor"], blk["shared"],
                                    self.rho, self.lr, step=self.t + 1)
        if c:
            for blk in self.blocks:
                self._copy_rows(self.x_all, blk["x"], blk["b"], blk["e"], True)
                self._copy_rows(self.u_all, blk["u"], blk["b"], blk["e"], True)
            D.dg_admm_consensus(self.x_all, self.u_all, self.z, self.a_all, self.g_off, self.g_copies, self.rho,
                                self.alpha, self.residuals)
            for blk in self.blocks:
                self._copy_rows(blk["u"], self.u_all, blk["b"], blk["e"], False)
                self._copy_rows(blk["anchor"], self.a_all, blk["b"], blk["e"], False)
        self.t += 1
