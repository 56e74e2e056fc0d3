"""Python face of libdogs: device buffers in the library's layout, batches of
views, thin wrappers with the C ABI's names, and the autograd boundary.

Layout conversion (numpy -> the structure-of-arrays parameter buffer) and
buffer allocation happen here; every step of the method runs in libdogs.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from . import synth as S


def _round_up(x: int, m: int) -> int:
    return (x + m - 1) // m * m


def sh_coefs(deg: int) -> int:
    return (deg + 1) ** 2


# ---------------------------------------------------------------------------
# parameter sets
# ---------------------------------------------------------------------------
class GaussianBuffer:
    """n Gaussians of SH degree `deg` in one float32 device tensor laid out as
    dg_gaussians: float4 (mean, opacity logit), float4 quaternion, float4
    (log-scale, 0), then 3 (deg+1)^2 SH planes of ld floats."""

    def __init__(self, n: int, deg: int, device="cuda", ld: Optional[int] = None,
                 data: Optional[torch.Tensor] = None):
        self.n, self.deg = int(n), int(deg)
        self.ld = int(ld) if ld is not None else _round_up(max(self.n, 1), 32)
        self.floats = (12 + 3 * sh_coefs(self.deg)) * self.ld
        if data is None:
            data = torch.zeros(self.floats, dtype=torch.float32, device=device)
        assert data.numel() == self.floats and data.dtype == torch.float32
        self.data = data
        self.struct = L.DgGaussians(data.data_ptr(), self.n, self.ld, self.deg, 0)

    @property
    def ref(self):
        return C.byref(self.struct)

    def like(self) -> "GaussianBuffer":
        return GaussianBuffer(self.n, self.deg, self.data.device, self.ld)

    def clone(self) -> "GaussianBuffer":
        return GaussianBuffer(self.n, self.deg, self.data.device, self.ld, self.data.clone())

    def copy_(self, other: "GaussianBuffer") -> "GaussianBuffer":
        self.data.copy_(other.data)
        return self

    # host-side packing -------------------------------------------------------
    @staticmethod
    def pack(g: S.Gaussians, ld: Optional[int] = None) -> np.ndarray:
        n, K = g.n, g.sh.shape[1]
        ld = ld if ld is not None else _round_up(max(n, 1), 32)
        a = np.zeros((12 + 3 * K) * ld, np.float32)
        mo = a[0:4 * ld].reshape(ld, 4)
        mo[:n, :3] = g.means
        mo[:n, 3] = g.opacity_logits
        a[4 * ld:8 * ld].reshape(ld, 4)[:n] = g.quats
        a[8 * ld:12 * ld].reshape(ld, 4)[:n, :3] = g.log_scales
        a[12 * ld:].reshape(3 * K, ld)[:, :n] = g.sh.reshape(n, 3 * K).T
        return a

    @staticmethod
    def unpack(a: np.ndarray, n: int, deg: int, ld: int) -> S.Gaussians:
        K = sh_coefs(deg)
        a = np.asarray(a, np.float32)
        mo = a[0:4 * ld].reshape(ld, 4)[:n]
        q = a[4 * ld:8 * ld].reshape(ld, 4)[:n]
        s = a[8 * ld:12 * ld].reshape(ld, 4)[:n, :3]
        sh = a[12 * ld:].reshape(3 * K, ld)[:, :n].T.reshape(n, K, 3)
        return S.Gaussians(mo[:, :3].copy(), q.copy(), s.copy(), mo[:, 3].copy(), sh.copy())

    @classmethod
    def from_synth(cls, g: S.Gaussians, device="cuda", ld: Optional[int] = None) -> "GaussianBuffer":
        a = cls.pack(g, ld)
        b = cls(g.n, g.sh_degree, device, ld if ld is not None else _round_up(max(g.n, 1), 32),
                torch.from_numpy(a).to(device))
        return b

    def to_synth(self) -> S.Gaussians:
        return self.unpack(self.data.detach().cpu().numpy(), self.n, self.deg, self.ld)

    def pad_lane(self) -> torch.Tensor:
        return self.data[8 * self.ld:12 * self.ld].view(self.ld, 4)[:, 3]


# ---------------------------------------------------------------------------
# cameras, plans and per-batch buffers
# ---------------------------------------------------------------------------
def camera_array(cams: Sequence[S.Camera]):
    arr = (L.DgCamera * len(cams))()
    for i, c in enumerate(cams):
        d = arr[i]
        d.width, d.height = int(c.width), int(c.height)
        d.fx, d.fy, d.cx, d.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        R = np.asarray(c.R, np.float32).reshape(9)
        t = np.asarray(c.t, np.float32).reshape(3)
        p = np.asarray(c.campos, np.float32).reshape(3)
        for k in range(9):
            d.R[k] = float(R[k])
        for k in range(3):
            d.t[k] = float(t[k])
            d.campos[k] = float(p[k])
        d.near_z = float(c.near)
        d.block = int(getattr(c, "block", 0))
    return arr


# compositing variant (warps per tile, instances staged per thread) of the
# forward and of the backward (0, 0 = the forward's) applied to new plans;
# the autotuner sets it from measurements
RASTER_VARIANT = [4, 2, 0, 0]


def set_raster_variant(warps: int, stage: int, warps_bwd: int = 0, stage_bwd: int = 0) -> None:
    RASTER_VARIANT[:] = [int(warps), int(stage), int(warps_bwd), int(stage_bwd)]


def apply_variant(plan, variant) -> None:
    plan.raster_warps, plan.raster_stage, plan.raster_warps_bwd, plan.raster_stage_bwd = [int(v) for v in variant]


def plan_views(cams: Sequence[S.Camera], blk_off: Sequence[int], tile_w=16, tile_h=16):
    arr = camera_array(cams)
    off = (C.c_int64 * len(blk_off))(*[int(v) for v in blk_off])
    plan = L.DgPlan()
    L.check(L.lib().dg_plan_views(arr, len(cams), off, len(blk_off) - 1, tile_w, tile_h, C.byref(plan)),
            "dg_plan_views")
    apply_variant(plan, RASTER_VARIANT)
    return arr, plan


def render_plan(cams: Sequence[S.Camera], n_gauss: int, tile_w=16, tile_h=16):
    arr = camera_array(cams)
    plan = L.DgPlan()
    L.check(L.lib().dg_render_plan(arr, len(cams), int(n_gauss), tile_w, tile_h, C.byref(plan)), "dg_render_plan")
    apply_variant(plan, RASTER_VARIANT)
    return arr, plan


def cams_to_device(arr, device="cuda") -> torch.Tensor:
    raw = np.frombuffer(bytes(arr), dtype=np.uint8).copy()
    return torch.from_numpy(raw).to(device)


class ViewBatch:
    """A planned batch of views over block-local copies, with the device
    buffers the rasteriser needs (records, tile rectangles, sorted instances,
    ranges, images, saved forward state)."""

    def __init__(self, cams: Sequence[S.Camera], blk_off: Sequence[int], tile_w=16, tile_h=16,
                 device="cuda", capacity: Optional[int] = None, keep_keys=False, loss_ws=False):
        self.cams = list(cams)
        self.blk_off = [int(v) for v in blk_off]
        self.device = device
        self.host_cams, self.plan = plan_views(self.cams, self.blk_off, tile_w, tile_h)
        self.dev_cams = cams_to_device(self.host_cams, device)
        p = self.plan
        self.n_rec, self.n_tiles, self.n_pixels = p.n_rec, p.n_tiles, p.n_pixels
        i32 = dict(dtype=torch.int32, device=device)
        self.rec = torch.zeros(max(p.n_rec, 1) * 12, dtype=torch.float32, device=device)
        self.rect = torch.zeros(max(p.n_rec, 1) * 2, **i32)
        self.ranges = torch.zeros(max(p.n_tiles, 1) * 3, **i32)     # [start, end) per tile, then the work order
        self.count = torch.zeros(1, **i32)
        self.status = torch.zeros(1, **i32)
        self.image = torch.zeros(max(p.n_pixels, 1) * 3, dtype=torch.float32, device=device)
        self.T_final = torch.zeros(max(p.n_pixels, 1), dtype=torch.float32, device=device)
        self.last = torch.zeros(max(p.n_pixels, 1), **i32)
        self.drec = torch.zeros(max(p.n_rec, 1) * 12, dtype=torch.float32, device=device)
        self.dL_dimage = torch.zeros_like(self.image)
        self.loss = torch.zeros(max(p.n_views, 1), dtype=torch.float64, device=device)
        self.keep_keys = keep_keys
        self.loss_ws = None
        if loss_ws:
            self.loss_ws = torch.zeros(L.lib().dg_loss_workspace_size(C.byref(self.plan)), dtype=torch.uint8,
                                       device=device)
        self.set_capacity(capacity if capacity is not None else max(4 * p.n_rec, 1 << 16))

    def set_capacity(self, cap: int) -> None:
        self.capacity = int(cap)
        dev = self.device
        self.vals = torch.zeros(max(self.capacity, 1), dtype=torch.int32, device=dev)
        self.keys = torch.zeros(max(self.capacity, 1), dtype=torch.int64, device=dev) if self.keep_keys else None
        ws = L.lib().dg_bin_sort_workspace_size(C.byref(self.plan), self.capacity)
        self.ws = torch.zeros(max(ws, 1), dtype=torch.uint8, device=dev)

    def enable_slots(self, slot_capacity: int) -> None:
        """Buffers of the deterministic backward: 9 floats per (record, tile)
        slot for slot_capacity slots, the slot offsets and the slot total."""
        self.slot_capacity = int(slot_capacity)
        dev = self.device
        self.part = torch.zeros(max(9 * self.slot_capacity, 1), dtype=torch.float32, device=dev)
        n = L.lib().dg_rasterize_bwd_slots_workspace_size(C.byref(self.plan))
        self.slot_ws = torch.zeros(max((n + 7) // 8, 1), dtype=torch.int64, device=dev)
        self.slots = torch.zeros(1, dtype=torch.int64, device=dev)

    # per-view image views (3, H, W)
    def view_image(self, v: int, buf: Optional[torch.Tensor] = None) -> torch.Tensor:
        c = self.host_cams[v]
        b = self.image if buf is None else buf
        o = 3 * c.pix_off
        return b[o:o + 3 * c.width * c.height].view(3, c.height, c.width)

    def view_pixels(self, v: int, buf: torch.Tensor) -> torch.Tensor:
        c = self.host_cams[v]
        return buf[c.pix_off:c.pix_off + c.width * c.height].view(c.height, c.width)


# ---------------------------------------------------------------------------
# wrappers with the C ABI's names
# ---------------------------------------------------------------------------
def dg_project(x: GaussianBuffer, vb: ViewBatch, stream=None) -> None:
    L.check(L.lib().dg_project(x.ref, L.ptr(vb.dev_cams), C.byref(vb.plan), L.ptr(vb.rec), L.ptr(vb.rect),
                               L.stream_handle(stream)), "dg_project")


def dg_bin_sort(vb: ViewBatch, stream=None) -> None:
    L.check(L.lib().dg_bin_sort(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), vb.capacity,
                                L.ptr(vb.keys), L.ptr(vb.vals), L.ptr(vb.ranges), L.ptr(vb.count), L.ptr(vb.ws),
                                vb.ws.numel(), L.ptr(vb.status), L.stream_handle(stream)), "dg_bin_sort")


def dg_rasterize_fwd(vb: ViewBatch, bg=(0.0, 0.0, 0.0), stream=None) -> None:
    L.check(L.lib().dg_rasterize_fwd(L.ptr(vb.rec), L.ptr(vb.vals), L.ptr(vb.ranges), L.ptr(vb.dev_cams),
                                     C.byref(vb.plan), L.floats(bg), L.ptr(vb.image), L.ptr(vb.T_final),
                                     L.ptr(vb.last), L.stream_handle(stream)), "dg_rasterize_fwd")


def dg_rasterize_count(vb: ViewBatch, bg=(0.0, 0.0, 0.0), stream=None) -> torch.Tensor:
    """dg_rasterize_fwd plus its pair counters: returns a device int64[2]
    (pairs examined while compositing, pairs that contributed)."""
    counts = torch.zeros(2, dtype=torch.int64, device=vb.image.device)
    L.check(L.lib().dg_rasterize_count(L.ptr(vb.rec), L.ptr(vb.vals), L.ptr(vb.ranges), L.ptr(vb.dev_cams),
                                       C.byref(vb.plan), L.floats(bg), L.ptr(vb.image), L.ptr(vb.T_final),
                                       L.ptr(vb.last), L.ptr(counts), L.stream_handle(stream)),
            "dg_rasterize_count")
    return counts


def dg_loss_l1(vb: ViewBatch, target: torch.Tensor, w_l1=1.0, stream=None) -> None:
    L.check(L.lib().dg_loss_l1(L.ptr(vb.image), L.ptr(target), L.ptr(vb.dev_cams), C.byref(vb.plan), w_l1,
                               L.ptr(vb.loss), L.ptr(vb.dL_dimage), L.stream_handle(stream)), "dg_loss_l1")


def dg_loss_dssim(vb: ViewBatch, target: torch.Tensor, w_l1=0.8, w_ssim=0.2, stream=None) -> None:
    ws = vb.loss_ws
    L.check(L.lib().dg_loss_dssim(L.ptr(vb.image), L.ptr(target), L.ptr(vb.dev_cams), C.byref(vb.plan), w_l1, w_ssim,
                                  L.ptr(vb.loss), L.ptr(vb.dL_dimage), L.ptr(ws), 0 if ws is None else ws.numel(),
                                  L.stream_handle(stream)), "dg_loss_dssim")


def dg_rasterize_bwd(vb: ViewBatch, x: GaussianBuffer, grads: GaussianBuffer, dL_dimage=None, bg=(0.0, 0.0, 0.0),
                     stream=None) -> None:
    g = vb.dL_dimage if dL_dimage is None else dL_dimage
    L.check(L.lib().dg_rasterize_bwd(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.vals), L.ptr(vb.ranges),
                                     L.ptr(vb.dev_cams), C.byref(vb.plan), L.floats(bg), L.ptr(vb.T_final),
                                     L.ptr(vb.last), L.ptr(g), x.ref, L.ptr(vb.drec), grads.ref,
                                     L.stream_handle(stream)), "dg_rasterize_bwd")


def dg_rasterize_bwd_records(vb: ViewBatch, bg=(0.0, 0.0, 0.0), dL_dimage=None, stream=None) -> None:
    g = vb.dL_dimage if dL_dimage is None else dL_dimage
    L.check(L.lib().dg_rasterize_bwd_records(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.vals), L.ptr(vb.ranges),
                                             L.ptr(vb.dev_cams),
                                             C.byref(vb.plan), L.floats(bg), L.ptr(vb.T_final), L.ptr(vb.last),
                                             L.ptr(g), L.ptr(vb.drec), L.stream_handle(stream)),
            "dg_rasterize_bwd_records")


def dg_rasterize_bwd_slots(vb: ViewBatch, bg=(0.0, 0.0, 0.0), dL_dimage=None, stream=None) -> None:
    """The deterministic compositing adjoint into vb.drec (needs
    vb.enable_slots() first)."""
    g = vb.dL_dimage if dL_dimage is None else dL_dimage
    L.check(L.lib().dg_rasterize_bwd_slots(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.vals), L.ptr(vb.ranges),
                                           L.ptr(vb.dev_cams), C.byref(vb.plan), L.floats(bg), L.ptr(vb.T_final),
                                           L.ptr(vb.last), L.ptr(g), L.ptr(vb.part), vb.slot_capacity,
                                           L.ptr(vb.slot_ws), vb.slot_ws.numel() * 8, L.ptr(vb.slots), L.ptr(vb.status),
                                           L.ptr(vb.drec), L.stream_handle(stream)), "dg_rasterize_bwd_slots")


def dg_xstep_from_records(vb: ViewBatch, x: GaussianBuffer, m: GaussianBuffer, v: GaussianBuffer,
                          anchor: Optional[GaussianBuffer], shared: Optional[torch.Tensor], rho, lr, beta1=0.9,
                          beta2=0.999, eps=1e-15, step=1, dev_step: Optional[torch.Tensor] = None,
                          stream=None) -> None:
    L.check(L.lib().dg_xstep_from_records(L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), L.ptr(vb.drec),
                                          x.ref, m.ref, v.ref, None if anchor is None else anchor.ref, L.ptr(shared),
                                          L.rho_arg(rho), L.floats(lr), beta1, beta2, eps, int(step),
                                          L.ptr(dev_step), L.stream_handle(stream)), "dg_xstep_from_records")


def dg_xstep_part(part: int, vb: ViewBatch, x: GaussianBuffer, m: GaussianBuffer, v: GaussianBuffer,
                  anchor: Optional[GaussianBuffer], shared: Optional[torch.Tensor], rho, lr, beta1=0.9,
                  beta2=0.999, eps=1e-15, step=1, dev_step: Optional[torch.Tensor] = None, stream=None,
                  ctas: int = 0, z_unshared: Optional[GaussianBuffer] = None,
                  gid: Optional[torch.Tensor] = None) -> None:
    """part 1: the x-step of the groups of copies without a kept record (after
    dg_project only; `ctas` > 0 bounds its grid); part 2: the rest (after
    dg_rasterize_bwd_records); part 0: both (= dg_xstep_from_records).
    z_unshared / gid: also store every unshared copy's stepped value in z."""
    L.check(L.lib().dg_xstep_part(int(part), int(ctas), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), L.ptr(vb.drec),
                                  x.ref, m.ref, v.ref, None if anchor is None else anchor.ref, L.ptr(shared),
                                  L.rho_arg(rho), L.floats(lr), beta1, beta2, eps, int(step), L.ptr(dev_step),
                                  None if z_unshared is None else z_unshared.ref, L.ptr(gid),
                                  L.stream_handle(stream)), "dg_xstep_part")


def xstep_stream_workspace(x: GaussianBuffer) -> torch.Tensor:
    """Device workspace of dg_xstep_stream for copies laid out as x."""
    nb = int(L.lib().dg_xstep_stream_workspace_size(x.ref))
    return torch.empty((nb + 15) // 16 * 4, dtype=torch.int32, device=x.data.device)


def dg_xstep_stream(vb: ViewBatch, x: GaussianBuffer, m: GaussianBuffer, v: GaussianBuffer,
                    anchor: Optional[GaussianBuffer], shared: Optional[torch.Tensor], rho, lr, ws: torch.Tensor,
                    beta1=0.9, beta2=0.999, eps=1e-15, step=1, dev_step: Optional[torch.Tensor] = None,
                    stream=None, ctas: int = 0, z_unshared: Optional[GaussianBuffer] = None,
                    gid: Optional[torch.Tensor] = None) -> None:
    """Part 1 of dg_xstep_part (the groups without a kept record) streamed by
    `ctas` persistent CTAs (0: one per SM), the same step bit for bit; ws from
    xstep_stream_workspace(x)."""
    L.check(L.lib().dg_xstep_stream(int(ctas), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), x.ref, m.ref,
                                    v.ref, None if anchor is None else anchor.ref, L.ptr(shared), L.rho_arg(rho),
                                    L.floats(lr), beta1, beta2, eps, int(step), L.ptr(dev_step),
                                    None if z_unshared is None else z_unshared.ref, L.ptr(gid), L.ptr(ws),
                                    ws.numel() * ws.element_size(), L.stream_handle(stream)), "dg_xstep_stream")


def dg_xstep_groups(vb: ViewBatch, x: GaussianBuffer, ws: torch.Tensor, stream=None) -> None:
    """Lists in ws (from xstep_stream_workspace(x)) the groups of copies
    without a kept record and those with one, for dg_xstep_listed."""
    L.check(L.lib().dg_xstep_groups(L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), x.ref, L.ptr(ws),
                                    ws.numel() * ws.element_size(), L.stream_handle(stream)), "dg_xstep_groups")


def dg_xstep_listed(part: int, vb: ViewBatch, x: GaussianBuffer, m: GaussianBuffer, v: GaussianBuffer,
                    anchor: Optional[GaussianBuffer], shared: Optional[torch.Tensor], rho, lr, ws: torch.Tensor,
                    beta1=0.9, beta2=0.999, eps=1e-15, step=1, dev_step: Optional[torch.Tensor] = None,
                    stream=None, ctas: int = 0, z_unshared: Optional[GaussianBuffer] = None,
                    gid: Optional[torch.Tensor] = None) -> None:
    """dg_xstep_part's part 1 (streamed by `ctas` CTAs, 0: one per SM) or
    part 2 (one CTA per listed group) over the lists dg_xstep_groups left in
    ws."""
    L.check(L.lib().dg_xstep_listed(int(part), int(ctas), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan),
                                    L.ptr(vb.drec), x.ref, m.ref, v.ref, None if anchor is None else anchor.ref,
                                    L.ptr(shared), L.rho_arg(rho), L.floats(lr), beta1, beta2, eps, int(step),
                                    L.ptr(dev_step), None if z_unshared is None else z_unshared.ref, L.ptr(gid),
                                    L.ptr(ws), ws.numel() * ws.element_size(), L.stream_handle(stream)),
            "dg_xstep_listed")


def dg_densify_stats(vb: ViewBatch, stats: torch.Tensor, stream=None) -> None:
    """Adds one iteration's densification statistic of every kept record into
    stats (float32, 2 per copy): the norm of its projected mean's gradient in
    normalised device units (from vb.drec) and a count."""
    L.check(L.lib().dg_densify_stats(L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), L.ptr(vb.drec),
                                     L.ptr(stats), L.stream_handle(stream)), "dg_densify_stats")


def dg_densify_decide(z: GaussianBuffer, g_off: torch.Tensor, g_copies: torch.Tensor, stats: torch.Tensor,
                      grad_threshold: float, percent_dense: float, extent: float, min_opacity: float,
                      stream=None):
    """Decision codes (int32) and output offsets (uint32 in an int32 tensor,
    n + 1 entries, total last) per global Gaussian of z."""
    n = z.n
    dev = z.data.device
    codes = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    counts = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    offsets = torch.empty(n + 1, dtype=torch.int32, device=dev)
    wsb = int(L.lib().dg_densify_workspace_size(n))
    ws = torch.empty(max(wsb, 4), dtype=torch.uint8, device=dev)
    L.check(L.lib().dg_densify_decide(z.ref, L.ptr(g_off), L.ptr(g_copies), L.ptr(stats), float(grad_threshold),
                                      float(percent_dense), float(extent), float(min_opacity), L.ptr(codes),
                                      L.ptr(counts), L.ptr(offsets), L.ptr(ws), wsb, L.stream_handle(stream)),
            "dg_densify_decide")
    return codes[:n], offsets


def dg_densify_emit(z: GaussianBuffer, codes: torch.Tensor, offsets: torch.Tensor, normals: torch.Tensor,
                    n_out: int, stream=None):
    """The densified set (n_out = offsets[n]) with each output's parent and
    whether it is the parent itself."""
    dev = z.data.device
    out = GaussianBuffer(n_out, z.deg, dev)
    src = torch.empty(max(n_out, 1), dtype=torch.int32, device=dev)
    orig = torch.empty(max(n_out, 1), dtype=torch.uint8, device=dev)
    L.check(L.lib().dg_densify_emit(z.ref, L.ptr(codes), L.ptr(offsets), L.ptr(normals), out.ref, L.ptr(src),
                                    L.ptr(orig), L.stream_handle(stream)), "dg_densify_emit")
    return out, src[:n_out], orig[:n_out]


def dg_densify_layout(codes: torch.Tensor, offsets: torch.Tensor, g_off: torch.Tensor, g_copies: torch.Tensor,
                      copy_gid: torch.Tensor, stream=None):
    """The densified copy layout in the old layout's order (device tensors):
    (new_g_off int64[n_new + 1], new_g_copies, new_copy_gid, carry int32[n_new_copies],
    copy_offsets uint32-in-int32[n_copies + 1])."""
    n_g, n_c = int(g_off.numel()) - 1, int(copy_gid.numel())
    dev = g_off.device
    n_new = int(offsets[n_g].item()) & 0xFFFFFFFF
    cap = max(2 * n_c, 1)
    new_g_off = torch.empty(n_new + 1, dtype=torch.int64, device=dev)
    new_g_copies = torch.empty(cap, dtype=torch.int32, device=dev)
    new_copy_gid = torch.empty(cap, dtype=torch.int32, device=dev)
    carry = torch.empty(cap, dtype=torch.int32, device=dev)
    copy_off = torch.empty(n_c + 1, dtype=torch.int32, device=dev)
    wsb = int(L.lib().dg_densify_layout_workspace_size(n_g, n_c))
    ws = torch.empty(max(wsb, 256) + 256, dtype=torch.uint8, device=dev)
    wp = (ws.data_ptr() + 255) & ~255
    L.check(L.lib().dg_densify_layout(L.ptr(codes), L.ptr(offsets), n_g, L.ptr(g_off), L.ptr(g_copies),
                                      L.ptr(copy_gid), n_c, L.ptr(new_g_off), L.ptr(new_g_copies),
                                      L.ptr(new_copy_gid), L.ptr(carry), L.ptr(copy_off), wp, wsb,
                                      L.stream_handle(stream)), "dg_densify_layout")
    n_new_c = int(copy_off[n_c].item()) & 0xFFFFFFFF
    return new_g_off, new_g_copies[:n_new_c], new_copy_gid[:n_new_c], carry[:n_new_c], copy_off


def dg_histogram_i32(v: torch.Tensor, lo: int, n_bins: int, stream=None) -> np.ndarray:
    """Host array of counts of v == lo + b, b < n_bins (one small copy back)."""
    counts = torch.empty(n_bins, dtype=torch.int32, device=v.device)
    L.check(L.lib().dg_histogram_i32(L.ptr(v), int(v.numel()), int(lo), int(n_bins), L.ptr(counts),
                                     L.stream_handle(stream)), "dg_histogram_i32")
    return counts.cpu().numpy().view(np.uint32).astype(np.int64)


def dg_gather_rows(src: GaussianBuffer, idx: torch.Tensor, dst: GaussianBuffer, stream=None) -> None:
    """dst row r = src row idx[r]; rows with idx[r] < 0 are left unchanged."""
    L.check(L.lib().dg_gather_rows(src.ref, L.ptr(idx), dst.ref, L.stream_handle(stream)), "dg_gather_rows")


def dg_reset_opacity(g: GaussianBuffer, cap: float = 0.01, m: Optional[GaussianBuffer] = None,
                     v: Optional[GaussianBuffer] = None, stream=None) -> None:
    """Opacities above cap brought down to it; the moments' opacity lanes zeroed."""
    L.check(L.lib().dg_reset_opacity(g.ref, float(cap), None if m is None else m.ref, None if v is None else v.ref,
                                     L.stream_handle(stream)), "dg_reset_opacity")


def dg_image_u8_to_f32(src: torch.Tensor, dst: torch.Tensor, stream=None) -> None:
    """dst (float32) = src (uint8) / 255, element by element."""
    assert src.dtype == torch.uint8 and dst.dtype == torch.float32 and src.numel() == dst.numel()
    L.check(L.lib().dg_image_u8_to_f32(L.ptr(src), L.ptr(dst), src.numel(), L.stream_handle(stream)),
            "dg_image_u8_to_f32")


def dg_image_f32_to_u8(src: torch.Tensor, dst: torch.Tensor, stream=None) -> None:
    """dst (uint8) = round(clamp(src, 0, 1) * 255)."""
    assert src.dtype == torch.float32 and dst.dtype == torch.uint8 and src.numel() == dst.numel()
    L.check(L.lib().dg_image_f32_to_u8(L.ptr(src), L.ptr(dst), src.numel(), L.stream_handle(stream)),
            "dg_image_f32_to_u8")


def dg_backward_xstep(vb: ViewBatch, x: GaussianBuffer, m: GaussianBuffer, v: GaussianBuffer,
                      anchor: Optional[GaussianBuffer], shared: Optional[torch.Tensor], rho, lr, beta1=0.9,
                      beta2=0.999, eps=1e-15, step=1, dev_step: Optional[torch.Tensor] = None, bg=(0.0, 0.0, 0.0),
                      dL_dimage=None, stream=None) -> None:
    """The compositing adjoint, then the fused projection adjoint + x-step."""
    dg_rasterize_bwd_records(vb, bg, dL_dimage, stream)
    dg_xstep_from_records(vb, x, m, v, anchor, shared, rho, lr, beta1, beta2, eps, step, dev_step, stream)


def dg_step_advance(dev_step: torch.Tensor, stream=None) -> None:
    L.check(L.lib().dg_step_advance(L.ptr(dev_step), L.stream_handle(stream)), "dg_step_advance")


def one_view_per_block(plan) -> bool:
    return all(plan.blk_view_off[k + 1] - plan.blk_view_off[k] <= 1 for k in range(plan.n_blocks))


def dg_adam_admm_step(x: GaussianBuffer, g: GaussianBuffer, m: GaussianBuffer, v: GaussianBuffer,
                      anchor: Optional[GaussianBuffer], shared: Optional[torch.Tensor], rho, lr,
                      beta1=0.9, beta2=0.999, eps=1e-15, step=1, dev_step: Optional[torch.Tensor] = None,
                      stream=None) -> None:
    L.check(L.lib().dg_adam_admm_step(x.ref, g.ref, m.ref, v.ref, None if anchor is None else anchor.ref,
                                      L.ptr(shared), L.rho_arg(rho), L.floats(lr), beta1, beta2, eps, int(step),
                                      L.ptr(dev_step), L.stream_handle(stream)), "dg_adam_admm_step")


def dg_admm_consensus(x: GaussianBuffer, u: GaussianBuffer, z: GaussianBuffer, anchor: GaussianBuffer,
                      g_off: torch.Tensor, g_copies: torch.Tensor, rho, alpha=1.0,
                      residuals: Optional[torch.Tensor] = None, stream=None) -> None:
    L.check(L.lib().dg_admm_consensus(x.ref, u.ref, z.ref, anchor.ref, L.ptr(g_off), L.ptr(g_copies),
                                      L.rho_arg(rho), float(alpha), L.ptr(residuals), L.stream_handle(stream)),
            "dg_admm_consensus")


def dg_admm_scale_duals(u: GaussianBuffer, shared: torch.Tensor, factor, stream=None) -> None:
    L.check(L.lib().dg_admm_scale_duals(u.ref, L.ptr(shared), L.floats(factor), L.stream_handle(stream)),
            "dg_admm_scale_duals")


def dg_admm_adapt(residuals: torch.Tensor, rho: torch.Tensor, factor: torch.Tensor, dev_step: torch.Tensor,
                  mu=10.0, tau_inc=2.0, tau_dec=2.0, freeze_after=2000, stream=None) -> None:
    """Eq. 10 on the device: rho (float32[5]) and factor (float32[5]) updated
    from the consensus residuals (float64[10]) while *dev_step - 1 < freeze_after."""
    L.check(L.lib().dg_admm_adapt(L.ptr(residuals), L.ptr(rho), L.ptr(factor), L.ptr(dev_step), float(mu),
                                  float(tau_inc), float(tau_dec), int(freeze_after), L.stream_handle(stream)),
            "dg_admm_adapt")


def dg_admm_rescale(u: GaussianBuffer, z: GaussianBuffer, anchor: GaussianBuffer, copy_gid: torch.Tensor,
                    shared: torch.Tensor, factor: torch.Tensor, stream=None) -> None:
    L.check(L.lib().dg_admm_rescale(u.ref, z.ref, anchor.ref, L.ptr(copy_gid), L.ptr(shared), L.ptr(factor),
                                    L.stream_handle(stream)), "dg_admm_rescale")


def dg_admm_anchor(z: GaussianBuffer, u: GaussianBuffer, copy_gid: torch.Tensor, shared: torch.Tensor,
                   anchor: GaussianBuffer, stream=None) -> None:
    L.check(L.lib().dg_admm_anchor(z.ref, u.ref, L.ptr(copy_gid), L.ptr(shared), anchor.ref,
                                   L.stream_handle(stream)), "dg_admm_anchor")


# ---------------------------------------------------------------------------
# composed passes
# ---------------------------------------------------------------------------
def forward(x: GaussianBuffer, vb: ViewBatch, bg=(0.0, 0.0, 0.0), stream=None, retry=True) -> None:
    """dg_project + dg_bin_sort + dg_rasterize_fwd.  With retry=True the
    instance count is checked on the host (one synchronisation) and the
    binning is redone with a larger capacity if it overflowed."""
    dg_project(x, vb, stream)
    vb.status.zero_()
    dg_bin_sort(vb, stream)
    if retry:
        m = int(vb.count.item()) & 0xFFFFFFFF
        if m > vb.capacity or int(vb.status.item()) & L.DG_STATUS_CAPACITY:
            vb.set_capacity(int(m * 1.25) + 1024)
            vb.status.zero_()
            dg_bin_sort(vb, stream)
    dg_rasterize_fwd(vb, bg, stream)


class RasterizeFn(torch.autograd.Function):
    """Autograd boundary: forward = dg_project + dg_bin_sort +
    dg_rasterize_fwd on a ViewBatch; backward = dg_rasterize_bwd (tile walk
    back to front from T_final and last, then the projection adjoint).  The
    differentiable input is the flat parameter tensor of a GaussianBuffer."""

    @staticmethod
    def forward(ctx, data: torch.Tensor, xbuf: GaussianBuffer, vb: ViewBatch, bg=(0.0, 0.0, 0.0)):
        assert data.data_ptr() == xbuf.data.data_ptr()
        forward(xbuf, vb, bg)
        ctx.xbuf, ctx.vb, ctx.bg = xbuf, vb, bg
        return vb.image[:3 * vb.n_pixels].clone()

    @staticmethod
    def backward(ctx, grad_image: torch.Tensor):
        xbuf, vb = ctx.xbuf, ctx.vb
        g = torch.zeros_like(vb.image)
        g[:3 * vb.n_pixels] = grad_image
        grads = xbuf.like()
        dg_rasterize_bwd(vb, xbuf, grads, dL_dimage=g.contiguous(), bg=ctx.bg)
        return grads.data, None, None, None


def rasterize(xbuf: GaussianBuffer, vb: ViewBatch, bg=(0.0, 0.0, 0.0)) -> torch.Tensor:
    """Differentiable render of all views in `vb`; returns the concatenated
    planar images (sum over views of 3 H W floats)."""
    return RasterizeFn.apply(xbuf.data, xbuf, vb, bg)
