"""Render serving over the consensus global model (Sec. 3.2: after training
only the global Gaussians z render novel views).

Continuous batching: requests carry an arrival time; the loop admits every
request that has arrived, as soon as a stream slot and HBM budget are free,
into a batch of mixed resolutions rendered by one dg_render call (one
launch per hot step for the whole batch).  Several batches are in flight at
once on separate CUDA streams, so work that arrives while others are on the
GPU overlaps with them.  A request's latency runs from its arrival to the
completion of its image in pinned host memory.
"""
from __future__ import annotations

import collections
import ctypes as C
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from . import dogs as D
from . import synth as S


class RenderBatch:
    """Device buffers and plan for one batch of views of the global model."""

    def __init__(self, z: D.GaussianBuffer, cams: Sequence[S.Camera], capacity: int, tile=(16, 16),
                 bg=(0.0, 0.0, 0.0), device="cuda"):
        self.z, self.cams, self.bg = z, list(cams), bg
        self.host_cams, self.plan = D.render_plan(self.cams, z.n, *tile)
        self.dev_cams = D.cams_to_device(self.host_cams, device)
        self.capacity = int(capacity)
        self.image = torch.empty(3 * self.plan.n_pixels, dtype=torch.float32, device=device)
        self.ws = torch.empty(L.lib().dg_render_workspace_size(C.byref(self.plan), self.capacity),
                              dtype=torch.uint8, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    @property
    def nbytes(self) -> int:
        return self.image.numel() * 4 + self.ws.numel()

    def launch(self, stream=None) -> None:
        self.status.zero_()
        L.check(L.lib().dg_render(self.z.ref, L.ptr(self.dev_cams), C.byref(self.plan), L.floats(self.bg),
                                  self.capacity, L.ptr(self.image), L.ptr(self.ws), self.ws.numel(),
                                  L.ptr(self.count), L.ptr(self.status), L.stream_handle(stream)), "dg_render")

    def view_image(self, v: int) -> torch.Tensor:
        c = self.host_cams[v]
        o = 3 * c.pix_off
        return self.image[o:o + 3 * c.width * c.height].view(3, c.height, c.width)


def render_views(z: D.GaussianBuffer, cams: Sequence[S.Camera], capacity: Optional[int] = None,
                 tile=(16, 16), bg=(0.0, 0.0, 0.0)) -> RenderBatch:
    """Render a batch synchronously, growing the instance capacity if needed."""
    npix = sum(c.width * c.height for c in cams)
    cap = capacity if capacity is not None else 2 * npix + 4096
    while True:
        rb = RenderBatch(z, cams, cap, tile, bg)
        rb.launch()
        torch.cuda.synchronize()
        m = int(rb.count.item()) & 0xFFFFFFFF
        if not (int(rb.status.item()) & L.DG_STATUS_CAPACITY):
            return rb
        cap = int(m * 1.25) + 4096


class _Slot:
    """One in-flight batch's resident buffers, allocated once: the image,
    the render workspace, count and status, the camera table, and pinned
    host staging for the image, count/status and camera table.  A slot is
    reused only after its previous batch retired (its event completed), so
    no buffer is written while the device or the host still reads it."""

    def __init__(self, ws_bytes: int, max_views: int, max_pixels: int, device):
        cam_bytes = C.sizeof(L.DgCamera) * max_views
        self.stream = torch.cuda.Stream(device)
        self.image = torch.empty(3 * max_pixels, dtype=torch.float32, device=device)
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=device)
        self.meta = torch.zeros(2, dtype=torch.int32, device=device)          # instance count, status
        self.dev_cams = torch.empty(cam_bytes, dtype=torch.uint8, device=device)
        self.host_image = torch.empty(3 * max_pixels, dtype=torch.float32, pin_memory=True)
        self.host_meta = torch.zeros(2, dtype=torch.int32, pin_memory=True)
        self.host_cams = torch.empty(cam_bytes, dtype=torch.uint8, pin_memory=True)

    @property
    def nbytes(self) -> int:
        return self.image.numel() * 4 + self.ws.numel() + self.dev_cams.numel() + 8


class RenderServer:
    """Continuous batching over the global model z.

    Admission by free HBM: when the server is provisioned (by calibrate(),
    or by the first run()), it reads the device's free memory and carves
    min(budget, free - reserve) into in-flight slots, each with resident
    buffers large enough for any batch of at most max_batch views and
    max_batch_pixels pixels.  A request is admitted as soon as it has
    arrived and a slot is free; arrivals join the open batch up to those
    limits, and batches on different slots overlap on the device.  A slot
    grows its workspace only if a batch's instances overflow it, and only
    into free HBM that is still within the budget.
    """

    def __init__(self, z: D.GaussianBuffer, budget_bytes: float = 20e9, max_batch: int = 8, n_streams: int = 4,
                 tile=(16, 16), bg=(0.0, 0.0, 0.0), inst_per_pixel: float = 2.0,
                 max_batch_pixels: int = 2 * 3840 * 2160,
                 resolutions: Sequence[tuple] = ((640, 480), (1280, 720), (1920, 1080), (3840, 2160)),
                 reserve_bytes: float = 1 << 30):
        self.z, self.budget, self.max_batch, self.tile, self.bg = z, float(budget_bytes), int(max_batch), tile, bg
        self.max_batch_pixels = int(max_batch_pixels)
        self.n_streams = int(n_streams)
        self.resolutions = [tuple(r) for r in resolutions]
        self.reserve = float(reserve_bytes)
        self.inst_per_pixel = inst_per_pixel
        self.slots: List[_Slot] = []
        self.free_hbm_at_provision: Optional[int] = None

    def calibrate(self, cams: Sequence[S.Camera], margin: float = 1.25) -> float:
        """Set the instance capacity per pixel from sample views of the model
        (margin x the largest instances-per-pixel ratio among them), so that
        a slot's workspace rarely has to grow, then provision the slots."""
        worst = 0.0
        for c in cams:
            rb = render_views(self.z, [c], tile=self.tile, bg=self.bg)
            m = int(rb.count.item()) & 0xFFFFFFFF
            worst = max(worst, m / float(c.width * c.height))
            del rb
        self.inst_per_pixel = max(self.inst_per_pixel, margin * worst)
        self.provision(force=True)
        return self.inst_per_pixel

    # ---- sizing ----------------------------------------------------------------
    def _plan(self, cams):
        return D.render_plan(list(cams), self.z.n, *self.tile)

    def _ws_size(self, plan, capacity: int) -> int:
        return int(L.lib().dg_render_workspace_size(C.byref(plan), int(capacity)))

    def _capacity_for(self, npix: int) -> int:
        return int(self.inst_per_pixel * npix) + 4096

    def _slot_ws_bytes(self) -> int:
        """A workspace that holds any admissible batch.  The workspace is a sum
        of terms in the records (views x Gaussians), the tiles, the pixels
        and the instances; the batch of max_batch views at the smallest
        resolution bounds the first, the largest resolution repeated up to
        max_batch_pixels the others, so their sum bounds every mix."""
        small = min(self.resolutions, key=lambda r: r[0] * r[1])
        large = max(self.resolutions, key=lambda r: r[0] * r[1])
        cam = lambda r: S.Camera(r[0], r[1], float(r[0]), float(r[0]), r[0] / 2, r[1] / 2, np.eye(3, dtype=np.float32),
                                 np.zeros(3, np.float32), np.zeros(3, np.float32))
        a = [cam(small)] * self.max_batch
        k = max(1, min(self.max_batch, self.max_batch_pixels // (large[0] * large[1])))
        b = [cam(large)] * k
        _, pa = self._plan(a)
        _, pb = self._plan(b)
        need = (self._ws_size(pa, self._capacity_for(small[0] * small[1] * self.max_batch))
                + self._ws_size(pb, self._capacity_for(self.max_batch_pixels)))
        return need + (1 << 20)

    def provision(self, force: bool = False) -> int:
        """Allocate the slots from free HBM within the budget.  Returns their count."""
        if self.slots and not force:
            return len(self.slots)
        self.slots = []
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        self.free_hbm_at_provision = int(free)
        ws = self._slot_ws_bytes()
        one = ws + 12 * self.max_batch_pixels + C.sizeof(L.DgCamera) * self.max_batch + 8
        usable = min(self.budget, free - self.reserve)
        n = int(min(self.n_streams, usable // one))
        if n < 1:
            raise RuntimeError(f"render server: one slot needs {one / 1e9:.2f} GB, "
                               f"{usable / 1e9:.2f} GB usable (free HBM {free / 1e9:.2f} GB, budget "
                               f"{self.budget / 1e9:.2f} GB)")
        dev = self.z.data.device
        self.slots = [_Slot(ws, self.max_batch, self.max_batch_pixels, dev) for _ in range(n)]
        return n

    def resident_bytes(self) -> int:
        return sum(s.nbytes for s in self.slots)

    def _fit_capacity(self, plan, ws_bytes: int) -> int:
        """The largest instance capacity whose workspace fits ws_bytes (0 if none)."""
        base = self._ws_size(plan, 0)
        if base > ws_bytes:
            return 0
        step = 1 << 20
        slope = max(1e-9, (self._ws_size(plan, step) - base) / step)
        cap = min(int((ws_bytes - base) / slope), 0xFFFFFFFE)
        while cap > 0 and self._ws_size(plan, cap) > ws_bytes:
            cap -= 4096
        return max(cap, 0)

    # ---- serving ---------------------------------------------------------------
    def _launch(self, slot_id: int, req: List[int], cams) -> dict:
        sl = self.slots[slot_id]
        arr, plan = self._plan(cams)
        cap = self._fit_capacity(plan, sl.ws.numel())
        npix = int(plan.n_pixels)
        raw = bytes(arr)
        sl.host_cams[:len(raw)].copy_(torch.frombuffer(bytearray(raw), dtype=torch.uint8))
        with torch.cuda.stream(sl.stream):
            sl.dev_cams[:len(raw)].copy_(sl.host_cams[:len(raw)], non_blocking=True)
            sl.meta.zero_()
            L.check(L.lib().dg_render(self.z.ref, L.ptr(sl.dev_cams), C.byref(plan), L.floats(self.bg), cap,
                                      L.ptr(sl.image), L.ptr(sl.ws), sl.ws.numel(), L.ptr(sl.meta),
                                      sl.meta.data_ptr() + 4, L.stream_handle(sl.stream)), "dg_render")
            sl.host_image[:3 * npix].copy_(sl.image[:3 * npix], non_blocking=True)
            sl.host_meta.copy_(sl.meta, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(sl.stream)
        return {"slot": slot_id, "req": req, "cams": list(cams), "host_cams": arr, "ev": ev, "cap": cap}

    def _grow(self, slot_id: int, need: int) -> None:
        """Give a slot a larger workspace, if free HBM within the budget allows."""
        sl = self.slots[slot_id]
        extra = need - sl.ws.numel()
        free, _ = torch.cuda.mem_get_info()
        if self.resident_bytes() + extra > self.budget or extra > free - self.reserve:
            raise RuntimeError(f"render server: a batch needs {need / 1e9:.2f} GB of workspace; free HBM "
                               f"{free / 1e9:.2f} GB and the budget do not allow it")
        sl.ws = None
        sl.ws = torch.empty(int(need), dtype=torch.uint8, device=self.z.data.device)

    def run(self, cams: Sequence[S.Camera], arrivals: np.ndarray, keep_images: bool = False,
            on_result: Optional[Callable[[int, torch.Tensor], None]] = None) -> Dict:
        """Serve requests cams[i] arriving at arrivals[i] seconds (wall clock
        from the start of the call).  A request's latency runs from its
        arrival to the end of its image's copy into pinned host memory.

        on_result(i, image) is called once per request as its batch retires,
        with a (3, H, W) view of the slot's pinned host buffer that stays
        valid only during the call; keep_images=True keeps a host copy of
        every image in the result's "images"."""
        self.provision()
        n = len(cams)
        pending = collections.deque(range(n))
        inflight: List[dict] = []
        free = list(range(len(self.slots)))[::-1]
        done_t = np.full(n, np.nan)
        images: List[Optional[torch.Tensor]] = [None] * n if keep_images else []
        retries = 0
        torch.cuda.synchronize()
        start_ev = torch.cuda.Event(enable_timing=True)
        start_ev.record()
        t0 = time.perf_counter()
        completed = 0
        max_inflight = 0
        while completed < n:
            now = time.perf_counter() - t0
            # retire finished batches
            for b in list(inflight):
                if not b["ev"].query():
                    continue
                sl = self.slots[b["slot"]]
                count, status = (int(v) & 0xFFFFFFFF for v in sl.host_meta.tolist())
                if status & L.DG_STATUS_CAPACITY:
                    # the instances overflowed the slot: grow its workspace and render again
                    npix = sum(c.width * c.height for c in b["cams"])
                    self.inst_per_pixel = max(self.inst_per_pixel, 1.25 * count / max(1, npix))
                    _, plan = self._plan(b["cams"])
                    self._grow(b["slot"], self._ws_size(plan, int(count * 1.25) + 4096))
                    inflight.remove(b)
                    nb = self._launch(b["slot"], b["req"], b["cams"])
                    inflight.append(nb)
                    retries += 1
                    continue
                el = start_ev.elapsed_time(b["ev"]) / 1e3
                for j, r in enumerate(b["req"]):
                    done_t[r] = el
                    if keep_images or on_result is not None:
                        hc = b["host_cams"][j]
                        o = 3 * hc.pix_off
                        img = sl.host_image[o:o + 3 * hc.width * hc.height].view(3, hc.height, hc.width)
                        if on_result is not None:
                            on_result(r, img)
                        if keep_images:
                            images[r] = img.clone()
                completed += len(b["req"])
                free.append(b["slot"])
                inflight.remove(b)
            # admit arrived requests into free slots
            while free and pending and arrivals[pending[0]] <= now:
                batch, npix = [], 0
                while pending and arrivals[pending[0]] <= now and len(batch) < self.max_batch:
                    c0 = cams[pending[0]]
                    if batch and npix + c0.width * c0.height > self.max_batch_pixels:
                        break
                    batch.append(pending.popleft())
                    npix += c0.width * c0.height
                slot = free.pop()
                inflight.append(self._launch(slot, batch, [cams[i] for i in batch]))
                max_inflight = max(max_inflight, len(inflight))
            if not inflight and pending:
                wait = arrivals[pending[0]] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
            elif inflight:
                time.sleep(0.0002)
        total = time.perf_counter() - t0
        lat = done_t - arrivals[:n]
        out = {"latency_s": lat, "p50_ms": float(np.percentile(lat, 50) * 1e3),
               "p99_ms": float(np.percentile(lat, 99) * 1e3), "views_per_s": n / total, "requests": n,
               "wall_s": total, "capacity_retries": retries, "max_inflight_batches": max_inflight,
               "slots": len(self.slots), "resident_gb": self.resident_bytes() / 1e9,
               "free_hbm_gb_at_provision": (self.free_hbm_at_provision or 0) / 1e9}
        if keep_images:
            out["images"] = images
        return out
