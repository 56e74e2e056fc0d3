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
from typing import Dict, List, Optional, Sequence

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


class RenderServer:
    def __init__(self, z: D.GaussianBuffer, budget_bytes: float = 20e9, max_batch: int = 8, n_streams: int = 4,
                 tile=(16, 16), bg=(0.0, 0.0, 0.0), inst_per_pixel: float = 2.0,
                 max_batch_pixels: int = 2 * 3840 * 2160):
        self.z, self.budget, self.max_batch, self.tile, self.bg = z, budget_bytes, max_batch, tile, bg
        self.max_batch_pixels = int(max_batch_pixels)
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        # pinned staging for each slot's images, allocated once up front: a
        # pinned allocation of this size takes tens to hundreds of
        # milliseconds, so batches are admitted only up to max_batch_pixels
        # (a single request larger than that grows its slot's buffer once)
        self.host_bufs: List[Optional[torch.Tensor]] = [
            torch.empty(3 * self.max_batch_pixels, dtype=torch.float32, pin_memory=True) for _ in range(n_streams)]
        self.inst_per_pixel = inst_per_pixel

    def calibrate(self, cams: Sequence[S.Camera], margin: float = 1.25) -> float:
        """Set the instance capacity per pixel from sample views of the model
        (margin x the largest instances-per-pixel ratio among them), so that
        serving rarely has to re-render a batch whose binning overflowed."""
        worst = 0.0
        for c in cams:
            rb = render_views(self.z, [c], tile=self.tile, bg=self.bg)
            m = int(rb.count.item()) & 0xFFFFFFFF
            worst = max(worst, m / float(c.width * c.height))
        self.inst_per_pixel = max(self.inst_per_pixel, margin * worst)
        return self.inst_per_pixel

    def _est_bytes(self, cams) -> int:
        npix = sum(c.width * c.height for c in cams)
        cap = int(self.inst_per_pixel * npix) + 4096
        # images + records + sort buffers, as the workspace query computes them
        _, plan = D.render_plan(list(cams), self.z.n, *self.tile)
        return 12 * npix + int(L.lib().dg_render_workspace_size(C.byref(plan), cap))

    def run(self, cams: Sequence[S.Camera], arrivals: np.ndarray) -> Dict:
        """Serve requests cams[i] arriving at arrivals[i] seconds (wall clock
        from the start of the call).  Returns latencies (s) and throughput."""
        n = len(cams)
        pending = collections.deque(range(n))
        inflight: List[dict] = []
        free = list(range(len(self.streams)))
        used = 0
        done_t = np.full(n, np.nan)
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
                if b["ev"].query():
                    rb = b["rb"]
                    if int(rb.status.item()) & L.DG_STATUS_CAPACITY:
                        # grow and re-render on the same slot
                        m = int(rb.count.item()) & 0xFFFFFFFF
                        self.inst_per_pixel = max(self.inst_per_pixel,
                                                  1.25 * m / max(1, sum(c.width * c.height for c in rb.cams)))
                        used -= rb.nbytes
                        b["rb"] = None
                        rb2 = self._make(b["slot"], rb.cams, int(m * 1.25) + 4096)
                        used += rb2.nbytes
                        self._launch(b, rb2)
                        retries += 1
                        continue
                    el = start_ev.elapsed_time(b["ev"]) / 1e3
                    for r in b["req"]:
                        done_t[r] = el
                    completed += len(b["req"])
                    used -= rb.nbytes
                    free.append(b["slot"])
                    inflight.remove(b)
            # admit arrived requests into free slots under the HBM budget
            while free and pending and arrivals[pending[0]] <= now:
                batch = []
                npix = 0
                while pending and arrivals[pending[0]] <= now and len(batch) < self.max_batch:
                    c0 = cams[pending[0]]
                    if batch and npix + c0.width * c0.height > self.max_batch_pixels:
                        break
                    cand = batch + [pending[0]]
                    need = self._est_bytes([cams[i] for i in cand])
                    if used + need > self.budget and batch:
                        break
                    if used + need > self.budget and inflight:
                        break
                    batch.append(pending.popleft())
                    npix += c0.width * c0.height
                if not batch:
                    break
                bc = [cams[i] for i in batch]
                npix = sum(c.width * c.height for c in bc)
                b = {"slot": free.pop(), "req": batch}
                rb = self._make(b["slot"], bc, int(self.inst_per_pixel * npix) + 4096)
                used += rb.nbytes
                self._launch(b, rb)
                inflight.append(b)
                max_inflight = max(max_inflight, len(inflight))
            if not inflight and pending:
                wait = arrivals[pending[0]] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
            elif inflight:
                time.sleep(0.0002)
        total = time.perf_counter() - t0
        lat = done_t - arrivals[:n]
        return {"latency_s": lat, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "views_per_s": n / total, "requests": n,
                "wall_s": total, "capacity_retries": retries, "max_inflight_batches": max_inflight}

    def _make(self, slot: int, cams, capacity: int) -> RenderBatch:
        # allocate on the slot's stream: the caching allocator then reuses the
        # memory only after that stream's work on it
        with torch.cuda.stream(self.streams[slot]):
            return RenderBatch(self.z, cams, capacity, self.tile, self.bg)

    def _launch(self, b: dict, rb: RenderBatch) -> None:
        slot = b["slot"]
        s = self.streams[slot]
        need = rb.image.numel()
        hb = self.host_bufs[slot]
        if hb is None or hb.numel() < need:
            hb = torch.empty(max(need, 3 * self.max_batch_pixels), dtype=torch.float32, pin_memory=True)
            self.host_bufs[slot] = hb
        with torch.cuda.stream(s):
            rb.launch(s)
            host = hb[:need]
            host.copy_(rb.image, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        b["rb"], b["ev"], b["host"] = rb, ev, host
