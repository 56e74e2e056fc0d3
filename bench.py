"""Benchmark: batched DOGS training iterations (fwd + bwd + ADMM) and render
serving at 6M Gaussians on one B300.

Workload (default "large"): synthetic aerial city of 6,000,000 Gaussians, SH
degree 3, FP32, split into K = 8 uneven blocks on a 2 x 4 ground grid (loads
Dirichlet(2) from the seed), 10 % of the Gaussians on interior borders shared
by 2-4 blocks (6.63M local copies); one 1920x1080 view per block per
iteration at 45 deg pitch (V = 8), loss 0.8 L1 + 0.2 D-SSIM against targets
rendered from a ground-truth set of the same law; Adam + ADMM penalty
(rho = 1e-3 on every property group); the consensus runs in every timed
step.  One step = project, bin_sort, rasterize_fwd, loss, rasterize_bwd,
adam_admm_step, admm_consensus for all 8 blocks, replayed from a CUDA graph.
The working set (~20 GB) is far above L2, so no flush is needed.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "train iters/s (fwd+bwd+ADMM) & render p50/p99 ms at 6M Gaussians, 1 B300"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 60; 100 for dogs2m_k4)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["large", "medium", "small", "raster4k", "single1m", "dogs2m_k4", "street"])
    ap.add_argument("--views-per-block", type=int, default=None,
                    help="views of each block per iteration (8: the V=64 variant; gradients then go through "
                         "the gradient buffer and the separate x-step)")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-seq", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-densify-probe", action="store_true", help="skip timing one densification at the end")
    ap.add_argument("--tile", default="16x16")
    ap.add_argument("--no-autotune", action="store_true", help="keep --tile and the default compositing variant")
    ap.add_argument("--idle-ctas", type=int, default=0,
                    help="CTAs per SM of the x-step part that runs beside compositing (0: one per SM streamed, "
                         "one per group of copies as a grid)")
    ap.add_argument("--idle-mode", default=None, choices=["stream", "stream_early", "grid"],
                    help="that x-step part: streamed by persistent CTAs beside the compositing adjoint, or a grid "
                         "launched after the projection (default: the autotuner's choice, else stream)")
    ap.add_argument("--no-overlap", action="store_true", help="run that x-step part inline on the main stream")
    ap.add_argument("--variant", default=None,
                    help="compositing variant W,S[,Wb,Sb] (warps per tile, staged per thread; backward)")
    ap.add_argument("--loss", default="dssim", choices=["dssim", "l1"])
    ap.add_argument("--profile", action="store_true", help="setup + warmup + a few eager steps only (for ncu)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.steps is None:
        args.steps = w.get("steps", 60)
    if args.views_per_block is None:
        args.views_per_block = w.get("views_per_block", 1)
    return args


# Workloads.  "large" is the headline (the K = 8, 6M-Gaussian aerial step with
# the consensus in every step); the others are the other measured configs:
#   raster4k   plain rasteriser fwd + bwd of one 128x128 view, 4,096 Gaussians
#   single1m   plain single-model 3DGS step: 1M Gaussians, one 1920x1080 view
#              from a grid camera (pitch 45-90 deg), Adam, no consensus
#   dogs2m_k4  K = 4 uneven blocks (loads 0.30/0.20/0.35/0.15), 2M Gaussians,
#              5 % shared, 8 views per block at 1600x1200, consensus every 100
#   street     street-level views (eye height, along the streets) of a 2M
#              Gaussian city, K = 4, one 1920x1080 view per block
# intv: consensus interval (1 = every step; None = no consensus);
# oracle_frac: the CPU baseline renders 1/oracle_frac of each block's copies.
WORKLOADS = {
    "large": dict(kind="dogs", n_global=6_000_000, cols=2, rows=4, shared=0.10, seed=1004, width=1920,
                  height=1080, pool=4, intv=1, rho=1e-3, oracle_frac=64, serve=True, densify=True),
    "small": dict(kind="dogs", n_global=200_000, cols=2, rows=2, shared=0.05, seed=1003, width=640, height=480,
                  pool=2, intv=1, rho=1e-3, oracle_frac=16),
    # same law and views as "large" at 1/6 of the Gaussians: a profiling case of a few GB, above L2
    "medium": dict(kind="dogs", n_global=1_000_000, cols=2, rows=4, shared=0.10, seed=1004, width=1920,
                   height=1080, pool=2, intv=1, rho=1e-3, oracle_frac=32),
    "raster4k": dict(kind="raster", n_global=4096, seed=1001, width=128, height=128),
    "single1m": dict(kind="dogs", n_global=1_000_000, cols=1, rows=1, shared=0.0, seed=1002, width=1920,
                     height=1080, pool=4, cameras="grid", intv=None, rho=0.0, oracle_frac=32, seq=False),
    "dogs2m_k4": dict(kind="dogs", n_global=2_000_000, cols=2, rows=2, shared=0.05, seed=1003, width=1600,
                      height=1200, pool=2, views_per_block=8, loads=(0.30, 0.20, 0.35, 0.15), intv=100,
                      rho=1e-3, oracle_frac=256, steps=100),
    "street": dict(kind="dogs", n_global=2_000_000, cols=2, rows=2, shared=0.10, seed=1006, width=1920,
                   height=1080, pool=4, cameras="street", log_scale_mu=-2.3, intv=1, rho=1e-3, oracle_frac=64),
}


def dist_setup():
    """One process per GPU under torchrun (replicas: every rank runs the whole
    workload on its own GPU; the only collectives are the timing barrier and
    the max over ranks).  NCCL with GPUs, gloo without (the CPU tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist, rank, ws
    return None, 0, 1


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "50", "-i", str(dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def wait_first(self, timeout: float = 3.0) -> None:
        """Return once nvidia-smi has written its first sample (it takes a few
        hundred ms to start), so that the samples cover the timed region; at
        most `timeout` seconds, and at once if the sampler is not running."""
        t0 = time.time()
        while self.p is not None and self.p.poll() is None and time.time() - t0 < timeout:
            if os.path.getsize(self.f.name) > 0:
                return
            time.sleep(0.02)

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1])); pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def traffic_for(kernel: str, workload: str):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on this workload and the kernel's source has not changed since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    entries = json.load(open(p)).get(kernel) or []
    for d in (entries if isinstance(entries, list) else [entries]):
        if d.get("workload") != workload:
            continue
        src = os.path.join(ROOT, "paper_2405_13943_b300", "csrc", d["source"])
        if os.path.exists(src) and hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == d["source_sha"]:
            return d
    return None


# ---------------------------------------------------------------------------
def build_workload(name: str, views_per_block: int = 1):
    from paper_2405_13943_b300 import synth as S
    w = WORKLOADS[name]
    return S.dogs_workload(w["n_global"], w["cols"], w["rows"], w["shared"], w["seed"],
                           views_per_step=views_per_block, pool=w["pool"], width=w["width"], height=w["height"],
                           loads=w.get("loads"), cameras=w.get("cameras", "aerial"),
                           log_scale_mu=w.get("log_scale_mu", -1.0))


def consensus_arg(w):
    """The trainer's consensus rule for a workload: every step (True), never
    (False), or every intv-th iteration as Alg. 2 has it (None: t mod intv)."""
    if w.get("intv") is None:
        return False
    return True if w["intv"] == 1 else None


def render_targets(gt_buf, views, tile):
    """Targets: the ground-truth set rendered at each pool entry's views, laid
    out as the training batch lays out its images (same view order/sizes),
    as 8-bit images like the training photographs they stand for.  Returns
    (float32 device targets = bytes / 255, uint8 device targets)."""
    import torch
    from paper_2405_13943_b300 import dogs as D
    from paper_2405_13943_b300 import serve
    out, out8 = [], []
    for vs in views:
        rb = serve.render_views(gt_buf, vs, tile=tile)
        b = torch.empty(rb.image.numel(), dtype=torch.uint8, device=rb.image.device)
        D.dg_image_f32_to_u8(rb.image, b)
        f = torch.empty_like(rb.image)
        D.dg_image_u8_to_f32(b, f)
        out.append(f)
        out8.append(b)
        del rb
    torch.cuda.synchronize()
    return out, out8


# FP32 operations of the method per (pixel, Gaussian) pair, a multiply-add
# counted as 2 and the exponential as 1.  Every pair a pass visits costs the
# evaluation: offset 2, quadratic form 9, exp 1, alpha = min(0.99, o G) 2
# -> 14.  A composited pair (alpha >= 1/255, before the stop) adds
#   forward:  T (1 - alpha) 2, weight alpha T 1, colour accumulation 6 -> 9
#   backward: T / (1 - alpha) 2, colour gradients alpha T dL/dC 4, dL/dalpha
#             from (c - B) and the background term 13, B update 9, dL/dG and
#             dL/do 2, dL/dpower 1, mean gradient 8, conic gradient 5,
#             accumulation of 9 sums 9 -> 53
# The forward visits the positions up to each pixel's stop, the backward the
# positions up to each pixel's last composited one (the sum of `last`).
FLOPS_EVAL = 14
FLOPS_FWD_USED = 9
FLOPS_BWD_USED = 53


def measure_fp32_peak(local: int, reps: int = 7) -> dict:
    """The device's FP32 rate from the library's FMA probe (8 independent
    chains of fused multiply-adds per thread, 8 CTAs of 256 threads per SM),
    timed with CUDA events, best of `reps` launches, with the SM clock
    sampled while it runs."""
    import torch
    from paper_2405_13943_b300 import _lib as L
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    blocks = 8 * n_sm
    out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    iters = 2048
    L.lib().dg_probe_fma(iters, blocks, L.ptr(out), L.stream_handle())      # warm
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.wait_first()
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        flops = 0
        for _ in range(10):
            flops += L.lib().dg_probe_fma(iters, blocks, L.ptr(out), L.stream_handle())
        e1.record()
        torch.cuda.synchronize()
        best = max(best, flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    c = clk.stop()
    if not math.isfinite(float(out[0].item())):
        raise RuntimeError("FMA probe produced a non-finite value")
    return {"tflops": round(best, 2), "sm_mhz_median": c.get("sm_mhz"), "sm_max_mhz": c.get("sm_max_mhz"),
            "how": f"dg_probe_fma: {blocks} CTAs x 256 threads x 8 FMA chains, CUDA events, best of {reps}",
            "nominal_tflops": round(n_sm * 128 * 2 * float(c.get("sm_max_mhz") or 2032.0) * 1e6 / 1e12, 2)}


def copy_groups(tr, rect):
    """Per copy: kept record in its block's view (bool), and per group of 128
    consecutive copies (the x-step's CTAs): any kept record."""
    n_c = tr.split.n_copies
    kept = np.zeros(n_c, bool)
    vis = (rect[:, 0] & 0xFFFF) != (rect[:, 1] & 0xFFFF)
    for c in tr.vb.host_cams:
        b, e = int(c.gauss_begin), int(c.gauss_end)
        kept[b:e] |= vis[int(c.rec_off):int(c.rec_off) + e - b]
    ng = -(-n_c // 128)
    grp = np.zeros(ng * 128, bool)
    grp[:n_c] = kept
    return kept, grp.reshape(ng, 128).any(1)


def algorithmic_bytes(tr, vb_rect_visible: int, n_visible_copies: int, active_groups=None, zfuse=False,
                      instances: int = 0, listed: bool = False, idle_tests: bool = True):
    sp = tr.split
    P = 59
    n_c = sp.n_copies
    n_sc = int(sp.blk_nshared.sum())
    cnt = np.diff(sp.g_off)
    sg = int((cnt > 1).sum())
    ug = int((cnt == 1).sum())
    sc = int(cnt[cnt > 1].sum())
    out = {
        # x, g, m, v read + x, m, v written per float; anchor read per shared float
        "adam_admm_step": n_c * P * 28 + n_sc * P * 4,
        # fused projection adjoint + x-step: x, m, v read and written per float, anchor per shared
        # float, and per visible record its 2D gradients (48 B) and rectangle (8 B)
        "xstep": n_c * P * 24 + n_sc * P * 4 + n_visible_copies * 56,
        # shared: x, u read + u, anchor written per copy float; z_prev read + z written per global float;
        # unshared: x read + z written
        "admm_consensus": P * (16 * sc + 8 * sg + 8 * ug),
        # every record (view, copy): mean/opacity read (16 B) + rect (8 B); visible records: rest of the
        # params (224 B) + record (48 B)
        "project": tr.vb.n_rec * 24 + n_visible_copies * 224 + vb_rect_visible * 48,
        # binning: both passes (count, scatter) read every record's rectangle (8 B) and each visible
        # record's culling fields (mean, conic, opacity: 32 B); the scatter writes an 8-byte
        # (depth, record) pair per kept instance, the segment sort reads it and writes the 4-byte value
        "bin_sort": 2 * 8 * tr.vb.n_rec + 2 * 32 * vb_rect_visible + 20 * instances,
    }
    if active_groups is not None:
        # split x-step: part 2 over the groups of 128 copies with a kept record, part 1 over the
        # others.  listed: the two lists are built first from every copy's 8-byte rectangle (and one
        # 4-byte entry per group); idle_tests: part 1 reads the rectangle of each of its copies to
        # find its groups (the grid form, or the streamed form building its own list)
        act = np.repeat(active_groups, 128)[:n_c]
        sh = sp.copy_shared().astype(bool)
        na, nsa = int(act.sum()), int((act & sh).sum())
        out["xstep"] = na * P * 24 + nsa * P * 4 + n_visible_copies * 56
        out["xstep_idle"] = (n_c - na) * (P * 24 + (8 if idle_tests else 0)) + (n_sc - nsa) * P * 4
        if listed:
            out["xstep_groups"] = n_c * 8 + 4 * len(active_groups)
        if zfuse:
            # the unshared copies' values stored into z (4 B per float) with their global ids (4 B)
            # here, so the consensus moves the shared globals' bytes only
            out["xstep"] += (na - nsa) * (P * 4 + 4)
            out["xstep_idle"] += (n_c - na - (n_sc - nsa)) * (P * 4 + 4)
            out["admm_consensus"] = P * (16 * sc + 8 * sg)
    return out


def run_ours(args, dist, rank, world):
    import torch
    from paper_2405_13943_b300 import _lib as L
    from paper_2405_13943_b300 import build as B
    from paper_2405_13943_b300 import dogs as D
    from paper_2405_13943_b300 import serve
    from paper_2405_13943_b300 import synth as S
    from paper_2405_13943_b300 import trainer as T

    B.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    W = WORKLOADS[args.workload]
    cons = consensus_arg(W)
    cons_values = (False, True) if cons is None else (cons,)
    tile = tuple(int(v) for v in args.tile.split("x"))
    t_setup = time.time()
    wl = build_workload(args.workload, args.views_per_block)
    z0 = D.GaussianBuffer.from_synth(wl.z0)
    gt = D.GaussianBuffer.from_synth(wl.gt)
    targets, targets8 = render_targets(gt, wl.views, tile)
    del gt
    if args.variant:
        D.set_raster_variant(*[int(v) for v in args.variant.split(",")])
    tr = T.DogsTrainer(wl.split, z0, wl.views, targets, rho=(W["rho"],) * 5, tile=tile, loss=args.loss,
                       overlap=not args.no_overlap, intv=W["intv"] or 100)
    tr.idle_ctas_per_sm = args.idle_ctas
    if args.idle_mode:
        tr.idle_mode = args.idle_mode
    m_max = tr.calibrate_capacity()
    tuned = None
    if not args.no_autotune and not args.profile and not args.variant:
        from paper_2405_13943_b300 import autotune
        tuned = autotune.tune(tr, use_cache=False, idle_modes=(args.idle_mode,) if args.idle_mode else ("stream", "grid"),
                              consensus=bool(cons))
        tile = tr.tile
        m_max = tr.calibrate_capacity()
    torch.cuda.synchronize()
    setup_s = time.time() - t_setup

    for _ in range(args.warmup):
        tr.step(consensus=cons)
    tr.prepare_graphs(cons_values)
    torch.cuda.synchronize()
    if tr.overflowed():
        raise RuntimeError("instance capacity overflow during warmup")
    if args.profile:
        # two eager iterations inside an NVTX range "dogs_step" (ncu --nvtx-include dogs_step/)
        torch.cuda.nvtx.range_push("dogs_step")
        for _ in range(2):
            tr.step(consensus=cons, graph=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            print(json.dumps({"profile_run": True, "instances": m_max}))
        return

    # ---- timed region: graph replays ------------------------------------------------
    clocks = ClockSampler(local)
    clocks.wait_first()
    barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_first = tr.t
    e0.record()
    for _ in range(args.steps):
        tr.step(consensus=cons)
    e1.record()
    torch.cuda.synchronize()
    barrier(dist)
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    if tr.overflowed():
        raise RuntimeError("instance capacity overflow in the timed region")
    ms = max_over_ranks(dist, ms)

    # ---- per-call durations (eager launches, events on the launching stream) ----------
    fused = tr.fused and D.one_view_per_block(tr.vb.plan)
    split = tr._split_xstep()
    zf = tr._zfuse(True)        # the x-step stores the unshared copies into z, as in the graph
    zargs = tr._zargs(zf)
    vb = tr.vb
    xs_args = (tr.x, tr.m, tr.v, tr.anchor, tr.shared, tr.rho, tr.lr)

    def bwd_fused():
        D.dg_rasterize_bwd_records(vb, bg=tr.bg)

    calls = [("project", lambda: D.dg_project(tr.x, vb))]
    listed = split and tr.listed_part2
    if split:       # the part that the graph runs on a side stream, timed here in sequence
        if listed:  # the two group lists, then part 1 over the first (streamed) or testing each group (grid)
            calls.append(("xstep_groups", lambda: D.dg_xstep_groups(vb, tr.x, tr.xs_ws)))
        if tr.idle_mode.startswith("stream") and listed:
            calls.append(("xstep_idle", lambda: D.dg_xstep_listed(1, vb, *xs_args, tr.xs_ws, step=1,
                                                                  dev_step=tr.dev_step,
                                                                  ctas=tr.n_sm * tr.idle_ctas_per_sm, **zargs)))
        elif tr.idle_mode.startswith("stream"):
            calls.append(("xstep_idle", lambda: D.dg_xstep_stream(vb, *xs_args, tr.xs_ws, step=1, dev_step=tr.dev_step,
                                                                  ctas=tr.n_sm * tr.idle_ctas_per_sm, **zargs)))
        else:
            calls.append(("xstep_idle", lambda: D.dg_xstep_part(1, vb, *xs_args, step=1, dev_step=tr.dev_step,
                                                                ctas=tr.n_sm * tr.idle_ctas_per_sm, **zargs)))
    calls += [("bin_sort", lambda: D.dg_bin_sort(vb)),
              ("rasterize_fwd", lambda: D.dg_rasterize_fwd(vb, tr.bg)),
              ("loss", lambda: tr._loss(tr.targets[tr.t % len(tr.view_sets)]))]
    if fused and listed:    # part 2 over the groups listed in tr.xs_ws by the xstep_groups call
        calls += [("rasterize_bwd", bwd_fused),
                  ("xstep", lambda: D.dg_xstep_listed(2, vb, *xs_args, tr.xs_ws, step=1, dev_step=tr.dev_step,
                                                      **zargs))]
    elif fused:     # compositing adjoint, then projection adjoint + x-step fused
        calls += [("rasterize_bwd", bwd_fused),
                  ("xstep", lambda: D.dg_xstep_part(2 if split else 0, vb, *xs_args, step=1,
                                                    dev_step=tr.dev_step, **zargs))]
    else:
        calls += [("rasterize_bwd", lambda: D.dg_rasterize_bwd(vb, tr.x, tr.grad, bg=tr.bg)),
                  ("adam_admm_step", lambda: D.dg_adam_admm_step(*xs_args[:1], tr.grad, *xs_args[1:], step=1,
                                                                 dev_step=tr.dev_step))]
    zc = tr.z_shared() if zf else tr.z
    calls.append(("admm_consensus", lambda: D.dg_admm_consensus(tr.x, tr.u, zc, tr.anchor, tr.g_off, tr.g_copies,
                                                                tr.rho, tr.alpha, tr.residuals)))
    names = [n for n, _ in calls]
    acc = {n: 0.0 for n in names}
    n_eager = max(3, min(args.steps, 20))
    l0 = L.lib().dg_launch_count()
    pairs = 0.0
    for i in range(n_eager):
        p = tr.t % len(tr.view_sets)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        vb.dev_cams.copy_(tr.cam_pool[p], non_blocking=True)
        D.dg_step_advance(tr.dev_step)
        # the GPU spins ~0.1 ms first, so the first call is already queued when
        # ev[0] is reached and its interval holds no host launch latency
        torch.cuda._sleep(200_000)
        ev[0].record()
        for k, (n, fn) in enumerate(calls):
            fn()
            ev[k + 1].record()
        torch.cuda.synchronize()
        for k, n in enumerate(names):
            acc[n] += ev[k].elapsed_time(ev[k + 1]) / n_eager
        # (pixel, Gaussian) pairs the backward evaluates: every list position
        # up to each pixel's last contributor
        pairs += float(vb.last[:vb.n_pixels].sum(dtype=torch.int64)) / n_eager
        tr.t += 1
    launches_per_step = (L.lib().dg_launch_count() - l0) / n_eager
    eager_ms = sum(acc.values())

    rect = vb.rect.view(-1, 2)[:vb.n_rec].cpu().numpy().view(np.uint32)
    vis_rec = int(((rect[:, 0] & 0xFFFF) != (rect[:, 1] & 0xFFFF)).sum())
    instances = int(vb.count.item())
    _, active_groups = copy_groups(tr, rect)
    alg = algorithmic_bytes(tr, vis_rec, vis_rec, active_groups if split else None, zf, instances,
                            listed=listed, idle_tests=not (listed and tr.idle_mode.startswith("stream")))
    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    kern = {}
    for n in names:
        d = {"ms": round(acc[n], 4)}
        if n in alg:
            d["gbs"] = round(alg[n] / (acc[n] * 1e-3) / 1e9, 1)
            d["frac_hbm"] = round(alg[n] / (acc[n] * 1e-3) / 1e9 / hbm_peak, 3)
        kern[n] = d
    # compositing kernels: FP32 work of the pairs they visit and composite
    # (counted by dg_rasterize_count on every pool entry, outside the timed
    # region) against the FP32 peak: SMs x 128 lanes x 2 x maximum SM clock
    seen = used = 0.0
    for p in range(len(tr.view_sets)):
        vb.dev_cams.copy_(tr.cam_pool[p])
        D.dg_project(tr.x, vb)
        D.dg_bin_sort(vb)
        c = D.dg_rasterize_count(vb, tr.bg).cpu().numpy()
        seen += float(c[0]) / len(tr.view_sets)
        used += float(c[1]) / len(tr.view_sets)
    fp32 = measure_fp32_peak(local)
    fp32_peak = fp32["tflops"]
    work = {"rasterize_fwd": (seen * FLOPS_EVAL + used * FLOPS_FWD_USED,
                              {"pairs_visited": int(seen), "pairs_composited": int(used)}),
            "rasterize_bwd": (pairs * FLOPS_EVAL + used * FLOPS_BWD_USED,
                              {"pairs_visited": int(pairs), "pairs_composited": int(used)})}
    for n, (flops, info) in work.items():
        tf = flops / (acc[n] * 1e-3) / 1e12
        kern[n].update({"tflops": round(tf, 2), "frac_fp32": round(tf / fp32_peak, 3), **info})
    # the longest-running kernel with a roofline model (an FLOP count or algorithmic bytes); on the
    # default workload that is also the longest of all, on smaller ones the loss can be longer
    dom = max((n for n in names if n in work or n in alg), key=lambda n: acc[n])
    tinfo = traffic_for(dom, f"{args.workload}:V{len(wl.views[0])}:{vb.plan.tile_w}x{vb.plan.tile_h}")
    traffic = tinfo["bytes_per_launch"] if tinfo else None
    if dom in ("rasterize_fwd", "rasterize_bwd"):
        achieved = kern[dom]["tflops"]
        roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": round(fp32_peak, 2),
                    "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 3),
                    "peak_source": f"measured FP32 FMA probe ({fp32['how']}; median SM clock "
                                   f"{fp32['sm_mhz_median']} MHz; nominal {fp32['nominal_tflops']} TFLOP/s)",
                    "traffic": traffic, "flops_per_launch": int(work[dom][0]), **work[dom][1]}
    else:
        achieved = alg[dom] / (acc[dom] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm_peak,
                    "unit": "GB/s", "frac": round(achieved / hbm_peak, 3), "peak_source": f"{peak_src} hbm_gbs",
                    "traffic": traffic, "algorithmic_bytes": int(alg[dom])}

    # ---- end to end through host buffers ---------------------------------------------------
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(tr, args, dist, targets8, cons, cons_values)

    # ---- sequential per-block comparator -----------------------------------------------------
    comparator = None
    if not args.no_seq and W.get("seq", True):
        seq = T.SequentialTrainer(wl.split, z0.clone(), wl.views, targets, rho=(W["rho"],) * 5, tile=tile,
                                  loss=args.loss, intv=W["intv"] or 100)
        seq.calibrate_capacity()
        for _ in range(2):
            seq.step(consensus=cons)
        torch.cuda.synchronize()
        # as many steps as the batched form times when the consensus is periodic
        # (one consensus in each window of intv steps); else a quarter of them
        n_seq = args.steps if cons is None else max(3, args.steps // 4)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(n_seq):
            seq.step(consensus=cons)
        s1.record()
        torch.cuda.synchronize()
        seq_ms = s0.elapsed_time(s1) / n_seq
        comparator = {"form": "sequential per-block (same kernels, one block at a time, no graph, consensus "
                              "gathers/scatters copies)", "ms_per_step": round(seq_ms, 3),
                      "iters_per_s": round(1e3 / seq_ms, 3), "speedup_batched": round(seq_ms / ms, 3)}
        del seq
        torch.cuda.empty_cache()

    # ---- render serving over the global model -----------------------------------------------------
    render = None
    if not args.no_serve and args.serve_seconds > 0 and W.get("serve"):
        render = run_serving(tr.z, args, tile)

    # ---- CPU baseline (oracle, bounded sample) --------------------------------------------------------
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baselines(wl, args)

    # ---- one densification of the trained state (off the per-iteration path: every 200 iterations) --
    densify = None
    if not args.no_densify_probe and W.get("densify"):
        densify = densify_probe(tr, wl, D)

    value = world * 1e3 / ms
    if rank == 0:
        line = {
            "metric": metric_of(args), "value": round(value, 4), "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (city-law aerial scene, seeded; targets 8-bit images)",
            "config": {"workload": workload_name(args, wl),
                       "blocks": wl.split.K, "copies": wl.split.n_copies, "views_per_step": len(wl.views[0]),
                       "tile": f"{tr.tile[0]}x{tr.tile[1]}",
                       "raster_variant": {"fwd": {"warps_per_tile": tr.vb.plan.raster_warps,
                                                  "staged_per_thread": tr.vb.plan.raster_stage},
                                          "bwd": {"warps_per_tile": tr.vb.plan.raster_warps_bwd or tr.vb.plan.raster_warps,
                                                  "staged_per_thread": tr.vb.plan.raster_stage_bwd or tr.vb.plan.raster_stage}},
                       "autotune": (None if tuned is None else
                                    {"best_ms": tuned["ms"], "tiles": len(tuned["candidates"]),
                                     "variants_per_tile": len(tuned["candidates"][0]["variants"]),
                                     "idle_mode_ms": tuned.get("idle_modes")}),
                       "loss": "0.8 L1 + 0.2 D-SSIM" if args.loss == "dssim" else "L1",
                       "consensus_every_timed_step": W["intv"] == 1,
                       "consensus_steps_timed": (args.steps if W["intv"] == 1 else 0 if W["intv"] is None else
                                                 sum(1 for t in range(t_first, t_first + args.steps)
                                                     if t % W["intv"] == 0)),
                       "cuda_graph": True,
                       "xstep_split": (None if not split else
                                       {"idle_groups_on_side_stream": round(1.0 - float(active_groups.mean()), 3),
                                        "mode": tr.idle_mode, "side_ctas_per_sm": tr.idle_ctas_per_sm}),
                       "unshared_z_stored_by_xstep": bool(zf),
                       "l2": "working set > L2 (no flush needed)", "instances_per_step": instances,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "setup_s": round(setup_s, 1)},
            "kernels_ms": kern, "eager_ms_per_step": round(eager_ms, 3),
            "roofline": roofline, "fp32_peak": fp32, "clocks": clk,
            "gpu_launches": int(launches_per_step * args.steps),
            "e2e": e2e, "comparator": comparator, "render": render, "cpu_baseline": cpu, "densify": densify,
        }
        print(json.dumps(line))


def raster_problem(args):
    """The plain rasteriser config: Gaussians of the cube law (SH degree 0,
    rendered colours U(0,1)), one pinhole view from (0, 0, -4) along +z, and
    the target rendered from a second seed's Gaussians."""
    from paper_2405_13943_b300 import synth as S
    w = WORKLOADS[args.workload]
    g = S.cube_scene(w["n_global"], w["seed"])
    gt = S.cube_scene(w["n_global"], w["seed"] + 1)
    cam = S.cube_camera(w["width"], w["height"])
    return g, gt, cam


def raster_cpu_baseline(args, threads=1, min_seconds=1.0):
    """The FP64 oracle's forward, L1 loss and backward of the whole config
    (no sampling), repeated for at least min_seconds."""
    from oracle import oracle as O
    O.build()
    g, gt, cam = raster_problem(args)
    x, xg = O.params_from(g), O.params_from(gt)
    plan = O.ViewPlan([cam], [(0, g.n)], 16, 16)
    tgt = O.render(xg, 0, plan)["views"][0]["image"]
    used = O.set_threads(threads)
    try:
        n, t0 = 0, time.perf_counter()
        while True:
            f = O.render(x, 0, plan)
            grad = O.l1(f["views"][0]["image"], tgt)[1]
            O.backward(x, 0, plan, f, [grad])
            n += 1
            if time.perf_counter() - t0 >= min_seconds:
                break
        dt = (time.perf_counter() - t0) / n
    finally:
        O.set_threads(1)
    return {"value": round(1.0 / dt, 3), "unit": "views/s", "cores": used, "kind": "oracle",
            "sample": f"the whole config (fwd + L1 + bwd of the view), {n} repetitions in {dt * n:.1f} s"}


def run_raster(args, dist, rank, world):
    """Plain rasteriser fwd + bwd of one view: project, bin_sort,
    rasterize_fwd, L1 loss, rasterize_bwd (compositing adjoint and the
    projection adjoint into a gradient buffer); one step = one view,
    replayed from a CUDA graph."""
    import torch
    from paper_2405_13943_b300 import _lib as L
    from paper_2405_13943_b300 import build as B
    from paper_2405_13943_b300 import dogs as D
    from paper_2405_13943_b300 import serve
    B.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    w = WORKLOADS[args.workload]
    g, gt, cam = raster_problem(args)
    xb = D.GaussianBuffer.from_synth(g)
    target = serve.render_views(D.GaussianBuffer.from_synth(gt), [cam]).image.clone()
    vb = D.ViewBatch([cam], [0, g.n], 16, 16)
    grads = xb.like()
    bg = (0.0, 0.0, 0.0)
    D.forward(xb, vb, bg)                     # sizes the instance capacity once
    tgt_dev = target.clone()

    def best_variant(call, fwd: bool):
        """The compositing variant (warps per tile, staged per thread) of the
        forward or the backward with the shortest time on this view."""
        best = None
        for w in (1, 2, 4, 8):
            for st in (1, 2):
                cur = [vb.plan.raster_warps, vb.plan.raster_stage, vb.plan.raster_warps_bwd, vb.plan.raster_stage_bwd]
                if fwd:
                    cur[0], cur[1] = w, st
                else:
                    cur[2], cur[3] = w, st
                D.apply_variant(vb.plan, cur)
                for _ in range(3):
                    call()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(20):
                    call()
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1)
                if best is None or t < best[0]:
                    best = (t, list(cur))
        D.apply_variant(vb.plan, best[1])

    D.dg_loss_l1(vb, tgt_dev, 1.0)
    best_variant(lambda: D.dg_rasterize_fwd(vb, bg), True)
    best_variant(lambda: D.dg_rasterize_bwd(vb, xb, grads, bg=bg), False)

    def step():
        D.dg_project(xb, vb)
        D.dg_bin_sort(vb)
        D.dg_rasterize_fwd(vb, bg)
        D.dg_loss_l1(vb, tgt_dev, 1.0)
        D.dg_rasterize_bwd(vb, xb, grads, bg=bg)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    if int(vb.status.item()) & L.DG_STATUS_CAPACITY:
        raise RuntimeError("instance capacity overflow")
    reps = max(args.steps, 1)
    clocks = ClockSampler(local)
    clocks.wait_first()
    barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop()
    ms = max_over_ranks(dist, e0.elapsed_time(e1) / reps)
    # per call, eager, CUDA events
    calls = [("project", lambda: D.dg_project(xb, vb)), ("bin_sort", lambda: D.dg_bin_sort(vb)),
             ("rasterize_fwd", lambda: D.dg_rasterize_fwd(vb, bg)),
             ("loss", lambda: D.dg_loss_l1(vb, tgt_dev, 1.0)),
             ("rasterize_bwd", lambda: D.dg_rasterize_bwd(vb, xb, grads, bg=bg))]
    acc = {n: 0.0 for n, _ in calls}
    n_eager = 50
    l0 = L.lib().dg_launch_count()
    for _ in range(n_eager):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)]
        torch.cuda._sleep(200_000)     # the first call queued before ev[0] is reached
        ev[0].record()
        for k, (n, fn) in enumerate(calls):
            fn()
            ev[k + 1].record()
        torch.cuda.synchronize()
        for k, (n, _) in enumerate(calls):
            acc[n] += ev[k].elapsed_time(ev[k + 1]) / n_eager
    launches_per_step = (L.lib().dg_launch_count() - l0) / n_eager
    c = D.dg_rasterize_count(vb, bg).cpu().numpy()
    seen, used = float(c[0]), float(c[1])
    D.dg_rasterize_fwd(vb, bg)
    pairs = float(vb.last[:vb.n_pixels].sum(dtype=torch.int64))
    fp32 = measure_fp32_peak(local)
    work = {"rasterize_fwd": seen * FLOPS_EVAL + used * FLOPS_FWD_USED,
            "rasterize_bwd": pairs * FLOPS_EVAL + used * FLOPS_BWD_USED}
    kern = {n: {"ms": round(acc[n], 4)} for n in acc}
    for n, fl in work.items():
        tf = fl / (acc[n] * 1e-3) / 1e12
        kern[n].update({"tflops": round(tf, 3), "frac_fp32": round(tf / fp32["tflops"], 4)})
    dom = max(work, key=lambda n: acc[n])
    roofline = {"bound": "alu", "kernel": dom, "achieved": kern[dom]["tflops"], "peak": fp32["tflops"],
                "unit": "TFLOP/s", "frac": kern[dom]["frac_fp32"],
                "peak_source": f"measured FP32 FMA probe ({fp32['how']})", "traffic": None,
                "flops_per_launch": int(work[dom]), "pairs_composited": int(used),
                "note": f"{vb.n_tiles} tiles: one CTA per tile leaves most of the {torch.cuda.get_device_properties(local).multi_processor_count} SMs idle; the view is latency-bound"}
    # end to end: the target crosses from pinned host memory and the loss comes back every step
    host_t = target.cpu().pin_memory()
    host_loss = [torch.zeros(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for i in range(reps):
        tgt_dev.copy_(host_t, non_blocking=True)
        graph.replay()
        host_loss[i % 2].copy_(vb.loss[:1], non_blocking=True)
        done[i % 2].record()
        if i > 0:
            done[(i - 1) % 2].synchronize()
            losses.append(float(host_loss[(i - 1) % 2][0]))
    done[(reps - 1) % 2].synchronize()
    losses.append(float(host_loss[(reps - 1) % 2][0]))
    e2e_ms = max_over_ranks(dist, (time.perf_counter() - t0) / reps * 1e3)
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        one = raster_cpu_baseline(args, 1)
        cpu = dict(raster_cpu_baseline(args, host_cores()), single_core={k: one[k] for k in ("value", "cores")})
    if rank == 0:
        print(json.dumps({
            "metric": metric_of(args), "value": round(world * 1e3 / ms, 2), "unit": "views/s", "n_gpus": world,
            "steps": reps, "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (cube law, seeded)",
            "config": {"workload": workload_name(args, None), "tile": "16x16", "cuda_graph": True,
                       "raster_variant": {"fwd": [vb.plan.raster_warps, vb.plan.raster_stage],
                                          "bwd": [vb.plan.raster_warps_bwd, vb.plan.raster_stage_bwd]},
                       "instances": int(vb.count.item()),
                       "l2": "working set < L2: replays run warm, as a one-view training loop would"},
            "kernels_ms": kern, "roofline": roofline, "fp32_peak": fp32, "clocks": clk,
            "gpu_launches": int(launches_per_step * reps),
            "e2e": {"value": round(world * 1e3 / e2e_ms, 2), "unit": "views/s", "ms_per_step": round(e2e_ms, 4),
                    "h2d_bytes_per_step": int(host_t.numel() * 4), "d2h_bytes_per_step": 8,
                    "loss_last": losses[-1]},
            "cpu_baseline": cpu}))


def run_e2e(tr, args, dist, targets8, cons=True, cons_values=(True,)):
    """Same iterations through the trainer with its targets in pinned host
    memory: every step's target images cross host -> device (copied one step
    ahead on a side stream while the previous step computes) and every step's
    per-view losses are copied back and read on the host (step t's while step
    t + 1 runs), all inside the timed region."""
    import torch
    host_t = [t.cpu().pin_memory() for t in targets8]
    tr.use_host_targets(host_t)
    for _ in range(2):
        tr.step(consensus=cons)
        tr.last_loss()
    tr.prepare_graphs(cons_values)
    torch.cuda.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    losses = []
    tr.step(consensus=cons)
    for _ in range(args.steps - 1):
        tr.step(consensus=cons)
        losses.append(float(tr.loss_of(tr.t - 2).sum()))    # the previous step's losses, on the host
    losses.append(float(tr.last_loss().sum()))
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / args.steps
    ms = max_over_ranks(dist, wall * 1e3)
    world = 1 if dist is None else dist.get_world_size()
    assert len(losses) == args.steps
    return {"value": round(world * 1e3 / ms, 4), "unit": "iter/s", "ms_per_step": round(ms, 3),
            "h2d_bytes_per_step": tr.h2d_bytes_per_step(), "d2h_bytes_per_step": int(tr.host_loss[0].numel() * 8),
            "loss_last": losses[-1],
            "timing": "host wall clock per step; each step's target (8-bit images) uploaded from pinned host "
                      "memory one step ahead on a copy stream and widened on the device, each step's losses "
                      "copied back and read on the host while the next step runs"}


def densify_probe(tr, wl, D):
    """The statistic over a few eager iterations (its kernel timed by CUDA
    events), then one densification of the 6M-Gaussian state timed on the
    host clock: decisions, emission, the layout rebuild and the state moved."""
    import torch
    from paper_2405_13943_b300 import densify as DZ
    cfg = DZ.DensifyConfig(interval=tr.intv * 10007, start=0, until=1 << 30)   # due only when called below
    tr.densify_cfg = cfg
    tr.extent = DZ.scene_extent([c for vs in tr.view_sets for c in vs])
    tr.dstats = torch.zeros(2 * tr.split.n_copies, dtype=torch.float32, device=tr.z.data.device)
    ms, walls, parts = [], [], []
    for rep in range(2):            # the first densification also pays one-time set-up (allocator, RNG)
        for _ in range(4):
            tr.step(consensus=True, graph=False)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            D.dg_densify_stats(tr.vb, tr.dstats)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t0 = time.perf_counter()
        out = DZ.densify(tr, cfg, tr.extent, tr.t)
        torch.cuda.synchronize()
        walls.append(time.perf_counter() - t0)
        parts.append(out.get("seconds"))
        tr.dstats.zero_()
    return {"stats_kernel_ms": round(float(np.median(ms)), 4), "densify_s": round(walls[-1], 3),
            "densify_s_first": round(walls[0], 3), "seconds_first": parts[0],
            "extent_m": round(tr.extent, 1), **{k: v for k, v in out.items()},
            "rule": "3DGS adaptive density control on the global model after a consensus: grad 2e-4, "
                    "percent_dense 0.01, min_opacity 0.005 (statistics of 4 iterations)"}


def run_serving(z, args, tile):
    from paper_2405_13943_b300 import serve
    from paper_2405_13943_b300 import synth as S
    rate = 200.0
    arr = S.poisson_arrivals(1005, rate, args.serve_seconds)
    res = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]
    cams = S.random_pose_cameras(1006, len(arr), res, [0.4, 0.3, 0.2, 0.1])
    srv = serve.RenderServer(z, budget_bytes=20e9, tile=tile)
    # warm the path and size the instance capacity on sample poses of the
    # same law (not the requests themselves)
    ipp = srv.calibrate(S.random_pose_cameras(1007, 64, res, [0.4, 0.3, 0.2, 0.1]))
    out = srv.run(cams, arr)
    return {"p50_ms": round(out["p50_ms"], 3), "p99_ms": round(out["p99_ms"], 3),
            "views_per_s": round(out["views_per_s"], 2), "requests": out["requests"], "rate_hz": rate,
            "duration_s": args.serve_seconds, "budget_gb": 20, "max_inflight_batches": out["max_inflight_batches"],
            "capacity_retries": out["capacity_retries"], "instances_per_pixel_capacity": round(ipp, 3),
            "slots": out["slots"], "resident_gb": round(out["resident_gb"], 2),
            "free_hbm_gb_at_provision": round(out["free_hbm_gb_at_provision"], 1),
            "mix": "640x480/1280x720/1920x1080/3840x2160 at 0.4/0.3/0.2/0.1, Poisson 200/s"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(wl, args, frac=64, threads=1):
    """The FP64 oracle, as it stands, on a bounded sample of one iteration:
    1/frac of every block's copies (seeded), the full-size views and loss, on
    `threads` host threads.  Full-iteration time is extrapolated as
    loss + frac x (the rest); the compositing part of that is an upper bound
    (denser scenes terminate pixels earlier), so the iter/s is a lower bound."""
    from oracle import oracle as O
    O.build()
    used = O.set_threads(threads)
    try:
        sp = wl.split
        rng = np.random.default_rng(0)
        keep = [np.sort(rng.choice(np.arange(sp.blk_off[k], sp.blk_off[k + 1]),
                                   max(1, (sp.blk_off[k + 1] - sp.blk_off[k]) // frac), replace=False))
                for k in range(sp.K)]
        cid = np.concatenate(keep)
        x = O.params_from(wl.z0.subset(sp.copy_gid[cid]))
        off = np.cumsum([0] + [len(i) for i in keep])
        rows = [(off[c.block], off[c.block + 1]) for c in wl.views[0]]
        plan = O.ViewPlan(wl.views[0], rows, 16, 16)
        tgt = [np.zeros((3, c.height, c.width)) for c in plan.cams]
        t0 = time.perf_counter()
        f = O.render(x, 3, plan)
        t1 = time.perf_counter()
        if args.loss == "dssim":
            grads = [O.dssim_loss(v["image"], t)[1] for v, t in zip(f["views"], tgt)]
        else:
            grads = [O.l1(v["image"], t)[1] for v, t in zip(f["views"], tgt)]
        t2 = time.perf_counter()
        b = O.backward(x, 3, plan, f, grads)
        m = np.zeros_like(x); v = np.zeros_like(x)
        shared = sp.copy_shared()[cid]
        gid = np.arange(x.shape[0], dtype=np.int32)
        z = x.copy(); u = np.zeros_like(x)
        O.adam_admm_step(x, np.ascontiguousarray(b["dparams"]), m, v, z, u, gid, shared, [1e-3] * 5,
                         [1.6e-4, 1e-3, 5e-3, 2.5e-3, 1.25e-4, 5e-2], 3)
        g_off = np.arange(x.shape[0] + 1, dtype=np.int64)
        O.consensus(x, u, z, g_off, gid, 3)
        t3 = time.perf_counter()
    finally:
        O.set_threads(1)
    rest = (t1 - t0) + (t3 - t2)
    full = (t2 - t1) + frac * rest
    return {"value": round(1.0 / full, 6), "unit": "iter/s", "cores": used, "kind": "oracle",
            "sample": f"1/{frac} of each block's copies ({x.shape[0]}), {len(plan.cams)} full-size views and loss; "
                      f"measured {t3 - t0:.1f} s, extrapolated {full:.1f} s per iteration",
            "sample_seconds": round(t3 - t0, 2)}


def cpu_baselines(wl, args):
    """The oracle timed single-threaded and on all of the host's cores."""
    frac = WORKLOADS[args.workload]["oracle_frac"]
    one = cpu_baseline(wl, args, frac, threads=1)
    allc = cpu_baseline(wl, args, frac, threads=host_cores())
    return dict(allc, single_core={k: one[k] for k in ("value", "cores", "sample_seconds")})


def workload_name(args, wl) -> str:
    w = WORKLOADS[args.workload]
    if w["kind"] == "raster":
        return (f"plain rasteriser fwd+bwd, one view: {w['n_global']} Gaussians in [-1,1]^3, SH0, "
                f"{w['width']}x{w['height']}, L1")
    cams = {"aerial": "aerial 45 deg", "grid": "grid cameras pitch 45-90 deg",
            "street": "street level"}[w.get("cameras", "aerial")]
    cons = {None: "no consensus", 1: "consensus every step"}.get(w["intv"], f"consensus every {w['intv']}")
    if wl.split.K == 1:
        return (f"single-model 3DGS, {w['n_global']} Gaussians SH3, V={len(wl.views[0])} x "
                f"{w['width']}x{w['height']} {cams}, Adam, {cons}")
    return (f"DOGS K={wl.split.K} batched, {w['n_global']} Gaussians SH3, {wl.split.n_copies} copies, "
            f"{round(100 * w['shared'])}% shared, V={len(wl.views[0])} x {w['width']}x{w['height']} {cams}, {cons}")


def metric_of(args) -> str:
    """The headline workload carries the benchmark's metric; the others name
    their own (same unit: training iterations per second, or views per
    second for the rasteriser alone)."""
    if args.workload == "large":
        return METRIC
    w = WORKLOADS[args.workload]
    if w["kind"] == "raster":
        return f"rasteriser fwd+bwd views/s, {w['n_global']} Gaussians {w['width']}x{w['height']}, 1 B300"
    what = "fwd+bwd+Adam" if w["intv"] is None else "fwd+bwd+ADMM"
    return f"train iters/s ({what}), {args.workload}: {w['n_global']} Gaussians, 1 B300"


def run_reference(args, dist, rank, world):
    """The oracle as the reference arm: each step = the bounded sample of one
    iteration, reported on the full-iteration scale (rank 0 only)."""
    if rank != 0:
        return
    if WORKLOADS[args.workload]["kind"] == "raster":
        cores = host_cores()
        vals = [raster_cpu_baseline(args, cores) for _ in range(max(1, min(args.steps, 3)))]
        v = float(np.mean([c["value"] for c in vals]))
        print(json.dumps({"impl": "reference", "metric": metric_of(args), "value": round(v, 3), "unit": "views/s",
                          "n_gpus": world, "steps": len(vals), "warmup": 0, "ms_per_step": round(1e3 / v, 3),
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic (cube law, seeded)", "config": {"workload": workload_name(args, None)},
                          "cpu_baseline": {"value": round(v, 3), "unit": "views/s", "cores": vals[0]["cores"],
                                           "kind": "oracle", "sample": vals[0]["sample"]},
                          "e2e": {"value": round(v, 3), "unit": "views/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return
    wl = build_workload(args.workload, getattr(args, "views_per_block", 1))
    steps = max(1, min(args.steps, 3))
    vals = []
    frac, cores = WORKLOADS[args.workload]["oracle_frac"], host_cores()
    for _ in range(min(args.warmup, 1)):
        cpu_baseline(wl, args, frac, cores)
    for _ in range(steps):
        vals.append(cpu_baseline(wl, args, frac, cores))
    v = float(np.mean([c["value"] for c in vals]))
    line = {"impl": "reference", "metric": metric_of(args), "value": round(v, 6), "unit": "iter/s", "n_gpus": world,
            "steps": steps, "warmup": min(args.warmup, 1), "ms_per_step": round(1e3 / v, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (city-law aerial scene, seeded)",
            "config": {"workload": workload_name(args, wl), "blocks": wl.split.K, "copies": wl.split.n_copies,
                       "views_per_step": len(wl.views[0]), "timing": "bounded sample per step, extrapolated"},
            "cpu_baseline": {"value": round(v, 6), "unit": "iter/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": round(v, 6), "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    dist, rank, world = dist_setup()
    raster = WORKLOADS[args.workload]["kind"] == "raster"
    if args.impl == "reference":
        run_reference(args, dist, rank, world)
    elif raster:
        run_raster(args, dist, rank, world)
    else:
        run_ours(args, dist, rank, world)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
