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
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "medium", "small"])
    ap.add_argument("--views-per-block", type=int, default=1,
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
                    help="CTAs per SM of the x-step part that runs beside compositing (0: one per group of copies)")
    ap.add_argument("--no-overlap", action="store_true", help="run that x-step part inline on the main stream")
    ap.add_argument("--variant", default=None,
                    help="compositing variant W,S[,Wb,Sb] (warps per tile, staged per thread; backward)")
    ap.add_argument("--loss", default="dssim", choices=["dssim", "l1"])
    ap.add_argument("--profile", action="store_true", help="setup + warmup + a few eager steps only (for ncu)")
    return ap.parse_args()


WORKLOADS = {
    "large": dict(n_global=6_000_000, cols=2, rows=4, shared=0.10, seed=1004, width=1920, height=1080, pool=4),
    "small": dict(n_global=200_000, cols=2, rows=2, shared=0.05, seed=1003, width=640, height=480, pool=2),
    # same law and views as "large" at 1/6 of the Gaussians: a profiling case of a few GB, above L2
    "medium": dict(n_global=1_000_000, cols=2, rows=4, shared=0.10, seed=1004, width=1920, height=1080, pool=2),
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
                           views_per_step=views_per_block, pool=w["pool"], width=w["width"], height=w["height"])


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


def algorithmic_bytes(tr, vb_rect_visible: int, n_visible_copies: int, active_groups=None, zfuse=False):
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
        # every copy: mean/opacity read (16 B) + rect (8 B); visible records: rest of the params (224 B)
        # + record (48 B)
        "project": n_c * 24 + n_visible_copies * 224 + vb_rect_visible * 48,
    }
    if active_groups is not None:
        # split x-step: part 2 over the groups of 128 copies with a kept record, part 1 over the
        # others (plus the 8-byte rectangle of each of its copies, read to find them)
        act = np.repeat(active_groups, 128)[:n_c]
        sh = sp.copy_shared().astype(bool)
        na, nsa = int(act.sum()), int((act & sh).sum())
        out["xstep"] = na * P * 24 + nsa * P * 4 + n_visible_copies * 56
        out["xstep_idle"] = (n_c - na) * (P * 24 + 8) + (n_sc - nsa) * P * 4
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
    tile = tuple(int(v) for v in args.tile.split("x"))
    t_setup = time.time()
    wl = build_workload(args.workload, args.views_per_block)
    z0 = D.GaussianBuffer.from_synth(wl.z0)
    gt = D.GaussianBuffer.from_synth(wl.gt)
    targets, targets8 = render_targets(gt, wl.views, tile)
    del gt
    if args.variant:
        D.set_raster_variant(*[int(v) for v in args.variant.split(",")])
    tr = T.DogsTrainer(wl.split, z0, wl.views, targets, rho=(1e-3,) * 5, tile=tile, loss=args.loss,
                       overlap=not args.no_overlap)
    tr.idle_ctas_per_sm = args.idle_ctas
    m_max = tr.calibrate_capacity()
    tuned = None
    if not args.no_autotune and not args.profile and not args.variant:
        from paper_2405_13943_b300 import autotune
        tuned = autotune.tune(tr, use_cache=False)
        tile = tr.tile
        m_max = tr.calibrate_capacity()
    torch.cuda.synchronize()
    setup_s = time.time() - t_setup

    for _ in range(args.warmup):
        tr.step(consensus=True)
    torch.cuda.synchronize()
    if tr.overflowed():
        raise RuntimeError("instance capacity overflow during warmup")
    if args.profile:
        # two eager iterations inside an NVTX range "dogs_step" (ncu --nvtx-include dogs_step/)
        torch.cuda.nvtx.range_push("dogs_step")
        for _ in range(2):
            tr.step(consensus=True, graph=False)
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
    e0.record()
    for _ in range(args.steps):
        tr.step(consensus=True)
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
    if split:       # the part that the graph runs on a side stream, timed here in sequence
        calls.append(("xstep_idle", lambda: D.dg_xstep_part(1, vb, *xs_args, step=1, dev_step=tr.dev_step,
                                                            **zargs)))
    calls += [("bin_sort", lambda: D.dg_bin_sort(vb)),
              ("rasterize_fwd", lambda: D.dg_rasterize_fwd(vb, tr.bg)),
              ("loss", lambda: tr._loss(tr.targets[tr.t % len(tr.view_sets)]))]
    if fused:       # compositing adjoint, then projection adjoint + x-step fused
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
    alg = algorithmic_bytes(tr, vis_rec, vis_rec, active_groups if split else None, zf)
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
    props = torch.cuda.get_device_properties(local)
    sm_max = float(clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2032.0))
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
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
                    "peak_source": f"FP32 from unit counts: {props.multi_processor_count} SMs x 128 lanes x 2 x "
                                   f"{sm_max:.0f} MHz",
                    "traffic": traffic, "flops_per_launch": int(work[dom][0]), **work[dom][1]}
    else:
        achieved = alg[dom] / (acc[dom] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm_peak,
                    "unit": "GB/s", "frac": round(achieved / hbm_peak, 3), "peak_source": f"{peak_src} hbm_gbs",
                    "traffic": traffic, "algorithmic_bytes": int(alg[dom])}

    # ---- end to end through host buffers ---------------------------------------------------
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(tr, args, dist, targets8)

    # ---- sequential per-block comparator -----------------------------------------------------
    comparator = None
    if not args.no_seq:
        del_bufs = None
        seq = T.SequentialTrainer(wl.split, z0.clone(), wl.views, targets, rho=(1e-3,) * 5, tile=tile,
                                  loss=args.loss)
        seq.calibrate_capacity()
        for _ in range(2):
            seq.step(consensus=True)
        torch.cuda.synchronize()
        n_seq = max(3, args.steps // 4)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(n_seq):
            seq.step(consensus=True)
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
    if not args.no_serve and args.serve_seconds > 0:
        render = run_serving(tr.z, args, tile)

    # ---- CPU baseline (oracle, bounded sample) --------------------------------------------------------
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline(wl, args)

    # ---- one densification of the trained state (off the per-iteration path: every 200 iterations) --
    densify = None
    if not args.no_densify_probe:
        densify = densify_probe(tr, wl, D)

    value = world * 1e3 / ms
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "iter/s", "n_gpus": world, "steps": args.steps,
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
                                     "variants_per_tile": len(tuned["candidates"][0]["variants"])}),
                       "loss": "0.8 L1 + 0.2 D-SSIM" if args.loss == "dssim" else "L1",
                       "consensus_every_timed_step": True, "cuda_graph": True,
                       "xstep_split": (None if not split else
                                       {"idle_groups_on_side_stream": round(1.0 - float(active_groups.mean()), 3),
                                        "side_ctas_per_sm": tr.idle_ctas_per_sm}),
                       "unshared_z_stored_by_xstep": bool(zf),
                       "l2": "working set > L2 (no flush needed)", "instances_per_step": instances,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "setup_s": round(setup_s, 1)},
            "kernels_ms": kern, "eager_ms_per_step": round(eager_ms, 3),
            "roofline": roofline, "clocks": clk, "gpu_launches": int(launches_per_step * args.steps),
            "e2e": e2e, "comparator": comparator, "render": render, "cpu_baseline": cpu, "densify": densify,
        }
        print(json.dumps(line))


def run_e2e(tr, args, dist, targets8):
    """Same iterations through the trainer with its targets in pinned host
    memory: every step's target images cross host -> device (copied one step
    ahead on a side stream while the previous step computes) and every step's
    per-view losses are copied back and read on the host (step t's while step
    t + 1 runs), all inside the timed region."""
    import torch
    host_t = [t.cpu().pin_memory() for t in targets8]
    tr.use_host_targets(host_t)
    for _ in range(2):
        tr.step(consensus=True)
        tr.last_loss()
    torch.cuda.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    losses = []
    tr.step(consensus=True)
    for _ in range(args.steps - 1):
        tr.step(consensus=True)
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
    ms = []
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
    wall = time.perf_counter() - t0
    return {"stats_kernel_ms": round(float(np.median(ms)), 4), "densify_s": round(wall, 3),
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
            "mix": "640x480/1280x720/1920x1080/3840x2160 at 0.4/0.3/0.2/0.1, Poisson 200/s"}


def cpu_baseline(wl, args, frac=64):
    """The FP64 oracle, as it stands, on a bounded sample of one iteration:
    1/frac of every block's copies (seeded), the full-size views and loss.
    Full-iteration time is extrapolated as loss + frac x (the rest); the
    compositing part of that is an upper bound (denser scenes terminate
    pixels earlier), so the iter/s is a lower bound."""
    from oracle import oracle as O
    O.build()
    sp = wl.split
    rng = np.random.default_rng(0)
    keep = [np.sort(rng.choice(np.arange(sp.blk_off[k], sp.blk_off[k + 1]),
                               max(1, (sp.blk_off[k + 1] - sp.blk_off[k]) // frac), replace=False))
            for k in range(sp.K)]
    cid = np.concatenate(keep)
    x = O.params_from(wl.z0.subset(sp.copy_gid[cid]))
    off = np.cumsum([0] + [len(i) for i in keep])
    rows = [(off[k], off[k + 1]) for k in range(sp.K)]
    plan = O.ViewPlan(wl.views[0], rows, 16, 16)
    tgt = [np.zeros((3, c.height, c.width)) for c in plan.cams]
    t0 = time.perf_counter()
    f = O.render(x, 3, plan)
    t1 = time.perf_counter()
    grads = [O.dssim_loss(v["image"], t)[1] for v, t in zip(f["views"], tgt)]
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
    rest = (t1 - t0) + (t3 - t2)
    full = (t2 - t1) + frac * rest
    return {"value": round(1.0 / full, 6), "unit": "iter/s", "cores": 1, "kind": "oracle",
            "sample": f"1/{frac} of each block's copies ({x.shape[0]}), {len(plan.cams)} full-size views and loss; "
                      f"measured {t3 - t0:.1f} s, extrapolated {full:.1f} s per iteration",
            "sample_seconds": round(t3 - t0, 2)}


def workload_name(args, wl) -> str:
    w = WORKLOADS[args.workload]
    return (f"DOGS K={wl.split.K} batched, {w['n_global']} Gaussians SH3, {wl.split.n_copies} copies, 10% shared, "
            f"V={len(wl.views[0])} x {w['width']}x{w['height']}")


def run_reference(args, dist, rank, world):
    """The oracle as the reference arm: each step = the bounded sample of one
    iteration, reported on the full-iteration scale (rank 0 only)."""
    if rank != 0:
        return
    wl = build_workload(args.workload, getattr(args, "views_per_block", 1))
    steps = max(1, min(args.steps, 3))
    vals = []
    for _ in range(min(args.warmup, 1)):
        cpu_baseline(wl, args)
    for _ in range(steps):
        vals.append(cpu_baseline(wl, args))
    v = float(np.mean([c["value"] for c in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "iter/s", "n_gpus": world,
            "steps": steps, "warmup": min(args.warmup, 1), "ms_per_step": round(1e3 / v, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (city-law aerial scene, seeded)",
            "config": {"workload": workload_name(args, wl), "blocks": wl.split.K, "copies": wl.split.n_copies,
                       "views_per_step": len(wl.views[0]), "timing": "bounded sample per step, extrapolated"},
            "cpu_baseline": {"value": round(v, 6), "unit": "iter/s", "cores": 1, "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": round(v, 6), "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    dist, rank, world = dist_setup()
    if args.impl == "reference":
        run_reference(args, dist, rank, world)
    else:
        run_ours(args, dist, rank, world)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
