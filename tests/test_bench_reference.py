"""bench.py's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys the benchmark contract asks of it, on the small
workload; and both arms name a workload with the same string."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_its_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "small"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "iter/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("DOGS K=4 batched, 200000 Gaussians")


def test_both_arms_name_the_workload_alike():
    sys.path.insert(0, ROOT)
    import bench
    import types
    wl = bench.build_workload("small")
    name = bench.workload_name(types.SimpleNamespace(workload="small"), wl)
    assert name == (f"DOGS K={wl.split.K} batched, 200000 Gaussians SH3, {wl.split.n_copies} copies, 5% shared, "
                    f"V={len(wl.views[0])} x 640x480 aerial 45 deg, consensus every step")


def test_every_workload_has_its_metric_and_consensus_rule():
    sys.path.insert(0, ROOT)
    import bench
    import types
    for name, w in bench.WORKLOADS.items():
        args = types.SimpleNamespace(workload=name)
        m = bench.metric_of(args)
        assert (m == bench.METRIC) == (name == "large"), name
        if w["kind"] == "dogs":
            c = bench.consensus_arg(w)
            assert c is (False if w["intv"] is None else True if w["intv"] == 1 else None), name


def test_reference_arm_of_the_rasteriser_config():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--workload", "raster4k"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    assert d["impl"] == "reference" and d["unit"] == "views/s" and d["value"] > 0
    assert d["cpu_baseline"]["cores"] >= 1 and d["e2e"]["h2d_bytes_per_step"] == 0
