"""The autotuner's choices on the host, with its three timing functions
replaced by fixed tables (no GPU): per tile shape the forward and the
backward variants are chosen from their own kernel times, independently;
the tile shape by its full-iteration time with those variants; the side
stream's form by the best of its two alternated timings, taken with the
consensus setting the caller gives; and the result is cached per workload
signature and applied again from the cache."""
import json
import types

import pytest

from paper_2405_13943_b300 import autotune as A

TILES = ((16, 16), (32, 8))
# (forward ms, backward ms) per tile shape and (warps, staged)
KT = {
    (16, 16): {(1, 1): (1.0, 2.0), (2, 1): (0.8, 2.4), (1, 2): (1.1, 1.9), (2, 2): (0.9, 2.2)},
    (32, 8): {(1, 1): (0.7, 2.6), (2, 1): (0.9, 2.5), (1, 2): (0.75, 2.55), (2, 2): (1.0, 2.7)},
}
STEP_MS = {(16, 16): 5.0, (32, 8): 5.3}


class FakeTrainer:
    def __init__(self):
        self.tile, self.variant, self.idle_mode = (16, 16), None, "grid"
        self.graphs = {"stale": object()}
        self.view_sets = [[types.SimpleNamespace(width=64, height=48)]]
        self.split = types.SimpleNamespace(K=2, n_copies=1000)
        self.x = types.SimpleNamespace(deg=3)
        self.log = []

    def set_tile(self, t):
        self.tile = tuple(t)

    def set_variant(self, *v):
        self.variant = v

    def _split_xstep(self):
        return True


@pytest.fixture
def fakes(monkeypatch, tmp_path):
    seq = {"stream": [5.2, 4.7], "grid": [4.9, 4.95]}
    seen = []

    def kernel_times(tr, steps):
        return KT[tr.tile][tr.variant[:2]]

    def time_steps(tr, steps):
        return STEP_MS[tr.tile]

    def time_graph_steps(tr, steps, consensus=False):
        seen.append((tr.idle_mode, consensus))
        return seq[tr.idle_mode].pop(0)

    monkeypatch.setattr(A, "_kernel_times", kernel_times)
    monkeypatch.setattr(A, "_time_steps", time_steps)
    monkeypatch.setattr(A, "_time_graph_steps", time_graph_steps)
    monkeypatch.setattr(A.D, "set_raster_variant", lambda *v: None)
    monkeypatch.setattr(A, "CACHE", str(tmp_path / "cache.json"))
    return seen


def test_choices_and_cache(fakes):
    tr = FakeTrainer()
    out = A.tune(tr, tiles=TILES, warps=(1, 2), stages=(1, 2), steps=1, use_cache=True, consensus=True)
    # 16x16: forward best (2, 1) at 0.8, backward best (1, 2) at 1.9; the step time picks 16x16
    assert out["tile"] == [16, 16] and out["fwd"] == [2, 1] and out["bwd"] == [1, 2]
    assert tr.tile == (16, 16) and tr.variant == (2, 1, 1, 2)
    # 32x8's own choice is recorded too: forward (1, 1) at 0.7, backward (2, 1) at 2.5
    c32 = [r for r in out["candidates"] if r["tile"] == [32, 8]][0]
    assert c32["fwd"] == [1, 1] and c32["bwd"] == [2, 1]
    # alternated, twice each, with the consensus passed through; best of each: stream 4.7, grid 4.9
    assert fakes == [("stream", True), ("grid", True), ("stream", True), ("grid", True)]
    assert out["idle_modes"] == {"stream": 4.7, "grid": 4.9}
    assert out["idle_mode"] == "stream" == tr.idle_mode
    assert not tr.graphs
    cached = json.load(open(A.CACHE))[A.signature(tr)]
    assert cached == {"tile": [16, 16], "fwd": [2, 1], "bwd": [1, 2], "ms": 5.0, "idle_mode": "stream"}
    # a second trainer of the same signature takes the cached choice without timing
    tr2 = FakeTrainer()
    tr2.tile = (32, 8)
    n_before = len(fakes)
    again = A.tune(tr2, tiles=TILES, warps=(1, 2), stages=(1, 2), steps=1, use_cache=True)
    assert again["cached"] and len(fakes) == n_before
    assert tr2.tile == (16, 16) and tr2.variant == (2, 1, 1, 2) and tr2.idle_mode == "stream"


def test_one_idle_form_is_not_timed(fakes):
    tr = FakeTrainer()
    out = A.tune(tr, tiles=TILES[:1], warps=(1, 2), stages=(1,), steps=1, use_cache=False, idle_modes=("grid",))
    assert out["idle_modes"] is None and fakes == []
    assert tr.idle_mode == "grid"
