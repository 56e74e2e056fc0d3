"""Checkpoint format on the host: a round trip restores every buffer bit for
bit with t, rho and the adaptive-penalty state, the anchors are rebuilt, and
a damaged, truncated or mismatched file is refused before any buffer is
written."""
import json
import os
import struct

import numpy as np
import pytest
import torch

from paper_2405_13943_b300 import checkpoint as CK
from paper_2405_13943_b300 import dogs as D
from paper_2405_13943_b300 import synth as S
from paper_2405_13943_b300.admm import AdaptivePenalty


class HostRun:
    """The state a DogsTrainer checkpoints, on host buffers."""

    def __init__(self, seed, adaptive=True, intv=100, split_seed=1):
        rng = np.random.default_rng(split_seed)
        xy = rng.uniform(0, 100, (500, 2))
        self.split, _ = S.block_split(xy, 2, 2, [0.25] * 4, 0.1)
        nc, ng = self.split.n_copies, 500
        self.z = D.GaussianBuffer(ng, 1, "cpu")
        for name in ("x", "u", "m", "v", "anchor"):
            setattr(self, name, D.GaussianBuffer(nc, 1, "cpu"))
        g = torch.Generator().manual_seed(seed)
        for name in ("z", "x", "u", "m", "v"):
            getattr(self, name).data.copy_(torch.randn(getattr(self, name).data.numel(), generator=g))
        self.t, self.rho = 1234, [1e4, 2e4, 1e4, 1e3, 5e3]
        self.lr, self.alpha, self.intv = [1.6e-4, 1e-3, 5e-3, 2.5e-3, 1.25e-4, 5e-2], 1.6, intv
        self.loss_kind, self.w_l1, self.w_ssim, self.bg = "dssim", 0.8, 0.2, (0.0, 0.0, 0.0)
        self.adaptive = AdaptivePenalty(self.rho, mu=8.0, freeze_after=3000) if adaptive else None
        self.graphs = {"stale": 1}
        self.anchor_rebuilt = 0

    def refresh_anchor(self):
        self.anchor_rebuilt += 1


def test_round_trip_is_bit_exact(tmp_path):
    a = HostRun(1)
    p = str(tmp_path / "run.ckpt")
    CK.save(a, p)
    assert not os.path.exists(p + ".tmp")
    b = HostRun(2)
    hdr = CK.load(b, p)
    for name in ("z", "x", "u", "m", "v"):
        assert torch.equal(getattr(a, name).data.view(torch.int32), getattr(b, name).data.view(torch.int32))
    assert (b.t, b.rho) == (1234, a.rho)
    assert b.adaptive.rho == a.adaptive.rho and b.adaptive.mu == 8.0 and b.adaptive.freeze_after == 3000
    assert b.anchor_rebuilt == 1 and b.graphs == {}
    assert hdr["data_start"] % CK.ALIGN == 0
    assert all(e["offset"] % CK.ALIGN == 0 for e in hdr["buffers"])


def test_nan_and_negative_zero_survive(tmp_path):
    a = HostRun(3)
    a.m.data[:4] = torch.tensor([float("nan"), -0.0, float("inf"), 1e-45])
    p = str(tmp_path / "odd.ckpt")
    CK.save(a, p)
    b = HostRun(4)
    CK.load(b, p)
    assert torch.equal(a.m.data.view(torch.int32), b.m.data.view(torch.int32))


def _corrupt(path, at, byte):
    with open(path, "r+b") as f:
        f.seek(at)
        old = f.read(1)
        f.seek(at)
        f.write(bytes([old[0] ^ byte]))


def test_damage_is_refused_before_writing(tmp_path):
    a = HostRun(5)
    p = str(tmp_path / "bad.ckpt")
    CK.save(a, p)
    hdr = CK.read_header(p)
    e = hdr["buffers"][3]
    _corrupt(p, hdr["data_start"] + e["offset"] + 17, 0x10)
    b = HostRun(6)
    before = {n: getattr(b, n).data.clone() for n in ("z", "x", "u", "m", "v")}
    with pytest.raises(CK.CheckpointError, match="CRC"):
        CK.load(b, p)
    for n, t in before.items():
        assert torch.equal(getattr(b, n).data, t)          # nothing overwritten
    assert b.t == 1234 and b.anchor_rebuilt == 0


def test_truncated_wrong_split_wrong_config(tmp_path):
    a = HostRun(7)
    p = str(tmp_path / "c.ckpt")
    CK.save(a, p)
    size = os.path.getsize(p)
    t = str(tmp_path / "t.ckpt")
    with open(p, "rb") as f, open(t, "wb") as g:
        g.write(f.read(size - 4096))
    b = HostRun(8)
    with pytest.raises(CK.CheckpointError, match="truncated"):
        CK.load(b, t)
    c = HostRun(9, split_seed=2)                     # another split
    with pytest.raises(CK.CheckpointError, match="split"):
        CK.load(c, p)
    d = HostRun(10, intv=50)
    with pytest.raises(CK.CheckpointError, match="intv"):
        CK.load(d, p)
    e = HostRun(11, adaptive=False)
    with pytest.raises(CK.CheckpointError, match="adaptive"):
        CK.load(e, p)
    junk = str(tmp_path / "junk")
    open(junk, "wb").write(b"not a checkpoint at all")
    with pytest.raises(CK.CheckpointError, match="not a DOGS"):
        CK.load(b, junk)


def test_header_is_plain_json(tmp_path):
    a = HostRun(12)
    p = str(tmp_path / "h.ckpt")
    CK.save(a, p)
    with open(p, "rb") as f:
        assert f.read(8) == CK.MAGIC
        hlen, start = struct.unpack("<QQ", f.read(16))
        h = json.loads(f.read(hlen))
    assert h["t"] == 1234 and [e["name"] for e in h["buffers"]] == list(CK.BUFFERS)
    assert start == -(-(24 + hlen) // 4096) * 4096


class DensifiedRun(HostRun):
    """A run whose layout changed after it started (a densification): it
    keeps the fingerprint of its original layout and installs a stored one."""

    def __init__(self, seed, layout_seed):
        super().__init__(seed, split_seed=1)
        self.split_origin = CK.split_fingerprint(self.split)
        if layout_seed != 1:                           # the run after its layout changed
            rng = np.random.default_rng(layout_seed)
            xy = rng.uniform(0, 100, (620, 2))
            self._install(S.block_split(xy, 2, 2, [0.25] * 4, 0.1)[0])
            g = torch.Generator().manual_seed(seed + 100)
            for name in ("z", "x", "u", "m", "v"):
                getattr(self, name).data.copy_(torch.randn(getattr(self, name).data.numel(), generator=g))
        self.dstats = torch.arange(2 * self.split.n_copies, dtype=torch.float32)
        self.installs = 0

    def _install(self, split):
        self.split = split
        self.z = D.GaussianBuffer(split.n_globals, 1, "cpu")
        for name in ("x", "u", "m", "v", "anchor"):
            setattr(self, name, D.GaussianBuffer(split.n_copies, 1, "cpu"))

    def install_split(self, split, z, x, m, v, u, calibrate=True):
        self.split, self.z, self.x, self.m, self.v, self.u = split, z, x, m, v, u
        self.dstats = torch.zeros(2 * split.n_copies, dtype=torch.float32)
        self.installs += 1


def test_densified_layout_is_stored_and_installed(tmp_path):
    a = DensifiedRun(21, layout_seed=7)
    p = str(tmp_path / "d.ckpt")
    CK.save(a, p)
    hdr = CK.read_header(p)
    assert {e["name"] for e in hdr["arrays"]} >= {"split.copy_gid", "split.g_copies", "dstats"}
    b = DensifiedRun(22, layout_seed=1)               # built on the original layout
    CK.load(b, p)
    assert b.installs == 1 and CK.split_fingerprint(b.split) == CK.split_fingerprint(a.split)
    for name in ("z", "x", "u", "m", "v"):
        assert torch.equal(getattr(a, name).data.view(torch.int32), getattr(b, name).data.view(torch.int32))
    assert torch.equal(a.dstats, b.dstats)
    # a run from another original layout refuses it
    c = DensifiedRun(23, layout_seed=1)
    c.split_origin = "another run"
    with pytest.raises(CK.CheckpointError, match="split"):
        CK.load(c, p)


def test_damaged_densified_checkpoint_leaves_the_trainer_untouched(tmp_path):
    """A densified checkpoint with one damaged buffer is refused before the
    stored layout is installed: the trainer keeps its layout and state."""
    a = DensifiedRun(31, layout_seed=7)
    p = str(tmp_path / "bad.ckpt")
    CK.save(a, p)
    hdr = CK.read_header(p)
    e = [b for b in hdr["buffers"] if b["name"] == "v"][0]
    with open(p, "r+b") as f:                         # flip one byte of the last buffer
        f.seek(hdr["data_start"] + e["offset"] + 100)
        byte = f.read(1)
        f.seek(hdr["data_start"] + e["offset"] + 100)
        f.write(bytes([byte[0] ^ 0x40]))
    b = DensifiedRun(32, layout_seed=1)
    split0, z0 = b.split, b.z.data.clone()
    with pytest.raises(CK.CheckpointError, match="CRC"):
        CK.load(b, p)
    assert b.installs == 0 and b.split is split0 and torch.equal(b.z.data, z0)


def test_densified_checkpoint_with_wrong_statistics_size_is_refused(tmp_path):
    a = DensifiedRun(33, layout_seed=7)
    a.dstats = torch.zeros(2 * a.split.n_copies + 2, dtype=torch.float32)
    p = str(tmp_path / "st.ckpt")
    CK.save(a, p)
    b = DensifiedRun(34, layout_seed=1)
    with pytest.raises(CK.CheckpointError, match="statistics"):
        CK.load(b, p)
    assert b.installs == 0
