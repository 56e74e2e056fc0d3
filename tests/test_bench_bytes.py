"""The byte model behind bench.py's HBM rooflines (the algorithmic bytes of
each timed call), checked against relations that hold for any split of the
copies, on a small synthetic split (host only):
- the two parts of the split x-step move, together, the one-part step's
  bytes, whatever groups hold a kept record;
- a part 1 that tests its groups reads 8 more bytes (one rectangle) per
  copy it steps; the group lists read every copy's rectangle and write one
  entry per group of 128;
- storing the unshared copies into z in the x-step (the iteration's
  consensus then covering the shared globals only) saves, per unshared
  global, the consensus's read of x (the x-step holds it already) and
  costs the global id's 4 bytes."""
import types

import numpy as np
import pytest

# parameters of one Gaussian at SH degree 3: 48 SH coefficients, mean 3,
# opacity 1, rotation 4, log-scale 3
P = 3 * 16 + 3 + 1 + 4 + 3
VIS = 1234          # visible records / copies: any count


@pytest.fixture(scope="module")
def model():
    import bench
    from paper_2405_13943_b300 import synth as S
    wl = S.dogs_workload(20_000, 2, 2, 0.1, 5, views_per_step=1, pool=1, width=64, height=48)
    tr = types.SimpleNamespace(split=wl.split, vb=types.SimpleNamespace(n_rec=wl.split.n_copies))
    return bench, tr


def groups_of(n_c, frac, seed):
    n_groups = -(-n_c // 128)
    return np.random.default_rng(seed).random(n_groups) < frac


@pytest.mark.parametrize("frac", [0.0, 0.3, 1.0])
def test_split_xstep_partitions_the_one_part_bytes(model, frac):
    bench, tr = model
    n_c = tr.split.n_copies
    act = groups_of(n_c, frac, 11)
    one = bench.algorithmic_bytes(tr, VIS, VIS)
    two = bench.algorithmic_bytes(tr, VIS, VIS, act, idle_tests=False)
    assert two["xstep"] + two["xstep_idle"] == one["xstep"]
    idle_copies = int((~np.repeat(act, 128)[:n_c]).sum())
    tested = bench.algorithmic_bytes(tr, VIS, VIS, act)
    assert tested["xstep_idle"] - two["xstep_idle"] == 8 * idle_copies
    assert "xstep_groups" not in tested
    listed = bench.algorithmic_bytes(tr, VIS, VIS, act, listed=True, idle_tests=False)
    assert listed["xstep_groups"] == 8 * n_c + 4 * len(act)
    assert listed["xstep"] == two["xstep"] and listed["xstep_idle"] == two["xstep_idle"]


def test_unshared_store_in_the_xstep_moves_bytes_out_of_the_consensus(model):
    bench, tr = model
    sp = tr.split
    cnt = np.diff(sp.g_off)
    ug = int((cnt == 1).sum())
    assert ug == sp.n_copies - int(sp.blk_nshared.sum()) > 0    # one copy per unshared global
    act = groups_of(sp.n_copies, 0.4, 12)
    keys = ("xstep", "xstep_idle", "admm_consensus")
    plain = bench.algorithmic_bytes(tr, VIS, VIS, act, zfuse=False, idle_tests=False)
    fused = bench.algorithmic_bytes(tr, VIS, VIS, act, zfuse=True, idle_tests=False)
    # per unshared global: the consensus no longer reads x and writes z (8 B per
    # parameter); the x-step writes z (4 B per parameter) and reads the global id (4 B)
    assert sum(fused[k] for k in keys) - sum(plain[k] for k in keys) == ug * (4 * P + 4 - 8 * P)
    # the consensus's remaining bytes are the shared globals' alone
    sg, sc = int((cnt > 1).sum()), int(cnt[cnt > 1].sum())
    assert fused["admm_consensus"] == plain["admm_consensus"] - 8 * P * ug
    assert fused["admm_consensus"] == P * (16 * sc + 8 * sg)


def test_one_part_xstep_counts_every_parameter_of_every_copy(model):
    """x, m, v read and written (24 B) for each parameter of each copy, the
    anchor read (4 B) for each shared copy's parameter, and 56 B per visible
    record (its 2D gradients and rectangle)."""
    bench, tr = model
    sp = tr.split
    one = bench.algorithmic_bytes(tr, VIS, VIS)
    n_sc = int(sp.copy_shared().astype(bool).sum())
    assert one["xstep"] == sp.n_copies * P * 24 + n_sc * P * 4 + VIS * 56
    # the separate path also reads the gradient (4 B per parameter)
    assert one["adam_admm_step"] - (one["xstep"] - VIS * 56) == sp.n_copies * P * 4
