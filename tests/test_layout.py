"""The library's host layout builder (dg_layout) gives the same global
numbering, block-local copies and sharing map as the reference numpy layout
of the input generator (synth.split_layout), and rejects a point in no
block."""
import numpy as np
import pytest

from paper_2405_13943_b300 import build as B
from paper_2405_13943_b300 import synth as S


@pytest.fixture(scope="module")
def DZ():
    B.build()
    from paper_2405_13943_b300 import densify
    return densify


# (300000, 8): past 65,536 points per thread, so the builder's passes run on
# several host threads where the machine has them
@pytest.mark.parametrize("n,K,seed", [(1, 1, 0), (500, 1, 1), (3000, 4, 2), (20000, 8, 3), (4000, 37, 4),
                                      (5000, 64, 5), (300000, 8, 7)])
def test_native_layout_equals_reference(DZ, n, K, seed):
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-50, 900, (n, 2))
    xy[: n // 10] = xy[0]                           # ties in position
    member = np.zeros((n, K), bool)
    member[np.arange(n), rng.integers(0, K, n)] = True
    extra = rng.random((n, K)) < (0.15 / K)
    member |= extra
    a, oa = S.split_layout(xy, member, np.zeros((K, 4)), 1.0)
    b, ob = DZ.native_layout(xy, member, np.zeros((K, 4)), 1.0)
    np.testing.assert_array_equal(oa, ob)
    for f in ("copy_gid", "blk_off", "blk_nshared", "g_off", "g_copies"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    assert a.n_shared_globals == b.n_shared_globals


def test_native_layout_rejects_a_point_in_no_block(DZ):
    member = np.zeros((3, 2), bool)
    member[0, 0] = member[2, 1] = True
    with pytest.raises(Exception):
        DZ.native_layout(np.zeros((3, 2)), member, np.zeros((2, 4)), 1.0)


@pytest.mark.parametrize("n", [3000, 200000])     # the larger one spans several host threads
def test_carried_copies_by_brute_force(DZ, n):
    """The copy whose state a new copy takes over: the parent's copy in the
    same block when the new Gaussian is its parent itself, else none."""
    rng = np.random.default_rng(6)
    K = 6
    xy = rng.uniform(0, 100, (n, 2))
    member = np.zeros((n, K), bool)
    member[np.arange(n), rng.integers(0, K, n)] = True
    member[rng.random(n) < 0.2, 2] = True
    old, _ = S.split_layout(xy, member, np.zeros((K, 4)), 1.0)
    outs = rng.integers(0, 3, n)                        # pruned, kept or cloned
    src = np.repeat(np.arange(n), outs)
    orig = np.ones(len(src), bool)
    orig[1:] &= src[1:] != src[:-1]                     # the second of a pair is the copy
    new, order = DZ.native_layout(rng.uniform(0, 100, (len(src), 2)), DZ.membership(old)[src],
                                  np.zeros((K, 4)), 1.0, K=K)
    src_new, orig_new = src[order], orig[order]
    got = DZ.carried_copies(old, new, src_new, orig_new)
    oblk = np.repeat(np.arange(K), np.diff(old.blk_off))
    nblk = np.repeat(np.arange(K), np.diff(new.blk_off))
    where = {(int(old.copy_gid[i]), int(oblk[i])): i for i in range(old.n_copies)}
    want = [where.get((int(src_new[g]), int(nblk[i])), -1) if orig_new[g] else -1
            for i, g in enumerate(new.copy_gid)]
    np.testing.assert_array_equal(got, want)
    assert 0 < (got >= 0).mean() < 1


def test_carry_rejects_an_id_out_of_range(DZ):
    rng = np.random.default_rng(8)
    n, K = 200, 3
    member = np.zeros((n, K), bool)
    member[np.arange(n), rng.integers(0, K, n)] = True
    old, _ = S.split_layout(rng.uniform(0, 10, (n, 2)), member, np.zeros((K, 4)), 1.0)
    src = np.arange(n)
    src[5] = n + 3                                      # a parent that the old layout does not have
    with pytest.raises(Exception):
        DZ.carried_copies(old, old, src, np.ones(n, bool))


@pytest.mark.parametrize("n,K,pattern", [(70000, 3, "all"), (70000, 64, "one"), (2, 64, "all")])
def test_native_layout_extreme_memberships(DZ, n, K, pattern):
    """Every point in every block (all globals shared), or all points in the
    last of many blocks (every other block empty), against the reference."""
    rng = np.random.default_rng(9)
    xy = rng.uniform(0, 50, (n, 2))
    member = np.zeros((n, K), bool)
    if pattern == "all":
        member[:] = True
    else:
        member[:, K - 1] = True
    a, oa = S.split_layout(xy, member, np.zeros((K, 4)), 1.0)
    b, ob = DZ.native_layout(xy, member, np.zeros((K, 4)), 1.0)
    np.testing.assert_array_equal(oa, ob)
    for f in ("copy_gid", "blk_off", "blk_nshared", "g_off", "g_copies"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    assert a.n_shared_globals == b.n_shared_globals == (n if pattern == "all" else 0)


@pytest.mark.parametrize("n,K", [(3000, 5), (150000, 64)])
def test_parent_membership_equals_the_old_membership(DZ, n, K):
    """dg_layout_membership gives each new Gaussian its parent's blocks, as
    the membership of the old layout indexed by the parents."""
    rng = np.random.default_rng(10)
    member = np.zeros((n, K), bool)
    member[np.arange(n), rng.integers(0, K, n)] = True
    member |= rng.random((n, K)) < 2.0 / K
    old, _ = S.split_layout(rng.uniform(0, 10, (n, 2)), member, np.zeros((K, 4)), 1.0)
    parent = np.concatenate([np.arange(n), rng.integers(0, n, n // 3)])
    np.testing.assert_array_equal(DZ.parent_membership(old, parent), DZ.membership(old)[parent])
    with pytest.raises(Exception):
        DZ.parent_membership(old, np.array([0, n]))


def test_native_layout_rejects_non_finite_positions(DZ):
    member = np.ones((4, 2), bool)
    for bad in (np.nan, np.inf, -np.inf):
        xy = np.zeros((4, 2))
        xy[2, 1] = bad
        with pytest.raises(Exception):
            DZ.native_layout(xy, member, np.zeros((2, 4)), 1.0)


def test_layout_rejects_copy_counts_beyond_int32(DZ):
    """2^25 points each held by all 64 blocks make 2^31 copies, more than the
    layout's 32-bit copy numbers hold: refused before any output is written
    (the outputs here are one element long; a write would overrun them)."""
    import ctypes as C
    from paper_2405_13943_b300 import _lib as L
    n, K = 1 << 25, 64
    member = np.full(n, np.uint64(0xFFFFFFFFFFFFFFFF))
    xy = np.zeros((n, 2))
    one32, one64 = np.zeros(1, np.int32), np.zeros(K + 1, np.int64)
    ns = np.zeros(1, np.int64)
    rc = L.lib().dg_layout(xy.ctypes.data, member.ctypes.data, n, K, one32.ctypes.data, one32.ctypes.data,
                           one64.ctypes.data, one64.ctypes.data, one64.ctypes.data, one32.ctypes.data,
                           ns.ctypes.data)
    assert rc == L.DG_ERR_INVALID
    assert L.lib().dg_layout_copies(member.ctypes.data, n) == 1 << 31
