"""The library's scene split (dg_scene_split, dg_scene_assign; host code of
Alg. 1 and the scale-factor overlap, Sec. 3.2) equals the oracle's, bit for
bit: cell of every point, tight boxes and block membership, including ties
in coordinates, empty cells, K = 1 and K = 64, and camera grouping."""
import numpy as np
import pytest

from paper_2405_13943_b300 import _lib as L
from paper_2405_13943_b300 import build as B
from paper_2405_13943_b300 import synth as S


@pytest.fixture(scope="module")
def SS():
    B.build()
    from paper_2405_13943_b300 import scene_split
    return scene_split


CASES = [(5000, 8, "uniform"), (4999, 7, "cluster"), (3000, 5, "ties"), (3, 6, "uniform"),
         (0, 3, "uniform"), (1000, 1, "uniform"), (20000, 64, "cluster"), (777, 12, "strip")]


def cloud(n, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.uniform(-500, 500, (n, 3))
    if kind == "cluster":
        return np.concatenate([rng.normal(200, 40, (n // 2, 3)), rng.uniform(0, 1000, (n - n // 2, 3))])
    if kind == "ties":                      # many equal coordinates: order by index decides
        return rng.integers(0, 12, (n, 3)).astype(np.float64)
    return rng.uniform(0, 1, (n, 3)) * [2000, 30, 5]


@pytest.mark.parametrize("n,K,kind", CASES)
def test_split_matches_oracle(SS, oracle, n, K, kind):
    pts = cloud(n, kind, n + K)
    cell, boxes = SS.split_cells(pts, K)
    oc, ob = oracle.scene_split(pts[:, :2], K)
    np.testing.assert_array_equal(cell, oc)
    np.testing.assert_array_equal(boxes, ob)
    for s in (1.0, 1.4, 1.5):
        m = SS.assign(pts, boxes, s, own=cell)
        np.testing.assert_array_equal(m, oracle.scene_assign(pts[:, :2], ob, s, own=oc))
    q = cloud(300, "uniform", 99) * 1.5
    np.testing.assert_array_equal(SS.assign(q, boxes, 1.4, nearest=True),
                                  oracle.scene_assign(q[:, :2], ob, 1.4, nearest=True))


def test_split_scene_layout(SS, oracle):
    """split_scene's copy layout holds exactly the oracle's memberships."""
    pts = cloud(6000, "cluster", 8)
    split, order = SS.split_scene(pts, 6, 1.4)
    oc, ob = oracle.scene_split(pts[:, :2], 6)
    om = oracle.scene_assign(pts[:, :2], ob, 1.4, own=oc)
    got = np.zeros_like(om)
    for k in range(6):
        got[order[split.copy_gid[split.blk_off[k]:split.blk_off[k + 1]]], k] = True
    np.testing.assert_array_equal(got, om)
    assert split.n_shared_globals == int((om.sum(1) >= 2).sum()) > 0
    # CSR over globals lists each global's copies in ascending block order
    for g in range(0, split.n_shared_globals, 97):
        cps = split.g_copies[split.g_off[g]:split.g_off[g + 1]]
        assert (split.copy_gid[cps] == g).all() and len(cps) >= 2
        assert np.all(np.diff(np.searchsorted(split.blk_off, cps, side="right")) > 0)


def test_split_views(SS, oracle):
    pts = cloud(4000, "uniform", 10)
    _, boxes = SS.split_cells(pts, 4)
    cams = S.grid_cameras(3, n_side=6, size=1000.0, width=64, height=48)
    for c in cams:
        c.campos = c.campos - np.float32([500, 500, 0])
    per = SS.split_views(cams, boxes, 1.4)
    pos = np.stack([c.campos[:2].astype(np.float64) for c in cams])
    want = oracle.scene_assign(pos, boxes, 1.4, nearest=True)
    for k in range(4):
        assert [id(v) for v in per[k]] != [id(c) for c in cams]      # copies, not the caller's
        assert [v.block for v in per[k]] == [k] * len(per[k])
        assert len(per[k]) == int(want[:, k].sum())
    assert sum(len(p) for p in per) >= len(cams)


def test_split_rejects_bad_input(SS):
    with pytest.raises(L.DogsError):
        SS.split_cells(np.zeros((4, 2)), 0)
    with pytest.raises(L.DogsError):
        SS.split_cells(np.zeros((4, 2)), 65)
    with pytest.raises(L.DogsError):
        SS.split_cells(np.array([[0.0, np.nan]]), 2)
    _, b = SS.split_cells(np.random.default_rng(0).uniform(0, 1, (10, 2)), 2)
    with pytest.raises(L.DogsError):
        SS.assign(np.zeros((2, 2)), b, 0.9)
    with pytest.raises(L.DogsError):
        SS.assign(np.zeros((2, 2)), b, 1.2, own=[0, 2])
