"""Pins of the oracle's scene split (Sec. 3.2 "Scene Splitting", Alg. 1):
hand-worked lattices, the balance the recursive bipartition guarantees, the
separation of cells by axis-aligned cuts, cuts across the longer side, the
imbalance of a uniform grid that Alg. 1 removes (Fig. 4), and the overlap
by the box scale factor s."""
import numpy as np
import pytest


def lattice(nx, ny):
    return np.array([(i, j) for i in range(nx) for j in range(ny)], np.float64)


def test_hand_lattice_k4(oracle):
    # 8 x 2 lattice: the root box is 7 x 1, cut in x at the median; each half
    # (3 x 1) is cut in x again; cells come out in the order Alg. 1 pushes them
    xy = lattice(8, 2)
    cell, boxes = oracle.scene_split(xy, 4)
    assert cell.tolist() == [0] * 4 + [1] * 4 + [2] * 4 + [3] * 4
    assert boxes.tolist() == [[0, 1, 0, 1], [2, 3, 0, 1], [4, 5, 0, 1], [6, 7, 0, 1]]


def test_hand_line_k3_and_square_tie(oracle):
    # K = 3: budgets 1 | 2, the lower child takes floor(9 * 1 / 3) = 3 points;
    # the leaf is pushed back before the upper child's two halves
    xy = np.stack([np.arange(9.0), np.zeros(9)], 1)
    cell, boxes = oracle.scene_split(xy, 3)
    assert cell.tolist() == [0, 0, 0, 1, 1, 1, 2, 2, 2]
    assert boxes[:, :2].tolist() == [[0, 2], [3, 5], [6, 8]]
    # a square cell is cut along x; equal coordinates go by point index
    sq = np.array([(0, 0), (1, 1), (0, 1), (1, 0)], np.float64)
    cell, _ = oracle.scene_split(sq, 2)
    assert cell.tolist() == [0, 1, 0, 1]
    # after re-fitting, a 2 x 4 lattice half is taller than wide: cut along y
    cell, boxes = oracle.scene_split(lattice(4, 4), 4)
    assert boxes.tolist() == [[0, 1, 0, 1], [0, 1, 2, 3], [2, 3, 0, 1], [2, 3, 2, 3]]


@pytest.mark.parametrize("n,K", [(1000, 8), (999, 7), (17, 5), (3, 4), (0, 2), (50, 1), (200, 64)])
def test_balance_floor_ceil(oracle, n, K):
    """Every cut hands floor(n k_lo / k) points to k_lo leaves, so every block
    ends with floor(n / K) or ceil(n / K) points (induction on the cut)."""
    rng = np.random.default_rng(n + K)
    xy = rng.standard_normal((n, 2)) * [100, 20]
    cell, boxes = oracle.scene_split(xy, K)
    counts = np.bincount(cell, minlength=K)
    assert counts.sum() == n
    assert counts.min() >= n // K and counts.max() <= -(-n // K)
    # tight boxes contain their points and touch them on every side
    for k in range(K):
        p = xy[cell == k]
        if len(p):
            assert boxes[k].tolist() == [p[:, 0].min(), p[:, 0].max(), p[:, 1].min(), p[:, 1].max()]
        else:
            assert np.isinf(boxes[k]).all()


def test_cells_are_separated(oracle):
    """Cells come from axis-aligned cuts, so their tight boxes have disjoint
    interiors (brute force over all pairs, continuous coordinates)."""
    rng = np.random.default_rng(3)
    xy = rng.uniform(0, 1000, (4000, 2))
    _, b = oracle.scene_split(xy, 11)
    for i in range(11):
        for j in range(i + 1, 11):
            ox = min(b[i, 1], b[j, 1]) - max(b[i, 0], b[j, 0])
            oy = min(b[i, 3], b[j, 3]) - max(b[i, 2], b[j, 2])
            assert ox <= 0 or oy <= 0, (i, j)


def test_cuts_cross_the_longer_side(oracle):
    """A strip 100 times longer than wide is cut into slabs across its length
    only; a strip that is tall is cut along y."""
    rng = np.random.default_rng(4)
    xy = rng.uniform(0, 1, (2000, 2)) * [1000, 10]
    cell, b = oracle.scene_split(xy, 8)
    order = np.argsort(b[:, 0])
    assert np.all(b[order[1:], 0] > b[order[:-1], 1])       # slabs ordered along x
    assert np.all(b[:, 3] - b[:, 2] > 9)                     # each spans the full width
    cell_t, bt = oracle.scene_split(xy[:, ::-1].copy(), 8)
    assert np.all(bt[:, 1] - bt[:, 0] > 9)


def test_balanced_where_a_uniform_grid_is_not(oracle):
    """A city with a dense centre: a 2 x 2 grid of equal cells leaves the
    block sizes far apart; the recursive bipartition does not (Fig. 4)."""
    rng = np.random.default_rng(5)
    xy = np.concatenate([rng.normal(300, 60, (6000, 2)), rng.uniform(0, 1000, (2000, 2))])
    lo, hi = xy.min(0), xy.max(0)
    gx = np.minimum(((xy[:, 0] - lo[0]) / (hi[0] - lo[0]) * 2).astype(int), 1)
    gy = np.minimum(((xy[:, 1] - lo[1]) / (hi[1] - lo[1]) * 2).astype(int), 1)
    grid = np.bincount(gx * 2 + gy, minlength=4)
    assert grid.max() > 5 * grid.min()
    cell, _ = oracle.scene_split(xy, 4)
    assert np.bincount(cell).tolist() == [2000] * 4


def test_overlap_by_scale_factor(oracle):
    xy = lattice(8, 2)
    cell, boxes = oracle.scene_split(xy, 4)
    # s = 3 on the cell [2, 3]: centre 2.5, half side 1.5 -> [1, 4]
    m = oracle.scene_assign(xy, boxes, 3.0, own=cell)
    x = xy[:, 0]
    assert m[:, 1].tolist() == ((x >= 1) & (x <= 4)).tolist()
    assert m[:, 0].tolist() == ((x >= -1) & (x <= 2)).tolist()
    # s = 1.5: [1.75, 3.25] holds only the cell's own lattice columns
    m = oracle.scene_assign(xy, boxes, 1.5, own=cell)
    assert (m.sum(1) == 1).all()
    # continuous cloud: s = 1 is the partition itself; larger s only adds
    rng = np.random.default_rng(6)
    pts = rng.uniform(0, 1000, (3000, 2))
    c, b = oracle.scene_split(pts, 8)
    prev = oracle.scene_assign(pts, b, 1.0, own=c)
    assert (prev.sum(1) == 1).all() and prev[np.arange(3000), c].all()
    for s in (1.2, 1.4, 2.0, 50.0):
        cur = oracle.scene_assign(pts, b, s, own=c)
        assert (cur | prev == cur).all()
        prev = cur
    assert prev.all()


def test_nearest_block_for_uncovered_positions(oracle):
    boxes = np.array([[0, 1, 0, 1], [10, 11, 0, 1], [np.inf, -np.inf, np.inf, -np.inf]])
    q = np.array([[3.0, 0.5], [8.0, 0.5], [5.5, 0.5], [0.5, 0.5]])
    m = oracle.scene_assign(q, boxes, 1.0, nearest=True)
    # 3 is 2 from box 0, 8 is 2 from box 1, 5.5 ties at 4.5 -> lowest index
    assert m.tolist() == [[1, 0, 0], [0, 1, 0], [1, 0, 0], [1, 0, 0]]
    assert not oracle.scene_assign(q[:3], boxes, 1.0).any()
