"""Pins of the oracle's densification (Sec. 4: 3DGS adaptive density control,
restated): the statistic by hand, every decision branch at and around its
threshold, the emission order, and the split children's distribution
against the covariance built by scipy's rotation."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2405_13943_b300 import synth as S


def gaussians(n, seed=3, deg=1):
    return O.params_from(S.cube_scene(n, seed, sh_degree=deg))


def test_quat_rotation_matches_scipy():
    rng = np.random.default_rng(5)
    for _ in range(20):
        q = rng.normal(size=4)
        want = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(O.quat_rotation(q), want, atol=1e-12)


def test_statistic_by_hand():
    # copy 0 seen in two 100x50 views, copy 1 in one (not kept), copy 2 in one
    kept = np.array([1, 1, 0, 1], bool)
    dm = np.array([[0.01, 0.0], [0.0, 0.02], [5.0, 5.0], [0.003, 0.004]])
    wh = np.array([[100, 50], [100, 50], [100, 50], [200, 200]])
    owner = np.array([0, 0, 1, 2])
    s, c = O.densify_stats(kept, dm, wh, owner, 3)
    np.testing.assert_allclose(s, [0.5 + 0.5, 0.0, np.hypot(0.3, 0.4)])
    np.testing.assert_allclose(c, [2, 0, 1])


def one_copy_csr(n):
    return np.arange(n + 1), np.arange(n)


def test_decisions_at_their_thresholds():
    z = gaussians(6)
    P = O.split_params(z, 1)
    g_off, g_cp = one_copy_csr(6)
    lo = np.log(0.005 / 0.995)
    P["opacity"][:] = 0.0
    P["scale"][:] = np.log(0.001)                      # small: clone side
    P["opacity"][0] = lo - 1e-3                        # prune, whatever its gradient
    s = np.array([1.0, 2e-4 * 10 * 1.0001, 2e-4 * 10 * 0.9999, 1.0, 0.0, 1.0])
    c = np.array([1.0, 10.0, 10.0, 1.0, 0.0, 1.0])
    P["scale"][3, 1] = np.log(0.01 * 5.0) + 1e-3       # largest scale above percent_dense * extent: split
    P["scale"][5, 2] = np.log(0.01 * 5.0) - 1e-3       # just below: clone
    codes = O.densify_decide(z, 1, s, c, g_off, g_cp, extent=5.0)
    assert list(codes) == [O.DENSIFY_PRUNE, O.DENSIFY_CLONE, O.DENSIFY_KEEP, O.DENSIFY_SPLIT,
                           O.DENSIFY_KEEP, O.DENSIFY_CLONE]


def test_decision_margins_by_hand():
    """The margin is the least relative distance from a threshold among the
    comparisons that led to the code, each quantity formed in FP64."""
    z = gaussians(4)
    P = O.split_params(z, 1)
    g_off, g_cp = one_copy_csr(4)
    logit = lambda p: np.log(p / (1.0 - p))
    P["opacity"][:] = [logit(0.006), logit(0.004), logit(0.5), logit(0.5)]
    P["scale"][:] = np.log(0.001)
    P["scale"][0, 2] = np.log(0.015)                   # largest scale 1.5x the split size
    s = np.array([2.2e-4 * 4, 2e-4 * 4, 0.0, 2e-4 * 4 * (1 - 1e-9)])
    c = np.array([4.0, 4.0, 0.0, 4.0])
    codes, m = O.densify_decide(z, 1, s, c, g_off, g_cp, return_margin=True)
    assert list(codes) == [O.DENSIFY_SPLIT, O.DENSIFY_PRUNE, O.DENSIFY_KEEP, O.DENSIFY_KEEP]
    np.testing.assert_allclose(m[0], 0.1, rtol=1e-9)   # gradient 2.2e-4 vs 2e-4; opacity 0.2, scale 0.5
    np.testing.assert_allclose(m[1], 0.2, rtol=1e-9)   # pruned: the opacity comparison alone
    np.testing.assert_allclose(m[2], (0.5 - 0.005) / 0.005, rtol=1e-9)   # never seen: opacity only
    assert m[3] < 1e-6                                 # a mean 1e-9 below its threshold: too near to test


def test_statistics_of_all_copies_decide_together():
    z = gaussians(2)
    O.split_params(z, 1)["opacity"][:] = 0.0
    O.split_params(z, 1)["scale"][:] = np.log(0.001)
    g_off = np.array([0, 2, 3])
    g_cp = np.array([0, 2, 1])                         # global 0 held by copies 0 and 2
    # each copy alone is below 2e-4 on average, the two together are above
    s = np.array([3e-4, 1e-4, 1.1e-4])
    c = np.array([1.0, 1.0, 1.0])
    codes = O.densify_decide(z, 1, s, c, g_off, g_cp)
    assert list(codes) == [O.DENSIFY_CLONE, O.DENSIFY_KEEP]


def test_emission_order_and_copies():
    z = gaussians(5)
    codes = np.array([O.DENSIFY_KEEP, O.DENSIFY_PRUNE, O.DENSIFY_CLONE, O.DENSIFY_SPLIT, O.DENSIFY_KEEP])
    xi = np.random.default_rng(1).normal(size=(5, 2, 3))
    zn, src, orig = O.densify_emit(z, 1, codes, xi)
    assert list(src) == [0, 2, 2, 3, 3, 4] and list(orig) == [True, True, False, False, False, True]
    np.testing.assert_array_equal(zn[0], z[0])
    np.testing.assert_array_equal(zn[1], z[2])
    np.testing.assert_array_equal(zn[2], z[2])
    np.testing.assert_array_equal(zn[5], z[4])
    P, Q = O.split_params(z, 1), O.split_params(zn, 1)
    for h in (3, 4):
        np.testing.assert_allclose(Q["scale"][h], P["scale"][3] - np.log(1.6), atol=1e-15)
        np.testing.assert_array_equal(Q["quat"][h], P["quat"][3])
        np.testing.assert_array_equal(Q["sh"][h], P["sh"][3])
        assert Q["opacity"][h] == P["opacity"][3]


def test_split_children_follow_the_parent_distribution():
    """Children means mu + R(q) S xi: over many draws their covariance is the
    parent's R S S^T R^T, built here with scipy's rotation."""
    z = gaussians(1, seed=11)
    P = O.split_params(z, 1)
    P["scale"][0] = np.log([0.3, 0.1, 0.05])
    n = 40000
    xi = np.random.default_rng(2).normal(size=(n, 2, 3))
    zs = np.repeat(z, n, axis=0)
    codes = np.full(n, O.DENSIFY_SPLIT)
    zn, _, _ = O.densify_emit(zs, 1, codes, xi)
    d = O.split_params(zn, 1)["mean"] - P["mean"][0]
    q = P["quat"][0]
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    want = R @ np.diag(np.exp(2 * P["scale"][0])) @ R.T
    got = d.T @ d / d.shape[0]
    assert np.abs(got - want).max() <= 0.02 * np.abs(want).max()
    assert np.abs(d.mean(0)).max() <= 0.01 * np.sqrt(np.diag(want)).max()


def test_opacity_reset_by_hand():
    z = gaussians(3)
    P = O.split_params(z, 1)
    P["opacity"][:] = [-10.0, 0.0, 3.0]
    r = O.split_params(O.reset_opacity(z, 1, 0.01), 1)
    cap = np.log(0.01 / 0.99)
    np.testing.assert_allclose(r["opacity"], [-10.0, cap, cap])
    np.testing.assert_allclose(1 / (1 + np.exp(-r["opacity"][1:])), 0.01)
    np.testing.assert_array_equal(r["mean"], P["mean"])
