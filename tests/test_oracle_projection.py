"""Pins of the oracle's projection (Sec. 3.1: Eq. 1, Sigma = R S S^T R^T;
EWA projection J W Sigma W^T J^T + 0.3 I; real SH colour)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2405_13943_b300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def one_gaussian(mean, quat, log_scale, ologit=0.0, sh=None, deg=0):
    K = (deg + 1) ** 2
    if sh is None:
        sh = np.zeros((1, K, 3), np.float32)
    return S.Gaussians(np.asarray([mean], np.float32), np.asarray([quat], np.float32),
                       np.asarray([log_scale], np.float32), np.asarray([ologit], np.float32),
                       np.asarray(sh, np.float32).reshape(1, K, 3))


def conic_inverse(rec, O):
    a, b, c = rec[O.REC_A], rec[O.REC_B], rec[O.REC_C]
    return np.linalg.inv(np.array([[a, b], [b, c]]))


def test_on_axis_covariance_matches_scipy_rotation(oracle):
    """On the optical axis with an axis-aligned camera the screen covariance
    is (f/tz)^2 Sigma_xy + 0.3 I, with Sigma = R diag(exp(2s)) R^T; R comes
    from scipy's quaternion routine (scalar-last), not from the oracle."""
    O = oracle
    rng = np.random.default_rng(0)
    cam = S.cube_camera(256, 256, f=200.0, distance=5.0)
    for _ in range(20):
        q = rng.standard_normal(4)
        q *= rng.uniform(0.5, 2.0) / np.linalg.norm(q)           # not normalised
        s = rng.normal(-2.0, 0.4, 3)
        g = one_gaussian([0, 0, 0], q, s)
        rec = O.project(O.params_from(g), 0, cam, 16, 16)["rec"][0]
        q = np.asarray(g.quats[0], np.float64)
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = Rq @ np.diag(np.exp(2 * np.asarray(g.log_scales[0], np.float64))) @ Rq.T
        want = (200.0 / 5.0) ** 2 * Sig[:2, :2] + 0.3 * np.eye(2)
        np.testing.assert_allclose(conic_inverse(rec, O), want, rtol=1e-10, atol=1e-12)


def test_axis_aligned_gaussian_has_diagonal_covariance(oracle):
    O = oracle
    cam = S.cube_camera(256, 256, f=100.0, distance=4.0)
    g = one_gaussian([0, 0, 0], [1, 0, 0, 0], [-2.0, -1.5, -1.0])
    rec = O.project(O.params_from(g), 0, cam, 16, 16)["rec"][0]
    s = np.exp(2 * np.array([-2.0, -1.5, -1.0], np.float32).astype(np.float64))
    np.testing.assert_allclose(conic_inverse(rec, O), np.diag((100 / 4.0) ** 2 * s[:2]) + 0.3 * np.eye(2),
                               rtol=1e-12)


def test_off_axis_ewa_matches_numerical_jacobian(oracle):
    """EWA splatting linearises the perspective map pi(t) = (fx tx/tz + cx,
    fy ty/tz + cy) at the Gaussian's centre.  Take that Jacobian by central
    differences of pi (not by the oracle's formula), rotate with a random
    camera, and compare the screen covariance and the projected mean."""
    O = oracle
    rng = np.random.default_rng(1)
    for i in range(20):
        Rc = Rotation.from_rotvec(rng.normal(0, 0.3, 3)).as_matrix().astype(np.float32)
        t = np.array([0.1, -0.2, 6.0], np.float32)
        cam = S.Camera(320, 240, 250.0, 260.0, 160.0, 120.0, Rc, t, -(Rc.T @ t), 0.2)
        mu = rng.uniform(-1.2, 1.2, 3)
        q = rng.standard_normal(4)
        s = rng.normal(-2.0, 0.3, 3)
        g = one_gaussian(mu, q, s)
        p = O.project(O.params_from(g), 0, cam, 16, 16)
        if not p["visible"][0]:
            continue
        rec = p["rec"][0]
        Rd, td = Rc.astype(np.float64), t.astype(np.float64)
        tc = Rd @ np.asarray(g.means[0], np.float64) + td

        def pi(v):
            return np.array([cam.fx * v[0] / v[2] + cam.cx, cam.fy * v[1] / v[2] + cam.cy])

        J = np.zeros((2, 3))
        h = 1e-6
        for k in range(3):
            e = np.zeros(3); e[k] = h
            J[:, k] = (pi(tc + e) - pi(tc - e)) / (2 * h)
        qq = np.asarray(g.quats[0], np.float64)
        Rq = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        Sig = Rq @ np.diag(np.exp(2 * np.asarray(g.log_scales[0], np.float64))) @ Rq.T
        want = J @ Rd @ Sig @ Rd.T @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(conic_inverse(rec, O), want, rtol=1e-6)
        np.testing.assert_allclose([rec[O.REC_MX], rec[O.REC_MY]], pi(tc), rtol=1e-12)
        assert rec[O.REC_DEPTH] == pytest.approx(tc[2], rel=1e-14)


def test_radius_and_tile_rect(oracle):
    """radius = ceil(3 sqrt(lambda_max)); rect = [floor((m - r)/tile),
    floor((m + r)/tile) + 1) clamped to the grid; culls behind the near plane
    and beyond the 1.3x frustum guard band."""
    O = oracle
    cam = S.cube_camera(100, 90, f=120.0, distance=4.0)
    g = one_gaussian([0.3, -0.2, 0.5], [0.9, 0.1, -0.3, 0.2], [-2.2, -1.7, -2.5])
    p = O.project(O.params_from(g), 0, cam, 16, 16)
    rec = p["rec"][0]
    lam = np.linalg.eigvalsh(conic_inverse(rec, O)).max()
    r = math.ceil(3 * math.sqrt(lam))
    assert rec[O.REC_RADIUS] == r
    mx, my = rec[O.REC_MX], rec[O.REC_MY]
    TX, TY = 7, 6
    rect = [min(max(math.floor((mx - r) / 16), 0), TX), min(max(math.floor((my - r) / 16), 0), TY),
            min(max(math.floor((mx + r) / 16) + 1, 0), TX), min(max(math.floor((my + r) / 16) + 1, 0), TY)]
    assert list(p["rect"][0]) == rect
    assert rec[O.REC_TILES] == (rect[2] - rect[0]) * (rect[3] - rect[1])
    # behind the near plane
    g2 = one_gaussian([0, 0, -3.9], [1, 0, 0, 0], [-2, -2, -2])
    assert O.project(O.params_from(g2), 0, cam, 16, 16)["visible"][0] == 0
    # outside the guard band: |x/z| > 1.3 * (W/2) / fx
    lim = 1.3 * 50 / 120.0
    g3 = one_gaussian([(lim + 0.01) * 4.0, 0, 0], [1, 0, 0, 0], [-2, -2, -2])
    g4 = one_gaussian([(lim - 0.01) * 4.0, 0, 0], [1, 0, 0, 0], [-2, -2, -2])
    assert O.project(O.params_from(g3), 0, cam, 16, 16)["visible"][0] == 0
    assert O.project(O.params_from(g4), 0, cam, 16, 16)["rec"][0][O.REC_DEPTH] == pytest.approx(4.0)


def test_depth_key_is_float_of_camera_z(oracle):
    O = oracle
    cam = S.cube_camera()
    g = S.cube_scene(200, 5)
    p = O.project(O.params_from(g), 0, cam, 16, 16)
    vis = p["visible"] == 1
    np.testing.assert_array_equal(p["depth_key"][vis], p["rec"][vis, O.REC_DEPTH].astype(np.float32))


# ---------------------------------------------------------------------------
# SH basis
# ---------------------------------------------------------------------------
def test_sh_table_values(oracle):
    O = oracle
    tab = json.load(open(os.path.join(GOLD, "real_sh_table.json")))
    rng = np.random.default_rng(2)
    for _ in range(10):
        d = rng.standard_normal(3); d /= np.linalg.norm(d)
        x, y, z = d
        for e in tab["entries"]:
            want = eval(e["form"], {"sqrt": math.sqrt, "pi": math.pi, "x": x, "y": y, "z": z})
            got, _ = O.sh_basis(e["l"], e["m"], d)
            assert got == pytest.approx(want, rel=1e-12, abs=1e-14), (e, got, want)


def test_sh_orthonormal_by_quadrature(oracle):
    """Gauss-Legendre in cos(theta) x uniform phi integrates products of two
    degree<=3 harmonics exactly."""
    O = oracle
    ct, wt = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phis = np.arange(nphi) * 2 * np.pi / nphi
    lms = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    Y = np.zeros((len(lms), len(ct) * nphi))
    W = np.zeros(len(ct) * nphi)
    col = 0
    for c, w in zip(ct, wt):
        s = math.sqrt(1 - c * c)
        for ph in phis:
            d = np.array([s * math.cos(ph), s * math.sin(ph), c])
            for i, (l, m) in enumerate(lms):
                Y[i, col] = O.sh_basis(l, m, d)[0]
            W[col] = w * 2 * np.pi / nphi
            col += 1
    G = (Y * W) @ Y.T
    np.testing.assert_allclose(G, np.eye(len(lms)), atol=1e-12)


def test_sh_addition_theorem(oracle):
    """sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a.b)."""
    O = oracle
    rng = np.random.default_rng(3)
    for _ in range(10):
        a = rng.standard_normal(3); a /= np.linalg.norm(a)
        b = rng.standard_normal(3); b /= np.linalg.norm(b)
        for l in range(4):
            s = sum(O.sh_basis(l, m, a)[0] * O.sh_basis(l, m, b)[0] for m in range(-l, l + 1))
            Pl = np.polynomial.legendre.legval(a @ b, [0] * l + [1])
            assert s == pytest.approx((2 * l + 1) / (4 * np.pi) * Pl, abs=1e-13)


def test_sh_gradient_tangential_by_fd(oracle):
    O = oracle
    rng = np.random.default_rng(4)
    for _ in range(10):
        d = rng.standard_normal(3); d /= np.linalg.norm(d)
        t = rng.standard_normal(3); t -= d * (d @ t); t /= np.linalg.norm(t)
        for l in range(4):
            for m in range(-l, l + 1):
                _, g = O.sh_basis(l, m, d)
                h = 1e-6
                dp = np.cos(h) * d + np.sin(h) * t
                dm = np.cos(h) * d - np.sin(h) * t
                fd = (O.sh_basis(l, m, dp)[0] - O.sh_basis(l, m, dm)[0]) / (2 * h)
                assert g @ t == pytest.approx(fd, abs=1e-8)


def test_colour_degree0_and_clamp(oracle):
    O = oracle
    cam = S.cube_camera()
    Y00 = 0.5 / math.sqrt(math.pi)
    sh = np.array([[[1.0, -0.5 / Y00 - 1.0, 0.2]]])
    g = one_gaussian([0, 0, 0], [1, 0, 0, 0], [-2, -2, -2], sh=sh)
    rec = O.project(O.params_from(g), 0, cam, 16, 16)["rec"][0]
    assert rec[O.REC_R] == pytest.approx(Y00 * 1.0 + 0.5)
    assert rec[O.REC_G] == 0.0 and rec[O.REC_RAWG] == pytest.approx(-Y00 * (0.5 / Y00 + 1.0) + 0.5)
    assert rec[O.REC_BL] == pytest.approx(Y00 * np.float32(0.2) + 0.5)
    assert rec[O.REC_OP] == pytest.approx(0.5)
