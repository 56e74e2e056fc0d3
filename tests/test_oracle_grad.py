"""Pin of the oracle's analytic backward by FP64 central finite differences
(h = 1e-6) on a 64-Gaussian 32x32 sub-problem, SH degree 3, two views (one of
them rotated and off-centre), non-black background, smooth loss
L = sum_v <w_v, image_v> with random weights.  Inputs are re-drawn until every
FP decision has relative margin >= 1e-4, so no decision flips within +-h."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2405_13943_b300 import synth as S
from tests._util import curate_gaussians, smooth_weights

BG = (0.1, 0.2, 0.3)


def subproblem(O, seed):
    rng = np.random.default_rng(seed)
    g = S.cube_scene(96, seed, sh_degree=3, log_scale_mu=-2.2, log_scale_sigma=0.3, extent=0.6)
    R2 = Rotation.from_rotvec([0.15, -0.25, 0.1]).as_matrix().astype(np.float32)
    t2 = np.array([0.2, -0.1, 3.5], np.float32)
    cams = [S.cube_camera(32, 32, f=36.0, distance=3.0),
            S.Camera(32, 32, 40.0, 38.0, 15.3, 16.9, R2, t2, -(R2.T @ t2), 0.2)]
    g = curate_gaussians(O, g, cams, 16, 16, thr=1e-4)
    g = g.subset(np.arange(min(64, g.n)))
    rows = [(0, g.n), (0, g.n)]
    plan = O.ViewPlan(cams, rows, 16, 16)
    return g, plan


def loss_and_grad(O, x, deg, plan, W):
    f = O.render(x, deg, plan, BG)
    L = sum(float((w * v["image"]).sum()) for w, v in zip(W, f["views"]))
    return L, f


@pytest.mark.parametrize("seed", [11, 12])
def test_backward_matches_central_differences(oracle, seed):
    O = oracle
    g, plan = subproblem(O, seed)
    x = O.params_from(g)
    deg = 3
    f0 = O.render(x, deg, plan, BG)
    margins = min(min(float(v["margin"].min()), float(v["margin_grad"].min())) for v in f0["views"])
    if margins < 1e-4:
        pytest.skip("draw has a near-threshold pixel decision")
    W = smooth_weights(seed + 100, plan.cams)
    grad = O.backward(x, deg, plan, f0, W, BG)["dparams"]
    h = 1e-6
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for j in range(x.shape[1]):
            xp = x.copy(); xp[i, j] += h
            xm = x.copy(); xm[i, j] -= h
            fd[i, j] = (loss_and_grad(O, xp, deg, plan, W)[0] - loss_and_grad(O, xm, deg, plan, W)[0]) / (2 * h)
    groups = O.split_params(np.arange(x.shape[1])[None, :].repeat(1, 0), deg)
    for name, cols in groups.items():
        cols = np.asarray(cols).reshape(-1)
        a, b = grad[:, cols], fd[:, cols]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel <= 1e-6, (name, rel)
    assert np.abs(fd).max() > 1e-3          # the problem is not trivial


def test_record_gradient_by_differences(oracle):
    """The compositing adjoint alone: perturb each projected record entry
    (mean2d, conic, opacity, colour) and difference the rendered loss."""
    O = oracle
    g, plan = subproblem(O, 13)
    x = O.params_from(g)
    f0 = O.render(x, 3, plan, BG)
    W = smooth_weights(7, plan.cams)
    drec = O.rasterize_bwd(f0["proj"], f0["bins"], plan, W, BG)
    cols = [O.REC_MX, O.REC_MY, O.REC_A, O.REC_B, O.REC_C, O.REC_OP, O.REC_R, O.REC_G, O.REC_BL]
    h = 1e-7
    rng = np.random.default_rng(0)
    rows = rng.choice(f0["proj"]["rec"].shape[0], 30, replace=False)
    for r in rows:
        if f0["proj"]["rec"][r, O.REC_VIS] != 1:
            continue
        for k, c in enumerate(cols):
            vals = []
            for s in (+1, -1):
                proj = {kk: vv.copy() for kk, vv in f0["proj"].items()}
                proj["rec"][r, c] += s * h
                vs = O.rasterize_fwd(proj, f0["bins"], plan, BG)
                vals.append(sum(float((w * v["image"]).sum()) for w, v in zip(W, vs)))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert drec[r, k] == pytest.approx(fd, rel=2e-5, abs=2e-6), (r, k)
