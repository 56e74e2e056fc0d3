"""GPU parity: every libdogs step against the FP64 oracle on the same seeded
inputs.  Integer stages (tile rectangles, keys, values, ranges, instance
counts) bit-exact; images within 1e-4 max abs per pixel channel; gradients
and ADMM-updated parameters within 1e-3 relative L2 per parameter group.
Inputs are curated by the oracle's decision margins (tests/_util.py): FP32
and FP64 may only disagree where a value sits on a threshold."""
import numpy as np
import pytest
import torch

from paper_2405_13943_b300 import synth as S
from tests._util import curate_gaussians, pixel_mask, report

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
REL_L2 = 1e-3
FLIP_TOL = 2e-2          # one flipped decision moves a pixel by at most ~alpha T |c|
# Pixels whose value decisions lie within relative 1e-4 of a threshold are
# left out of the 1e-4 comparison.  A Gaussian of screen std s puts about
# 2 pi s^2 eps pixels within eps of its 1/255 cut, ~0.1 % of the pixels of
# these scenes at eps = 1e-4; the budget sits just above that.
EXCLUDE_FRAC = 2e-3
# Pixels where the two sides actually differ beyond 1e-4 (a decision taken
# the other way): at most 0.01 % of the pixels, and only where excluded.
FLIP_FRAC = 1e-4
GROUPS = ("means", "quats", "log_scales", "sh", "opacity_logits")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_13943_b300 import build as B
    B.build()
    from paper_2405_13943_b300 import dogs
    return dogs


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def decode_rect(rect):
    r = rect.reshape(-1, 2).astype(np.uint32)
    return np.stack([r[:, 0] & 0xFFFF, r[:, 0] >> 16, r[:, 1] & 0xFFFF, r[:, 1] >> 16], 1).astype(np.int64)


def oracle_params_groups(O, dx, deg):
    gp = O.split_params(dx, deg)
    return {"means": gp["mean"], "quats": gp["quat"], "log_scales": gp["scale"], "sh": gp["sh"],
            "opacity_logits": gp["opacity"]}


def run_pair(D, O, g, cams, rows, blk_off, tw, th, bg, weights_seed=5, thr=1e-4):
    """Forward + backward on both sides.  rows: per view its copy range."""
    xbuf = D.GaussianBuffer.from_synth(g)
    vb = D.ViewBatch(cams, blk_off, tw, th, keep_keys=True)
    D.forward(xbuf, vb, bg)
    torch.cuda.synchronize()
    x = O.params_from(g)
    plan = O.ViewPlan(cams, rows, tw, th)
    f = O.render(x, g.sh_degree, plan, bg)
    masks = pixel_mask(f["views"], thr)
    gmasks = pixel_mask(f["views"], thr, grad=True)
    rng = np.random.default_rng(weights_seed)
    W = [rng.uniform(-1, 1, (3, c.height, c.width)) * m[None] for c, m in zip(cams, gmasks)]
    dimg = torch.zeros_like(vb.image)
    for v, w in enumerate(W):
        vb.view_image(v, dimg).copy_(torch.from_numpy(w.astype(np.float32)))
    grads = xbuf.like()
    D.dg_rasterize_bwd(vb, xbuf, grads, dL_dimage=dimg, bg=bg)
    torch.cuda.synchronize()
    ob = O.backward(x, g.sh_degree, plan, f, W, bg)
    return xbuf, vb, grads, f, ob, masks, plan


def check_forward(D, O, vb, f, masks, plan):
    n_rec = vb.n_rec
    rect_gpu = decode_rect(vb.rect.cpu().numpy()[:2 * n_rec])
    vis_o = f["proj"]["rec"][:, O.REC_VIS] == 1
    vis_g = rect_gpu[:, 2] > rect_gpu[:, 0]
    np.testing.assert_array_equal(vis_g, vis_o)
    np.testing.assert_array_equal(rect_gpu[vis_o], f["proj"]["rect"][vis_o])
    rec = vb.rec.cpu().numpy()[:12 * n_rec].reshape(n_rec, 12)[vis_o]
    orc = f["proj"]["rec"][vis_o]
    np.testing.assert_allclose(rec[:, 0:2], orc[:, 0:2], rtol=0, atol=2e-3)                  # mean2d (px)
    for gi, oi in ((2, O.REC_A), (3, O.REC_B), (4, O.REC_C)):
        assert rel_l2(rec[:, gi], orc[:, oi]) < 1e-4
    np.testing.assert_allclose(rec[:, 5], orc[:, O.REC_OP], atol=1e-5)
    np.testing.assert_allclose(rec[:, [6, 7, 8]], orc[:, [O.REC_R, O.REC_G, O.REC_BL]], atol=1e-5)
    # depth is the key's low word: bit-exact
    np.testing.assert_array_equal(rec[:, 9].astype(np.float32).view(np.uint32),
                                  f["proj"]["depth_key"][vis_o].view(np.uint32))
    M = int(vb.count.item())
    assert M == f["bins"]["M"]
    np.testing.assert_array_equal(vb.keys.cpu().numpy()[:M].view(np.uint64), f["bins"]["keys"])
    np.testing.assert_array_equal(vb.vals.cpu().numpy()[:M].view(np.uint32), f["bins"]["vals"])
    np.testing.assert_array_equal(vb.ranges.cpu().numpy()[:2 * plan.n_tiles].view(np.uint32),
                                  f["bins"]["ranges"].reshape(-1))
    check_work_order(vb.ranges.cpu().numpy().view(np.uint32), plan.n_tiles)
    excluded = flipped = 0
    for v, ov in enumerate(f["views"]):
        img = vb.view_image(v).cpu().numpy()
        m = masks[v]
        excluded += int((~m).sum())
        err = np.abs(img - ov["image"]).max(0)
        flipped += int((err > IMG_TOL).sum())
        assert err[m].max(initial=0.0) <= IMG_TOL, (v, err[m].max())
        # excluded pixels: at most one flipped 1/255-skip or T-stop decision
        assert err[~m].max(initial=0.0) <= FLIP_TOL, (v, err[~m].max())
        Tf = vb.view_pixels(v, vb.T_final).cpu().numpy()
        assert np.abs(Tf - ov["T_final"])[m].max(initial=0.0) <= IMG_TOL
        last = vb.view_pixels(v, vb.last).cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(last[m], ov["last"][m])
    total = sum(c.width * c.height for c in plan.cams)
    report("forward", pixels=total, excluded=excluded, flipped=flipped)
    assert excluded <= max(2, EXCLUDE_FRAC * total), excluded
    assert flipped <= max(1, FLIP_FRAC * total), flipped


def check_work_order(r, n_tiles):
    """The tiles after the ranges: a permutation, by descending instance
    count n in quarter-octave buckets (the leading one of n and the two bits
    after it), empty tiles last."""
    order = r[2 * n_tiles:3 * n_tiles].astype(np.int64)
    np.testing.assert_array_equal(np.sort(order), np.arange(n_tiles))
    cnt = (r[1:2 * n_tiles:2] - r[0:2 * n_tiles:2]).astype(np.int64)[order]
    e = np.array([int(c).bit_length() - 1 for c in cnt])
    top = np.array([(int(c) << 2) >> int(k) if c > 0 else 0 for c, k in zip(cnt, e)])   # 4..7: 1.xx in binary
    mag = np.where(cnt > 0, 4 * e + top, -1)
    assert np.all(np.diff(mag) <= 0)


def check_backward(D, O, g, grads, ob, deg):
    gs = grads.to_synth()
    og = oracle_params_groups(O, ob["dparams"], deg)
    for name in GROUPS:
        a = getattr(gs, name)
        b = og[name]
        r = rel_l2(a, b)
        assert r <= REL_L2, (name, r)


def test_small_single_view_forward_backward(D, oracle):
    """4,096 Gaussians in [-1,1]^3, SH degree 0, 128x128, 16x16 tiles."""
    O = oracle
    cam = S.cube_camera()
    g = curate_gaussians(O, S.cube_scene(4096, 1001), [cam], 16, 16)
    assert g.n > 3900
    xbuf, vb, grads, f, ob, masks, plan = run_pair(D, O, g, [cam], [(0, g.n)], [0, g.n], 16, 16, (0, 0, 0))
    check_forward(D, O, vb, f, masks, plan)
    check_backward(D, O, g, grads, ob, 0)
    check_counts(D, O, vb, f, masks, plan, (0, 0, 0))


def test_clamped_alpha_forward_backward(D, oracle):
    """A third of the Gaussians at opacity 0.9975 (logit 6): near their centres
    o G reaches the 0.99 clamp, which the kernels take in the exponent, and
    the backward's adjoint gives zero d alpha / d power there (those instances
    take its clamp-aware row loop).  Images, T_final, last and gradients
    against the oracle, which clamps alpha = min(0.99, o G) in FP64."""
    O = oracle
    cam = S.cube_camera()
    g = S.cube_scene(3000, 1007)
    g.opacity_logits[::3] = 6.0
    g = curate_gaussians(O, g, [cam], 16, 16)
    xbuf, vb, grads, f, ob, masks, plan = run_pair(D, O, g, [cam], [(0, g.n)], [0, g.n], 16, 16, (0.1, 0.2, 0.3))
    r = f["proj"]["rec"]
    hi = np.nonzero((r[:, O.REC_VIS] == 1) & (r[:, O.REC_OP] > 0.99))[0]
    assert hi.size > 100                                    # clamp-capable instances in view
    # (pixel, instance) pairs with o G >= 0.99 among the pixel centres near those means
    clamped = 0
    for i in hi:
        px = np.floor(r[i, O.REC_MX]) + np.arange(-2, 3) + 0.5
        py = np.floor(r[i, O.REC_MY]) + np.arange(-2, 3) + 0.5
        X, Y = np.meshgrid(px - r[i, O.REC_MX], py - r[i, O.REC_MY])
        G = np.exp(-0.5 * (r[i, O.REC_A] * X * X + 2 * r[i, O.REC_B] * X * Y + r[i, O.REC_C] * Y * Y))
        inside = np.logical_and.outer((py > 0) & (py < cam.height), (px > 0) & (px < cam.width))
        clamped += int(((r[i, O.REC_OP] * G >= 0.99) & inside).sum())
    assert clamped > 50
    check_forward(D, O, vb, f, masks, plan)
    check_backward(D, O, g, grads, ob, 0)


@pytest.mark.parametrize("tw,th", [(16, 16), (32, 8), (8, 32)])
def test_multi_block_multi_view_sh3(D, oracle, tw, th):
    """Three blocks (two views, none, one view), ragged image sizes, SH
    degree 3, non-black background, every tile shape."""
    O = oracle
    g0 = S.cube_scene(900, 42, sh_degree=3, log_scale_mu=-2.6)
    cams = [S.cube_camera(70, 45, f=60.0), S.cube_camera(33, 66, f=40.0), S.cube_camera(128, 50, f=90.0)]
    from scipy.spatial.transform import Rotation
    R = Rotation.from_rotvec([0.1, 0.3, -0.05]).as_matrix().astype(np.float32)
    t = np.array([0.3, -0.1, 4.2], np.float32)
    cams[1] = S.Camera(33, 66, 40.0, 44.0, 15.0, 35.0, R, t, -(R.T @ t), 0.2)
    cams[0].block, cams[1].block, cams[2].block = 0, 0, 2
    # curate per block against that block's views
    parts = [g0.subset(np.arange(0, 400)), g0.subset(np.arange(400, 600)), g0.subset(np.arange(600, 900))]
    parts[0] = curate_gaussians(O, parts[0], cams[:2], tw, th)
    parts[2] = curate_gaussians(O, parts[2], cams[2:], tw, th)
    g = S.Gaussians.concat(parts)
    off = np.cumsum([0] + [p.n for p in parts]).tolist()
    rows = [(off[0], off[1]), (off[0], off[1]), (off[2], off[3])]
    bg = (0.2, 0.1, 0.3)
    xbuf, vb, grads, f, ob, masks, plan = run_pair(D, O, g, cams, rows, off, tw, th, bg)
    check_forward(D, O, vb, f, masks, plan)
    check_backward(D, O, g, grads, ob, 3)
    # copies of the block with no view get exactly zero gradient
    gs = grads.to_synth()
    assert np.all(gs.means[off[1]:off[2]] == 0) and np.all(gs.sh[off[1]:off[2]] == 0)
    check_counts(D, O, vb, f, masks, plan, bg)
    check_binning_without_list(D, vb, f)


def check_binning_without_list(D, vb, f):
    """A workspace below dg_bin_sort_workspace_size (but at least the
    minimum) bins without the visible-record list, scanning every record:
    the same keys, values and ranges, bit for bit, as the oracle's."""
    import ctypes as C
    from paper_2405_13943_b300 import _lib as L
    lib = L.lib()
    full = lib.dg_bin_sort_workspace_size(C.byref(vb.plan), vb.capacity)
    small = lib.dg_bin_sort_workspace_min_size(C.byref(vb.plan), vb.capacity)
    assert 0 < small < full
    ws = torch.zeros(full - 1, dtype=torch.uint8, device=vb.ws.device)     # one byte short of the list
    vb.keys.zero_(); vb.vals.zero_(); vb.ranges.zero_()
    L.check(lib.dg_bin_sort(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), vb.capacity,
                            L.ptr(vb.keys), L.ptr(vb.vals), L.ptr(vb.ranges), L.ptr(vb.count), L.ptr(ws),
                            ws.numel(), L.ptr(vb.status), None), "dg_bin_sort")
    torch.cuda.synchronize()
    M = int(vb.count.item())
    assert M == f["bins"]["M"]
    np.testing.assert_array_equal(vb.keys.cpu().numpy()[:M].view(np.uint64), f["bins"]["keys"])
    np.testing.assert_array_equal(vb.vals.cpu().numpy()[:M].view(np.uint32), f["bins"]["vals"])
    np.testing.assert_array_equal(vb.ranges.cpu().numpy()[:2 * vb.plan.n_tiles].view(np.uint32),
                                  f["bins"]["ranges"].reshape(-1))
    check_work_order(vb.ranges.cpu().numpy().view(np.uint32), vb.plan.n_tiles)
    tiny = torch.zeros(small - 1, dtype=torch.uint8, device=vb.ws.device)
    assert lib.dg_bin_sort(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), vb.capacity,
                           L.ptr(vb.keys), L.ptr(vb.vals), L.ptr(vb.ranges), L.ptr(vb.count), L.ptr(tiny),
                           tiny.numel(), L.ptr(vb.status), None) == L.DG_ERR_WORKSPACE


def check_counts(D, O, vb, f, masks, plan, bg):
    """dg_rasterize_count: the forward's outputs bit for bit, and the pair
    counters equal the oracle's per-pixel work summed (exactly when no pixel
    sits at a decision margin)."""
    before = [t.clone() for t in (vb.image, vb.T_final, vb.last)]
    counts = D.dg_rasterize_count(vb, bg).cpu().numpy()
    for a, b in zip(before, (vb.image, vb.T_final, vb.last)):
        assert torch.equal(a, b)
    oc = O.rasterize_counts(f["proj"], f["bins"], plan)
    seen = sum(int(c["seen"].sum()) for c in oc)
    used = sum(int(c["used"].sum()) for c in oc)
    excluded = sum(int((~m).sum()) for m in masks)
    assert counts[1] <= int(vb.last[:vb.n_pixels].sum()) <= counts[0]
    if excluded == 0:
        assert (counts[0], counts[1]) == (seen, used)
    else:
        assert abs(counts[0] - seen) <= 1e-3 * seen and abs(counts[1] - used) <= 1e-3 * used


# (width, height) per view: odd widths and offsets take the element-wise
# staging of the D-SSIM passes; widths and plane offsets that are multiples of
# four take the 16-byte copies (views 0 and 1 of the second set)
LOSS_VIEWS = [[(75, 41), (40, 64)], [(64, 48), (40, 64), (75, 41), (132, 70)]]


@pytest.mark.parametrize("sizes", LOSS_VIEWS)
def test_losses_match_oracle(D, oracle, sizes):
    O = oracle
    cams = [S.cube_camera(w, h) for w, h in sizes]
    nv = len(cams)
    vb = D.ViewBatch(cams, [0, 0], 16, 16, loss_ws=True)
    imgs = [S.random_image(7 + v, c.height, c.width) for v, c in enumerate(cams)]
    tgts = [np.clip(im + S.random_like(20 + v, im.shape, 0.2), 0, 1) for v, im in enumerate(imgs)]
    target = torch.zeros_like(vb.image)
    for v in range(nv):
        vb.view_image(v).copy_(torch.from_numpy(imgs[v]))
        vb.view_image(v, target).copy_(torch.from_numpy(tgts[v]))
    D.dg_loss_l1(vb, target, 1.0)
    torch.cuda.synchronize()
    for v in range(nv):
        L1, g1 = O.l1(imgs[v], tgts[v])
        assert vb.loss[v].item() == pytest.approx(L1, rel=1e-5)
        assert rel_l2(vb.view_image(v, vb.dL_dimage).cpu().numpy(), g1) < 1e-6
    D.dg_loss_dssim(vb, target, 0.8, 0.2)
    torch.cuda.synchronize()
    for v in range(nv):
        Ld, gd = O.dssim_loss(imgs[v], tgts[v], 0.2)
        assert vb.loss[v].item() == pytest.approx(Ld, rel=1e-5)
        assert rel_l2(vb.view_image(v, vb.dL_dimage).cpu().numpy(), gd) < REL_L2


def random_admm_problem(seed, n_pts=3000, deg=3):
    rng = np.random.default_rng(seed)
    xy = rng.uniform(0, 100, (n_pts, 2))
    split, order = S.block_split(xy, 2, 2, [0.3, 0.2, 0.35, 0.15], 0.1)
    base = S.cube_scene(n_pts, seed, sh_degree=deg).subset(order)
    x = base.subset(split.copy_gid)
    # copies drift apart; duals on shared copies only
    pert = lambda a, s: (a + S.random_like(seed + s, a.shape, 0.05)).astype(np.float32)
    x = S.Gaussians(pert(x.means, 1), pert(x.quats, 2), pert(x.log_scales, 3), pert(x.opacity_logits, 4), pert(x.sh, 5))
    sh = split.copy_shared().astype(bool)
    u = S.Gaussians(*(pert(np.zeros_like(a), 10 + i) * np.where(sh, 1, 0).reshape((-1,) + (1,) * (a.ndim - 1))
                      for i, a in enumerate((x.means, x.quats, x.log_scales, x.opacity_logits, x.sh))))
    return split, base, x, u


def consensus_case(D, O, alpha, seed):
    split, z0, x, u = random_admm_problem(seed)
    deg = 3
    dev = "cuda"
    xb, ub = D.GaussianBuffer.from_synth(x), D.GaussianBuffer.from_synth(u)
    zb = D.GaussianBuffer.from_synth(z0)
    an = xb.like()
    g_off = torch.from_numpy(split.g_off).to(dev)
    g_cp = torch.from_numpy(split.g_copies).to(dev)
    res = torch.zeros(10, dtype=torch.float64, device=dev)
    rho = [2.0, 3.0, 5.0, 7.0, 11.0]
    D.dg_admm_consensus(xb, ub, zb, an, g_off, g_cp, rho, alpha, res)
    torch.cuda.synchronize()
    ox, ou, oz = O.params_from(x), O.params_from(u), O.params_from(z0)
    ores = O.consensus(ox, ou, oz, split.g_off, split.g_copies, deg, alpha=alpha, rho=rho)
    zg, ug, ag = zb.to_synth(), ub.to_synth(), an.to_synth()
    oz_g = oracle_params_groups(O, oz, deg)
    ou_g = oracle_params_groups(O, ou, deg)
    for name in GROUPS:
        assert rel_l2(getattr(zg, name), oz_g[name]) < REL_L2, ("z", name)
        assert rel_l2(getattr(ug, name), ou_g[name]) < REL_L2, ("u", name)
    # anchor = z[gid] - u on shared copies
    sh = split.copy_shared().astype(bool)
    for name in GROUPS:
        want = oz_g[name][split.copy_gid[sh]] - ou_g[name][sh]
        assert rel_l2(getattr(ag, name)[sh], want) < REL_L2, ("anchor", name)
    np.testing.assert_allclose(res.cpu().numpy(), ores, rtol=1e-3)
    return split


@pytest.mark.parametrize("alpha", [1.0, 1.6])
def test_consensus_matches_oracle(D, oracle, alpha):
    consensus_case(D, oracle, alpha, 3)


def test_adam_admm_step_matches_oracle(D, oracle):
    O = oracle
    split, z0, x, u = random_admm_problem(9)
    deg = 3
    dev = "cuda"
    n = x.n
    grad = S.Gaussians(*(S.random_like(40 + i, a.shape, 0.3) for i, a in
                         enumerate((x.means, x.quats, x.log_scales, x.opacity_logits, x.sh))))
    m0 = S.Gaussians(*(S.random_like(50 + i, a.shape, 0.01) for i, a in
                       enumerate((x.means, x.quats, x.log_scales, x.opacity_logits, x.sh))))
    v0 = S.Gaussians(*(np.abs(S.random_like(60 + i, a.shape, 0.01)) for i, a in
                       enumerate((x.means, x.quats, x.log_scales, x.opacity_logits, x.sh))))
    xb, gb, mb, vb_ = (D.GaussianBuffer.from_synth(a) for a in (x, grad, m0, v0))
    ub, zb = D.GaussianBuffer.from_synth(u), D.GaussianBuffer.from_synth(z0)
    an = xb.like()
    gid = torch.from_numpy(split.copy_gid).to(dev)
    shared = torch.from_numpy(split.copy_shared()).to(dev)
    D.dg_admm_anchor(zb, ub, gid, shared, an)
    rho = [1e4, 1e4, 1e4, 1e3, 1e4]          # the paper's penalties
    lr = [1.6e-4, 1e-3, 5e-3, 2.5e-3, 1.25e-4, 5e-2]
    D.dg_adam_admm_step(xb, gb, mb, vb_, an, shared, rho, lr, 0.9, 0.999, 1e-15, 3)
    torch.cuda.synchronize()
    ox, og, om, ov = (O.params_from(a) for a in (x, grad, m0, v0))
    oz, ou = O.params_from(z0), O.params_from(u)
    O.adam_admm_step(ox, og, om, ov, oz, ou, split.copy_gid, split.copy_shared(), rho, lr, deg, 0.9, 0.999, 1e-15, 3)
    for buf, ref in ((xb, ox), (mb, om), (vb_, ov)):
        got = buf.to_synth()
        want = oracle_params_groups(O, ref, deg)
        for name in GROUPS:
            assert rel_l2(getattr(got, name), want[name]) < REL_L2, name
    assert torch.all(xb.pad_lane() == 0)


def test_empty_scene_and_capacity_overflow(D, oracle):
    O = oracle
    cam = S.cube_camera(48, 40)
    bg = (0.3, 0.2, 0.1)
    # no Gaussians at all
    g0 = S.cube_scene(0, 1)
    xb = D.GaussianBuffer.from_synth(g0)
    vb = D.ViewBatch([cam], [0, 0], 16, 16)
    D.forward(xb, vb, bg)
    img = vb.view_image(0).cpu().numpy()
    assert np.all(img[0] == np.float32(0.3)) and np.all(img[2] == np.float32(0.1))
    # capacity overflow: ranges emptied, status raised, then a retry renders right
    g = curate_gaussians(O, S.cube_scene(500, 8, log_scale_mu=-2.0), [cam], 16, 16)
    xb = D.GaussianBuffer.from_synth(g)
    vb = D.ViewBatch([cam], [0, g.n], 16, 16, capacity=10)
    D.forward(xb, vb, bg, retry=False)
    torch.cuda.synchronize()
    assert int(vb.status.item()) & 1
    assert int(vb.count.item()) > 10
    assert np.all(vb.ranges.cpu().numpy()[:2 * vb.n_tiles] == 0)
    D.forward(xb, vb, bg, retry=True)
    f = O.render(O.params_from(g), 0, O.ViewPlan([cam], [(0, g.n)], 16, 16), bg)
    m = f["views"][0]["margin"] >= 1e-4
    err = np.abs(vb.view_image(0).cpu().numpy() - f["views"][0]["image"]).max(0)
    assert err[m].max() <= IMG_TOL


def test_binning_is_deterministic(D):
    cam = S.cube_camera()
    g = S.cube_scene(4096, 77)
    xb = D.GaussianBuffer.from_synth(g)
    vb = D.ViewBatch([cam], [0, g.n], 16, 16, keep_keys=True)
    outs = []
    for _ in range(3):
        D.forward(xb, vb)
        torch.cuda.synchronize()
        outs.append((vb.vals.clone(), vb.image.clone()))
    for v, im in outs[1:]:
        assert torch.equal(v, outs[0][0]) and torch.equal(im, outs[0][1])


def test_autograd_function_matches_direct_calls(D):
    cam = S.cube_camera()
    g = S.cube_scene(2000, 5)
    xb = D.GaussianBuffer.from_synth(g)
    vb = D.ViewBatch([cam], [0, g.n], 16, 16)
    data = xb.data.detach().requires_grad_(True)
    xb2 = D.GaussianBuffer(g.n, 0, "cuda", xb.ld, data)
    img = D.RasterizeFn.apply(data, xb2, vb, (0, 0, 0))
    w = torch.from_numpy(S.random_like(3, tuple(img.shape))).cuda()
    (img * w).sum().backward()
    grads = xb.like()
    D.dg_rasterize_bwd(vb, xb, grads, dL_dimage=torch.cat([w, torch.zeros(vb.image.numel() - w.numel(), device="cuda")]))
    torch.cuda.synchronize()
    assert torch.allclose(data.grad, grads.data, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("warps", [1, 2, 4, 8])
@pytest.mark.parametrize("stage", [1, 2])
def test_every_compositing_variant_matches_oracle(D, oracle, warps, stage):
    """Each compositing variant (warps per tile, instances staged per thread)
    against the oracle: same images (the per-pixel sequence does not depend
    on the variant) and gradients within tolerance, on a two-view scene with
    lists longer than one staging round."""
    O = oracle
    cams = [S.cube_camera(90, 70, f=80.0), S.cube_camera(64, 64, f=60.0)]
    g = curate_gaussians(O, S.cube_scene(3000, 91, sh_degree=2, log_scale_mu=-2.4), cams, 16, 16)
    D.set_raster_variant(warps, stage)
    try:
        xbuf, vb, grads, f, ob, masks, plan = run_pair(D, O, g, cams, [(0, g.n), (0, g.n)], [0, g.n], 16, 16,
                                                       (0.05, 0.1, 0.15))
        assert (vb.plan.raster_warps, vb.plan.raster_stage) == (warps, stage)
        check_forward(D, O, vb, f, masks, plan)
        check_backward(D, O, g, grads, ob, 2)
        check_counts(D, O, vb, f, masks, plan, (0.05, 0.1, 0.15))
    finally:
        D.set_raster_variant(4, 2)


@pytest.mark.parametrize("fwd,bwd", [((2, 1), (1, 1)), ((1, 2), (4, 1))])
def test_separate_backward_variant(D, oracle, fwd, bwd):
    """The backward runs its own variant (plan.raster_warps_bwd /
    raster_stage_bwd) and still matches the oracle."""
    O = oracle
    cams = [S.cube_camera(90, 70, f=80.0), S.cube_camera(64, 64, f=60.0)]
    g = curate_gaussians(O, S.cube_scene(3000, 93, sh_degree=1, log_scale_mu=-2.4), cams, 16, 16)
    D.set_raster_variant(*fwd, *bwd)
    try:
        xbuf, vb, grads, f, ob, masks, plan = run_pair(D, O, g, cams, [(0, g.n), (0, g.n)], [0, g.n], 16, 16,
                                                       (0.05, 0.1, 0.15))
        p = vb.plan
        assert (p.raster_warps, p.raster_stage, p.raster_warps_bwd, p.raster_stage_bwd) == (*fwd, *bwd)
        check_forward(D, O, vb, f, masks, plan)
        check_backward(D, O, g, grads, ob, 1)
    finally:
        D.set_raster_variant(4, 2)


def test_consensus_with_many_copies_per_global(D, oracle):
    """Globals held by 1 to 7 blocks: the batched fast path (up to four
    copies) and the generic path (more) against the oracle."""
    O = oracle
    rng = np.random.default_rng(21)
    n_glob, K = 600, 8
    members = [np.sort(rng.choice(K, rng.integers(1, 8), replace=False)) for _ in range(n_glob)]
    gid = np.array([i for k in range(K) for i in range(n_glob) if k in members[i]], np.int32)
    g_cp = np.argsort(gid, kind="stable").astype(np.int32)
    g_off = np.concatenate([[0], np.cumsum(np.bincount(gid, minlength=n_glob))]).astype(np.int64)
    base = S.cube_scene(n_glob, 5, sh_degree=1)
    x = base.subset(gid)
    jit = lambda a, s: (a + S.random_like(s, a.shape, 0.1)).astype(np.float32)
    x = S.Gaussians(jit(x.means, 1), jit(x.quats, 2), jit(x.log_scales, 3), jit(x.opacity_logits, 4), jit(x.sh, 5))
    u = S.Gaussians(*(S.random_like(10 + i, a.shape, 0.05) for i, a in
                      enumerate((x.means, x.quats, x.log_scales, x.opacity_logits, x.sh))))
    xb, ub, zb = D.GaussianBuffer.from_synth(x), D.GaussianBuffer.from_synth(u), D.GaussianBuffer.from_synth(base)
    an = xb.like()
    res = torch.zeros(10, dtype=torch.float64, device="cuda")
    rho = [1.0, 2.0, 3.0, 4.0, 5.0]
    D.dg_admm_consensus(xb, ub, zb, an, torch.from_numpy(g_off).cuda(), torch.from_numpy(g_cp).cuda(), rho, 1.4, res)
    torch.cuda.synchronize()
    ox, ou, oz = O.params_from(x), O.params_from(u), O.params_from(base)
    ores = O.consensus(ox, ou, oz, g_off, g_cp, 1, alpha=1.4, rho=rho)
    zg, ug = zb.to_synth(), ub.to_synth()
    oz_g, ou_g = oracle_params_groups(O, oz, 1), oracle_params_groups(O, ou, 1)
    for name in GROUPS:
        assert rel_l2(getattr(zg, name), oz_g[name]) < REL_L2, ("z", name)
        assert rel_l2(getattr(ug, name), ou_g[name]) < REL_L2, ("u", name)
    np.testing.assert_allclose(res.cpu().numpy(), ores, rtol=1e-3)
    assert np.diff(g_off).max() > 4


def test_scale_duals_matches_oracle(D, oracle):
    """Eq. 10's rescale of the scaled duals: shared copies scale by the
    per-group factor, the rest stay untouched, padding lanes stay zero."""
    O = oracle
    split, z0, x, _ = random_admm_problem(12)
    deg = 3
    # nonzero values on every copy, to see that the non-shared ones stay put
    u = S.Gaussians(*(S.random_like(70 + i, a.shape, 0.5) for i, a in
                      enumerate((x.means, x.quats, x.log_scales, x.opacity_logits, x.sh))))
    ub = D.GaussianBuffer.from_synth(u)
    shared = torch.from_numpy(split.copy_shared()).to("cuda")
    factor = [2.0, 0.5, 0.3, 1.0, 4.0 / 3.0]
    D.dg_admm_scale_duals(ub, shared, factor)
    torch.cuda.synchronize()
    ou = O.params_from(u)
    O.scale_duals(ou, split.copy_shared(), factor, deg)
    got = ub.to_synth()
    want = oracle_params_groups(O, ou, deg)
    for name in GROUPS:
        np.testing.assert_allclose(getattr(got, name), want[name], rtol=1e-6, atol=0, err_msg=name)
    assert torch.all(ub.pad_lane() == 0)


def test_fused_backward_xstep_matches_oracle(D, oracle):
    """dg_backward_xstep (adjoint and Adam + penalty step in one pass) equals
    the oracle's backward followed by its x-step, on blocks with one view
    each (one with none), shared and unshared copies, SH degree 3."""
    O = oracle
    g0 = S.cube_scene(700, 44, sh_degree=3, log_scale_mu=-2.6)
    cams = [S.cube_camera(70, 45, f=60.0), S.cube_camera(128, 50, f=90.0)]
    cams[0].block, cams[1].block = 0, 2
    parts = [curate_gaussians(O, g0.subset(np.arange(0, 300)), cams[:1], 16, 16), g0.subset(np.arange(300, 450)),
             curate_gaussians(O, g0.subset(np.arange(450, 700)), cams[1:], 16, 16)]
    g = S.Gaussians.concat(parts)
    off = np.cumsum([0] + [p.n for p in parts]).tolist()
    rows = [(off[0], off[1]), (off[2], off[3])]
    bg = (0.2, 0.1, 0.3)
    deg, n = 3, g.n
    xbuf = D.GaussianBuffer.from_synth(g)
    vb = D.ViewBatch(cams, off, 16, 16)
    assert D.one_view_per_block(vb.plan)
    D.forward(xbuf, vb, bg)
    torch.cuda.synchronize()
    x = O.params_from(g)
    plan = O.ViewPlan(cams, rows, 16, 16)
    f = O.render(x, deg, plan, bg)
    gmasks = pixel_mask(f["views"], 1e-4, grad=True)
    rng = np.random.default_rng(6)
    W = [rng.uniform(-1, 1, (3, c.height, c.width)) * m[None] for c, m in zip(cams, gmasks)]
    dimg = torch.zeros_like(vb.image)
    for v, w in enumerate(W):
        vb.view_image(v, dimg).copy_(torch.from_numpy(w.astype(np.float32)))
    ob = O.backward(x, deg, plan, f, W, bg)
    # optimiser state, duals and the sharing flags
    like = lambda seed, s: S.Gaussians(*(S.random_like(seed + i, a.shape, s) for i, a in
                                         enumerate((g.means, g.quats, g.log_scales, g.opacity_logits, g.sh))))
    m0 = like(50, 0.01)
    v0 = S.Gaussians(*(np.abs(a) for a in (lambda t: (t.means, t.quats, t.log_scales, t.opacity_logits, t.sh))(like(60, 0.01))))
    z0, u0 = like(70, 0.5), like(80, 0.05)
    shared = (rng.uniform(size=n) < 0.4).astype(np.uint8)
    mb, vb_, zb, ub = (D.GaussianBuffer.from_synth(a) for a in (m0, v0, z0, u0))
    gid = torch.arange(n, dtype=torch.int32, device="cuda")
    sh_t = torch.from_numpy(shared).cuda()
    an = xbuf.like()
    D.dg_admm_anchor(zb, ub, gid, sh_t, an)
    rho = [1e4, 1e4, 1e4, 1e3, 1e4]
    lr = [1.6e-4, 1e-3, 5e-3, 2.5e-3, 1.25e-4, 5e-2]
    D.dg_backward_xstep(vb, xbuf, mb, vb_, an, sh_t, rho, lr, 0.9, 0.999, 1e-15, 3, bg=bg, dL_dimage=dimg)
    torch.cuda.synchronize()
    ox, om, ov = x.copy(), O.params_from(m0), O.params_from(v0)
    O.adam_admm_step(ox, ob["dparams"], om, ov, O.params_from(z0), O.params_from(u0), np.arange(n),
                     shared, rho, lr, deg, 0.9, 0.999, 1e-15, 3)
    for buf, ref in ((xbuf, ox), (mb, om), (vb_, ov)):
        got = buf.to_synth()
        want = oracle_params_groups(O, ref, deg)
        for name in GROUPS:
            assert rel_l2(getattr(got, name), want[name]) < REL_L2, name
    assert torch.all(xbuf.pad_lane() == 0)


def test_fused_xstep_rejects_blocks_with_several_views(D):
    cams = [S.cube_camera(32, 32), S.cube_camera(32, 32)]
    g = S.cube_scene(50, 3)
    xbuf = D.GaussianBuffer.from_synth(g)
    vb = D.ViewBatch(cams, [0, g.n], 16, 16)
    assert not D.one_view_per_block(vb.plan)
    with pytest.raises(Exception):
        D.dg_backward_xstep(vb, xbuf, xbuf.like(), xbuf.like(), None, None, [1.0] * 5, [1e-3] * 6)
