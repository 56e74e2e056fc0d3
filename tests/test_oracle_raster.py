"""Pins of the oracle's binning and compositing (Sec. 3.1, Eq. 2)."""
import math

import numpy as np
import pytest

from paper_2405_13943_b300 import synth as S


def one(mean, log_scale, ologit, colour, quat=(1, 0, 0, 0)):
    Y00 = 0.5 / math.sqrt(math.pi)
    sh = ((np.asarray(colour, np.float64) - 0.5) / Y00).reshape(1, 1, 3)
    return S.Gaussians(np.asarray([mean], np.float32), np.asarray([quat], np.float32),
                       np.asarray([[log_scale] * 3], np.float32), np.asarray([ologit], np.float32),
                       sh.astype(np.float32))


def render1(O, g, cam, tw=16, th=16, bg=(0, 0, 0)):
    plan = O.ViewPlan([cam], [(0, g.n)], tw, th)
    f = O.render(O.params_from(g), g.sh_degree, plan, bg)
    return f, plan


def test_lone_isotropic_gaussian_closed_form(oracle):
    """One isotropic Gaussian (scale sigma) on the optical axis at depth tz,
    opacity o, colour c, black background: pixel = c o exp(-d^2 / (2 s^2)),
    s^2 = (f sigma / tz)^2 + 0.3, wherever 1/255 <= alpha < 0.99 and the pixel's
    tile lies in the Gaussian's tile rectangle; 0 elsewhere."""
    O = oracle
    cam = S.cube_camera(96, 80, f=110.0, distance=4.0)
    sigma, o_logit, c = math.exp(-2.0), 0.4, np.array([0.9, 0.5, 0.2])
    g = one([0.0, 0.0, 0.0], -2.0, o_logit, c)
    f, plan = render1(O, g, cam)
    img = f["views"][0]["image"]
    rec = f["proj"]["rec"][0]
    x0, y0, x1, y1 = f["proj"]["rect"][0]
    o = 1 / (1 + math.exp(-np.float32(o_logit)))
    sig = float(np.float32(sigma))
    s2 = (110.0 * math.exp(float(np.float32(-2.0))) / 4.0) ** 2 + 0.3
    colour = rec[O.REC_R:O.REC_R + 3]
    np.testing.assert_allclose(colour, c, rtol=1e-6)
    want = np.zeros_like(img)
    for py in range(80):
        for px in range(96):
            if not (x0 <= px // 16 < x1 and y0 <= py // 16 < y1):
                continue
            d2 = (px + 0.5 - 48.0) ** 2 + (py + 0.5 - 40.0) ** 2
            a = o * math.exp(-d2 / (2 * s2))
            if a < 1 / 255:
                continue
            want[:, py, px] = colour * min(a, 0.99)
    np.testing.assert_allclose(img, want, atol=1e-14)
    assert sig > 0


def test_occlusion_and_transmittance_stop(oracle):
    """Three wide Gaussians on the axis, the optical axis through a pixel
    centre: alpha_1 = 0.99 (clamped), alpha_2 = 0.98 composited with
    T = 0.01, then T = 2e-4; alpha_3 = 0.6 would give T = 8e-5 < 1e-4, so the
    third is not composited and the pixel ignores everything behind."""
    O = oracle
    cam = S.cube_camera(129, 129, f=100.0, distance=4.0)
    cam.cx = cam.cy = 64.5
    c1, c2, c3 = [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]
    logit = lambda p: math.log(p / (1 - p))
    parts = [one([0, 0, 0.0], -0.5, 10.0, c1), one([0, 0, 1.0], -0.5, logit(0.98), c2),
             one([0, 0, 2.0], -0.5, logit(0.6), c3)]
    g = S.Gaussians.concat(parts)
    f, _ = render1(O, g, cam)
    v = f["views"][0]
    o2 = 1 / (1 + math.exp(-float(np.float32(logit(0.98)))))
    want = 0.99 * np.array(c1) + o2 * 0.01 * np.array(c2)
    np.testing.assert_allclose(v["image"][:, 64, 64], want, rtol=1e-6, atol=1e-12)
    assert v["T_final"][64, 64] == pytest.approx(0.01 * (1 - o2), rel=1e-12)
    assert v["last"][64, 64] == 2


def test_transmittance_product_no_stop(oracle):
    """Layers that never reach the stop: T_final = prod (1 - alpha_i) and
    C = sum c_i alpha_i prod_{j<i}(1 - alpha_j) + T_final * bg."""
    O = oracle
    cam = S.cube_camera(33, 33, f=100.0, distance=4.0)
    cam.cx = cam.cy = 16.5
    logit = lambda p: math.log(p / (1 - p))
    ps = [0.3, 0.5, 0.2, 0.7]
    cols = [[0.1, 0.2, 0.3], [0.9, 0.1, 0.5], [0.4, 0.4, 0.4], [0.2, 0.8, 0.6]]
    g = S.Gaussians.concat([one([0, 0, 0.5 * i], 0.0, logit(p), c) for i, (p, c) in enumerate(zip(ps, cols))])
    bg = (0.25, 0.5, 0.75)
    f, _ = render1(O, g, cam, bg=bg)
    al = [1 / (1 + math.exp(-float(np.float32(logit(p))))) for p in ps]
    Y00 = 0.5 / math.sqrt(math.pi)
    cols = [np.asarray(np.float32((np.asarray(c) - 0.5) / Y00), np.float64) * Y00 + 0.5 for c in cols]
    T, C = 1.0, np.zeros(3)
    for a, c in zip(al, cols):
        C += np.asarray(c) * a * T
        T *= 1 - a
    C += T * np.asarray(bg)
    v = f["views"][0]
    np.testing.assert_allclose(v["image"][:, 16, 16], C, rtol=1e-12)
    assert v["T_final"][16, 16] == pytest.approx(T, rel=1e-12)
    assert v["last"][16, 16] == 4


def brute_force_view(O, rec, rect, dk, vis, cam, tw, th, bg):
    """One view: per pixel, gather exactly the records whose tile rectangle
    contains the pixel's tile, order them by (float depth, record index) and
    composite front to back.  No keys, no sort of a global list, no ranges.
    A positive exponent (a conic that is not positive definite, or rounding)
    is taken as 0, as the compositing rule states."""
    img = np.zeros((3, cam.height, cam.width))
    n = rec.shape[0]
    for py in range(cam.height):
        for px in range(cam.width):
            tx, ty = px // tw, py // th
            cand = [i for i in range(n) if vis[i] and rect[i, 0] <= tx < rect[i, 2]
                    and rect[i, 1] <= ty < rect[i, 3]]
            cand.sort(key=lambda i: (float(dk[i]), i))
            T, C = 1.0, np.zeros(3)
            for i in cand:
                r = rec[i]
                dx, dy = r[O.REC_MX] - (px + 0.5), r[O.REC_MY] - (py + 0.5)
                pw = -0.5 * (r[O.REC_A] * dx * dx + r[O.REC_C] * dy * dy) - r[O.REC_B] * dx * dy
                pw = min(pw, 0.0)
                a = min(0.99, r[O.REC_OP] * math.exp(pw))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                C += r[O.REC_R:O.REC_R + 3] * a * T
                T *= 1 - a
            img[:, py, px] = C + T * np.asarray(bg)
    return img


def brute_force(O, x, deg, cams, rows, tw, th, bg):
    out = []
    for cam, (b, e) in zip(cams, rows):
        p = O.project(x[b:e], deg, cam, tw, th)
        out.append(brute_force_view(O, p["rec"], p["rect"], p["depth_key"], p["visible"], cam, tw, th, bg))
    return out


def test_tiled_equals_per_pixel_brute_force(oracle):
    """Two views with ragged edges (40x35 and 23x47 pixels, 16x16 and 8x16
    tiles) over different Gaussian ranges."""
    O = oracle
    g = S.cube_scene(60, 77, log_scale_mu=-2.3)
    x = O.params_from(g)
    for tw, th in ((16, 16), (8, 16)):
        cams = [S.cube_camera(40, 35, f=30.0), S.cube_camera(23, 47, f=25.0)]
        rows = [(0, 40), (20, 60)]
        plan = O.ViewPlan(cams, rows, tw, th)
        bg = (0.1, 0.2, 0.3)
        f = O.render(x, 0, plan, bg)
        want = brute_force(O, x, 0, cams, rows, tw, th, bg)
        for v in range(2):
            np.testing.assert_allclose(f["views"][v]["image"], want[v], atol=1e-12)


def test_positive_exponent_is_clamped_not_skipped(oracle):
    """A record whose conic is indefinite (b^2 > a c) has a positive exponent
    at pixels along its negative diagonal: those pairs composite with
    alpha = min(0.99, o), not skipped.  Its mean sits exactly on a pixel
    centre.  The tiled oracle and the brute force agree, and the pixel one
    step down the diagonal shows the clamped alpha."""
    O = oracle
    cam = S.cube_camera(24, 20, f=30.0)
    g = S.cube_scene(12, 5, log_scale_mu=-2.3)
    plan = O.ViewPlan([cam], [(0, 12)], 8, 8)
    x = O.params_from(g)
    proj = O.project_views(x, 0, plan)
    vis = np.nonzero(proj["rec"][:, O.REC_VIS] == 1)[0]
    i = int(vis[0])
    r = proj["rec"][i]
    r[O.REC_MX], r[O.REC_MY] = 10.5, 9.5                # the centre of pixel (10, 9)
    r[O.REC_A], r[O.REC_B], r[O.REC_C] = 0.5, 1.0, 0.5  # indefinite
    r[O.REC_OP] = 0.6
    r[O.REC_R:O.REC_R + 3] = (0.9, 0.4, 0.2)
    proj["depth_key"][i] = np.float32(1e-3)             # in front of every other record
    proj["rect"][i] = (0, 0, 3, 3)                      # every tile of the view
    b = O.bin_sort(proj, plan, cull=False)
    f = O.rasterize_fwd(proj, b, plan)[0]
    want = brute_force_view(O, proj["rec"], proj["rect"], proj["depth_key"], proj["rec"][:, O.REC_VIS] == 1,
                            cam, 8, 8, (0.0, 0.0, 0.0))
    np.testing.assert_allclose(f["image"], want, atol=1e-12)
    # pixel (11, 8): dx = -1, dy = 1, exponent -0.5 (0.5 + 0.5) + 1 = 0.5 > 0 -> alpha = 0.6 in front
    front = 0.6 * np.array([0.9, 0.4, 0.2])
    assert np.all(f["image"][:, 8, 11] >= front - 1e-12)
    assert f["T_final"][8, 11] <= 0.4 + 1e-12


def test_keys_values_ranges_properties(oracle):
    O = oracle
    g = S.cube_scene(300, 9)
    cams = [S.cube_camera(128, 128), S.cube_camera(64, 48, f=60.0)]
    plan = O.ViewPlan(cams, [(0, 300), (100, 250)], 16, 16)
    x = O.params_from(g)
    proj = O.project_views(x, 0, plan)
    b = O.bin_sort(proj, plan, cull=False)
    keys, vals, ranges = b["keys"], b["vals"], b["ranges"]
    # ascending (key, value)
    order = np.lexsort((vals, keys))
    np.testing.assert_array_equal(order, np.arange(len(keys)))
    # every record once per tile of its rectangle, with its depth bits
    vis = proj["rec"][:, O.REC_VIS] == 1
    assert b["M"] == int(proj["rec"][vis, O.REC_TILES].sum())
    # culling keeps a subset: the same list with the unreachable tiles removed
    bc = O.bin_sort(proj, plan)
    assert 0 < bc["M"] < b["M"]
    full = set(zip(keys.tolist(), vals.tolist()))
    assert set(zip(bc["keys"].tolist(), bc["vals"].tolist())) <= full
    for r in np.nonzero(vis)[0][:50]:
        v = proj["view"][r]
        x0, y0, x1, y1 = proj["rect"][r]
        tiles = sorted(plan.tile_off[v] + ty * plan.tiles_x[v] + tx for ty in range(y0, y1) for tx in range(x0, x1))
        mine = sorted((keys[vals == r] >> np.uint64(32)).astype(np.int64).tolist())
        assert mine == tiles
        assert np.all((keys[vals == r] & np.uint64(0xFFFFFFFF)) == proj["depth_key"][r:r + 1].view(np.uint32)[0])
    # ranges partition the sorted list by tile
    assert ranges[0, 0] == 0 and ranges[-1, 1] == len(keys)
    np.testing.assert_array_equal(ranges[1:, 0], ranges[:-1, 1])
    for t in range(plan.n_tiles):
        s, e = ranges[t]
        assert np.all((keys[s:e] >> np.uint64(32)) == t)


def test_empty_scene_gives_background(oracle):
    O = oracle
    g = S.cube_scene(0, 1)
    cam = S.cube_camera(20, 20)
    plan = O.ViewPlan([cam], [(0, 0)], 16, 16)
    f = O.render(O.params_from(g), 0, plan, (0.3, 0.2, 0.1))
    v = f["views"][0]
    np.testing.assert_array_equal(v["image"][0], 0.3)
    np.testing.assert_array_equal(v["T_final"], 1.0)
    assert f["bins"]["M"] == 0


def test_work_counts(oracle):
    """Work counters of the compositing: with the occluding stack above the
    centre pixel examines 3 positions (the third stops it) and composites 2;
    for a lone Gaussian every pixel of its tiles examines 1 position and
    the composited ones are exactly the pixels it colours."""
    O = oracle
    cam = S.cube_camera(129, 129, f=100.0, distance=4.0)
    cam.cx = cam.cy = 64.5
    logit = lambda p: math.log(p / (1 - p))
    g = S.Gaussians.concat([one([0, 0, 0.0], -0.5, 10.0, [1, 0, 0]), one([0, 0, 1.0], -0.5, logit(0.98), [0, 1, 0]),
                            one([0, 0, 2.0], -0.5, logit(0.6), [0, 0, 1])])
    f, plan = render1(O, g, cam)
    cnt = O.rasterize_counts(f["proj"], f["bins"], plan)[0]
    assert (cnt["seen"][64, 64], cnt["used"][64, 64]) == (3, 2)
    assert (cnt["used"] <= cnt["seen"]).all()
    assert (cnt["used"] >= (f["views"][0]["last"] > 0)).all()
    cam1 = S.cube_camera(96, 80, f=110.0, distance=4.0)
    g1 = one([0.0, 0.0, 0.0], -2.0, 0.4, [0.9, 0.5, 0.2])
    f1, plan1 = render1(O, g1, cam1)
    c1 = O.rasterize_counts(f1["proj"], f1["bins"], plan1)[0]
    x0, y0, x1, y1 = f1["proj"]["rect"][0]
    in_rect = np.zeros((80, 96), bool)
    in_rect[y0 * 16:y1 * 16, x0 * 16:x1 * 16] = True
    np.testing.assert_array_equal(c1["seen"], in_rect.astype(np.uint32))
    np.testing.assert_array_equal(c1["used"], (f1["views"][0]["image"].max(0) > 0).astype(np.uint32))


def test_box_qmin_against_dense_sampling(oracle):
    """Minimum of a positive definite quadratic form over a box: never above
    any sampled point of the box, and reached to within the sampling error."""
    O = oracle
    rng = np.random.default_rng(17)
    for _ in range(300):
        L = rng.standard_normal((2, 2)) * rng.uniform(0.01, 2.0)
        Q = L @ L.T + np.eye(2) * 1e-3
        a, b, c = Q[0, 0], Q[0, 1], Q[1, 1]
        X0, Y0 = rng.uniform(-20, 20, 2)
        X1, Y1 = X0 + rng.uniform(0.1, 16), Y0 + rng.uniform(0.1, 16)
        m = O.box_qmin(a, b, c, X0, X1, Y0, Y1)
        xs, ys = np.linspace(X0, X1, 301), np.linspace(Y0, Y1, 301)
        X, Y = np.meshgrid(xs, ys)
        q = a * X * X + 2 * b * X * Y + c * Y * Y
        assert m <= q.min() + 1e-9 * (1 + q.min())
        h = max(X1 - X0, Y1 - Y0) / 300
        assert q.min() - m <= 2 * (abs(a) + abs(b) + abs(c)) * h * (h + 2 * max(abs(X0), abs(X1), abs(Y0), abs(Y1)))
        if X0 <= 0 <= X1 and Y0 <= 0 <= Y1:
            assert m == 0.0


def test_culled_tiles_cannot_reach_the_alpha_cut(oracle):
    """Brute force: for every (record, tile) of its rectangle that binning
    leaves out, every pixel centre of the tile has o exp(-q/2) < 1/255."""
    O = oracle
    g = S.cube_scene(400, 23, log_scale_mu=-2.2)
    cams = [S.cube_camera(96, 80, f=90.0)]
    plan = O.ViewPlan(cams, [(0, g.n)], 16, 16)
    proj = O.project_views(O.params_from(g), 0, plan)
    bc = O.bin_sort(proj, plan)
    kept = set(zip((bc["keys"] >> np.uint64(32)).astype(np.int64).tolist(), bc["vals"].tolist()))
    dropped = 0
    for r in np.nonzero(proj["rec"][:, O.REC_VIS] == 1)[0]:
        rec = proj["rec"][r]
        x0, y0, x1, y1 = proj["rect"][r]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                if (ty * plan.tiles_x[0] + tx, r) in kept:
                    continue
                dropped += 1
                X, Y = np.meshgrid(np.arange(tx * 16, tx * 16 + 16) + 0.5 - rec[O.REC_MX],
                                   np.arange(ty * 16, ty * 16 + 16) + 0.5 - rec[O.REC_MY])
                q = rec[O.REC_A] * X * X + 2 * rec[O.REC_B] * X * Y + rec[O.REC_C] * Y * Y
                assert (rec[O.REC_OP] * np.exp(-0.5 * q)).max() < 1 / 255
    assert dropped > 0


def test_culling_changes_no_image_or_gradient(oracle):
    """Rendering and the adjoint with and without tile culling agree bit for
    bit: the dropped pairs are all below the 1/255 cut."""
    O = oracle
    g = S.cube_scene(600, 29, sh_degree=1, log_scale_mu=-2.4)
    cams = [S.cube_camera(80, 64, f=70.0), S.cube_camera(48, 72, f=50.0)]
    plan = O.ViewPlan(cams, [(0, g.n), (0, g.n)], 16, 16)
    x = O.params_from(g)
    bg = (0.1, 0.2, 0.3)
    fc, fu = O.render(x, 1, plan, bg), O.render(x, 1, plan, bg, cull=False)
    assert fc["bins"]["M"] < fu["bins"]["M"]
    for v, (vc, vu) in enumerate(zip(fc["views"], fu["views"])):
        for k in ("image", "T_final"):
            np.testing.assert_array_equal(vc[k], vu[k])
        # `last` indexes each tile's list, which culling shortens: the record
        # it points at is the same
        for f, vw in ((fc, vc), (fu, vu)):
            H, W_ = vw["last"].shape
            ty, tx = np.meshgrid(np.arange(H) // 16, np.arange(W_) // 16, indexing="ij")
            t = plan.tile_off[v] + ty * plan.tiles_x[v] + tx
            start = f["bins"]["ranges"][t, 0].astype(np.int64)
            pos = np.maximum(start + vw["last"].astype(np.int64) - 1, 0)
            vw["last_rec"] = np.where(vw["last"] > 0, f["bins"]["vals"][pos].astype(np.int64), -1)
        np.testing.assert_array_equal(vc["last_rec"], vu["last_rec"])
        assert (vc["last"] <= vu["last"]).all()
    W = [np.random.default_rng(3 + v).uniform(-1, 1, (3, c.height, c.width)) for v, c in enumerate(cams)]
    bc, bu = O.backward(x, 1, plan, fc, W, bg), O.backward(x, 1, plan, fu, W, bg)
    np.testing.assert_allclose(bc["dparams"], bu["dparams"], rtol=1e-12, atol=1e-15)


def test_threaded_oracle_equals_one_thread(oracle):
    """The oracle's host threads split pixels and Gaussians only: images, T,
    last and the record gradients agree with the one-thread run (the
    gradients up to the order of their FP64 sums)."""
    O = oracle
    g = S.cube_scene(400, 31, sh_degree=2, log_scale_mu=-2.4)
    cams = [S.cube_camera(64, 48, f=60.0), S.cube_camera(40, 56, f=40.0)]
    plan = O.ViewPlan(cams, [(0, 400), (100, 400)], 16, 16)
    x = O.params_from(g)
    W = [np.random.default_rng(2 + v).uniform(-1, 1, (3, c.height, c.width)) for v, c in enumerate(cams)]
    try:
        O.set_threads(1)
        f1 = O.render(x, 2, plan)
        b1 = O.backward(x, 2, plan, f1, W)
        assert O.set_threads(4) in (1, 4)
        f4 = O.render(x, 2, plan)
        b4 = O.backward(x, 2, plan, f4, W)
    finally:
        O.set_threads(1)
    for v in range(2):
        for k in ("image", "T_final", "last"):
            np.testing.assert_array_equal(f1["views"][v][k], f4["views"][v][k])
    np.testing.assert_allclose(b4["dparams"], b1["dparams"], rtol=1e-12, atol=1e-15)
