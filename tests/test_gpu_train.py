"""Batched K-block DOGS iterations: the single-launch batched path equals K
independent per-block runs with a gather/scatter consensus (the paper's
distributed semantics, Alg. 2, restated on one device), and CUDA-graph
replays equal eager launches."""
import numpy as np
import pytest
import torch

from paper_2405_13943_b300 import synth as S

pytestmark = pytest.mark.gpu

REL_L2 = 1e-3


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_13943_b300 import build as B
    B.build()
    from paper_2405_13943_b300 import dogs, serve, trainer
    return dogs, serve, trainer


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def small_setup(D, srv, seed=7):
    wl = S.dogs_workload(40_000, 2, 2, 0.1, seed, views_per_step=1, pool=2, width=200, height=150)
    z0 = D.GaussianBuffer.from_synth(wl.z0)
    gt = D.GaussianBuffer.from_synth(wl.gt)
    targets = [srv.render_views(gt, vs).image.clone() for vs in wl.views]
    return wl, z0, targets


def groups(buf):
    s = buf.to_synth()
    return {k: getattr(s, k) for k in ("means", "quats", "log_scales", "sh", "opacity_logits")}


def test_batched_equals_sequential_per_block(mods):
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv)
    kw = dict(rho=(1e-2,) * 5, loss="dssim", intv=2)
    bt = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, **kw)
    bt.calibrate_capacity()
    sq = T.SequentialTrainer(wl.split, z0.clone(), wl.views, targets, **kw)
    sq.calibrate_capacity()
    for _ in range(4):                 # consensus at t = 0 and t = 2
        bt.step(graph=False)
        sq.step()
    torch.cuda.synchronize()
    assert not bt.overflowed()
    # gather the sequential copies into the batched layout
    x_seq = bt.x.like()
    for blk in sq.blocks:
        sq._copy_rows(x_seq, blk["x"], blk["b"], blk["e"], True)
    gb, gs = groups(bt.x), groups(x_seq)
    for k in gb:
        assert rel_l2(gs[k], gb[k]) < REL_L2, k
    zb, zs = groups(bt.z), groups(sq.z)
    for k in zb:
        assert rel_l2(zs[k], zb[k]) < REL_L2, k
    # the copies moved away from their start
    g0 = groups(T.gather_copies(z0, bt.gid))
    assert rel_l2(gb["means"], g0["means"]) > 0


def test_graph_replay_equals_eager(mods):
    """Graph replays launch exactly the eager sequence.  Each iteration starts
    both trainers from the same state (the eager one gets a copy of the
    graph one's buffers), then compares: identical images, gradients and
    updated parameters equal up to the order of the float atomics.  Covers
    both pool entries and iterations with and without the consensus."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=8)
    kw = dict(rho=(1e-3,) * 5, loss="l1", intv=3)
    a = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, **kw)
    b = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, **kw)
    a.calibrate_capacity()
    b.vb.set_capacity(a.vb.capacity)
    for _ in range(4):
        for f in ("x", "m", "v", "u", "z", "anchor"):
            getattr(b, f).copy_(getattr(a, f))
        a.step(graph=True)
        b.step(graph=False)
        torch.cuda.synchronize()
        assert torch.equal(a.vb.image, b.vb.image)
        assert rel_l2(a.grad.data.cpu().numpy(), b.grad.data.cpu().numpy()) < 1e-5
        assert rel_l2(a.x.data.cpu().numpy(), b.x.data.cpu().numpy()) < 1e-6
        assert torch.allclose(a.vb.loss, b.vb.loss, rtol=1e-6)


def test_consensus_keeps_dual_mean_zero(mods):
    """After a consensus the duals of every shared global average to zero
    (Appendix, proof of Eq. 8b), so the complete and simplified z agree."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=9)
    tr = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, rho=(1e-2,) * 5, loss="l1", intv=1)
    tr.calibrate_capacity()
    for _ in range(3):
        tr.step(graph=False)
    torch.cuda.synchronize()
    u = groups(tr.u)["means"].astype(np.float64)
    x = groups(tr.x)["means"].astype(np.float64)
    z = groups(tr.z)["means"].astype(np.float64)
    sp = wl.split
    cnt = np.diff(sp.g_off)
    for i in np.nonzero(cnt > 1)[0][:2000]:
        cp = sp.g_copies[sp.g_off[i]:sp.g_off[i + 1]]
        assert np.abs(u[cp].mean(0)).max() < 1e-4
        assert np.abs(z[i] - (x[cp] + 0 * u[cp]).mean(0)).max() < 1e-3 * max(1.0, np.abs(z[i]).max())


def test_adaptive_penalty_follows_eq10(mods):
    """Adaptive penalty in the batched trainer, on the device inside the
    captured graphs: after each consensus before the freeze, rho is the
    oracle's Eq. 10 applied to the residuals that consensus produced, with no
    host read in between."""
    D, srv, T = mods
    from oracle import oracle as O
    from paper_2405_13943_b300.admm import AdaptivePenalty
    wl, z0, targets = small_setup(D, srv, seed=11)
    rho0 = (1e-4, 1.0, 1e-4, 10.0, 1e-3)
    ap = AdaptivePenalty(rho0, freeze_after=6)
    bt = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, rho=rho0, loss="l1", intv=2, adaptive=ap)
    bt.calibrate_capacity()
    changed = 0
    for t in range(10):
        before = bt.current_rho()
        bt.step(graph=True)
        torch.cuda.synchronize()
        after = bt.current_rho()
        if t % 2 == 0:
            want = O.adaptive_rho(before, bt.residuals.cpu().numpy(), t, freeze_after=6)
            assert after == pytest.approx(want, rel=1e-6), t
            changed += after != before
        else:
            assert after == before
    assert changed >= 1              # the deliberately unbalanced start moves rho
    assert bt.rho == list(ap.rho) and len(bt.graphs) <= 4      # rho changes drop no graph
    assert not bt.overflowed()


def test_device_rescale_keeps_the_unscaled_duals(mods):
    """dg_admm_adapt + dg_admm_rescale after a consensus: the unscaled duals
    rho * u of the shared copies are unchanged by the rescale, and the
    anchors are z - u afterwards."""
    D, srv, T = mods
    from oracle import oracle as O
    from paper_2405_13943_b300.admm import AdaptivePenalty
    wl, z0, targets = small_setup(D, srv, seed=11)
    rho0 = (1e-4, 1.0, 1e-4, 10.0, 1e-3)
    ap = AdaptivePenalty(rho0, freeze_after=6)
    bt = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, rho=rho0, loss="l1", intv=1, adaptive=ap)
    bt.calibrate_capacity()
    sh = wl.split.copy_shared().astype(bool)
    deg = z0.deg
    grp = np.array([0] * 3 + [1] * 4 + [2] * 3 + [3] * (3 * (deg + 1) ** 2) + [4])
    rescaled = 0
    for t in range(4):
        before = bt.current_rho()
        bt.adaptive, saved = None, bt.adaptive          # the iteration and its consensus, no Eq. 10
        bt.step(graph=False)
        bt.adaptive = saved
        u_before = O.params_from(bt.u.to_synth())
        D.dg_admm_adapt(bt.residuals, bt.rho_dev, bt.factor_dev, bt.dev_step, ap.mu, ap.tau_inc, ap.tau_dec,
                        ap.freeze_after)
        D.dg_admm_rescale(bt.u, bt.z, bt.anchor, bt.gid, bt.shared, bt.factor_dev)
        torch.cuda.synchronize()
        after = bt.current_rho()
        rescaled += after != before
        u_after = O.params_from(bt.u.to_synth())
        y0 = u_before[sh] * np.array(before)[grp]
        y1 = u_after[sh] * np.array(after)[grp]
        np.testing.assert_allclose(y1, y0, rtol=1e-6, atol=1e-30)
        an = O.params_from(bt.anchor.to_synth())
        zz = O.params_from(bt.z.to_synth())
        np.testing.assert_allclose(an[sh], zz[wl.split.copy_gid[sh]] - u_after[sh], rtol=1e-5, atol=1e-6)
    assert rescaled >= 1


def test_training_on_a_recursive_split(mods):
    """Blocks from Alg. 1 (K = 3, not a power of two, s = 1.4) train through
    the batched path exactly as through the per-block path, and the
    iterations lower the loss."""
    D, srv, T = mods
    from paper_2405_13943_b300 import scene_split as SS
    z = S.city_scene(30_000, 21, sh_degree=1)
    gt = D.GaussianBuffer.from_synth(S.city_scene(30_000, 22, sh_degree=1, layout_seed=21))
    cams = S.grid_cameras(23, n_side=4, size=1000.0, width=160, height=120)
    split, z, view_sets = SS.make_blocks(z, cams, 3, 1.4, views_per_step=2, pool=2)
    assert split.K == 3 and split.n_shared_globals > 0
    targets = [srv.render_views(gt, vs).image.clone() for vs in view_sets]
    z0 = D.GaussianBuffer.from_synth(z)
    kw = dict(rho=(1e-2,) * 5, loss="l1", intv=2)
    bt = T.DogsTrainer(split, z0.clone(), view_sets, targets, **kw)
    bt.calibrate_capacity()
    sq = T.SequentialTrainer(split, z0.clone(), view_sets, targets, **kw)
    sq.calibrate_capacity()
    for _ in range(4):
        bt.step(graph=False)
        sq.step()
    torch.cuda.synchronize()
    x_seq = bt.x.like()
    for blk in sq.blocks:
        sq._copy_rows(x_seq, blk["x"], blk["b"], blk["e"], True)
    gb, gs = groups(bt.x), groups(x_seq)
    for k in gb:
        assert rel_l2(gs[k], gb[k]) < REL_L2, k
    first = None
    for t in range(40):
        bt.step(graph=True)
        if t % 2 == 1:
            torch.cuda.synchronize()
            cur = float(bt.vb.loss.sum())
            first = cur if first is None else first
    assert not bt.overflowed()
    assert cur < first


def test_checkpoint_resume(mods, tmp_path):
    """A run saved after 3 iterations and loaded into a fresh trainer holds
    the saved state bit for bit (anchors included), and 3 more iterations of
    the resumed and of the uninterrupted run agree up to the order of the
    float atomics."""
    D, srv, T = mods
    from paper_2405_13943_b300.admm import AdaptivePenalty
    wl, z0, targets = small_setup(D, srv, seed=13)
    kw = dict(rho=(1e-2, 1e-2, 1e-2, 1e-3, 1e-2), loss="dssim", intv=2)
    a = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, adaptive=AdaptivePenalty(kw["rho"]), **kw)
    a.calibrate_capacity()
    for _ in range(3):
        a.step()
    p = str(tmp_path / "a.ckpt")
    a.save_checkpoint(p)
    saved = {n: getattr(a, n).data.clone() for n in ("z", "x", "u", "m", "v", "anchor")}
    b = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, adaptive=AdaptivePenalty(kw["rho"]), **kw)
    b.calibrate_capacity()
    b.step()                                     # state to be overwritten
    b.load_checkpoint(p)
    for n, t in saved.items():
        assert torch.equal(getattr(b, n).data.view(torch.int32), t.view(torch.int32)), n
    assert (b.t, b.rho, b.adaptive.rho) == (a.t, a.rho, a.adaptive.rho)
    for _ in range(3):
        a.step()
        b.step()
    torch.cuda.synchronize()
    assert b.t == a.t == 6 and b.current_rho() == a.current_rho()
    for buf in ("x", "z", "u"):
        ga, gb = groups(getattr(a, buf)), groups(getattr(b, buf))
        for k in ga:
            assert rel_l2(gb[k], ga[k]) < REL_L2, (buf, k)


def test_fused_xstep_equals_separate_calls(mods):
    """The trainer's fused adjoint + x-step and the two separate calls,
    iteration by iteration from identical state, agree up to the order of the
    float atomics of the compositing adjoint."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=17)
    kw = dict(rho=(1e-2,) * 5, loss="dssim", intv=2)
    a = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, fused=True, **kw)
    a.calibrate_capacity()
    b = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, fused=False, **kw)
    b.calibrate_capacity()
    assert D.one_view_per_block(a.vb.plan)
    for _ in range(3):
        for n in ("x", "m", "v", "u", "z", "anchor"):
            getattr(b, n).copy_(getattr(a, n))
        b.t = a.t
        a.step(graph=False)
        b.step(graph=False)
        torch.cuda.synchronize()
        for n in ("x", "m", "v"):
            ga, gb = groups(getattr(a, n)), groups(getattr(b, n))
            for k in ga:
                assert rel_l2(gb[k], ga[k]) < REL_L2, (n, k)
    assert not a.overflowed()


def test_host_targets_equal_device_targets(mods):
    """Targets kept in pinned host memory and uploaded one step ahead give
    the same iterations as device-resident targets (graph replays queued
    back to back, the step counter advanced on the device)."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=19)
    kw = dict(rho=(1e-2,) * 5, loss="l1", intv=2)
    a = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, **kw)
    a.calibrate_capacity()
    b = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, **kw)
    b.calibrate_capacity()
    b.use_host_targets([t.cpu() for t in targets])
    la, lb = [], []
    for i in range(5):
        a.step()
        la.append(a.vb.loss.cpu().numpy())
        b.step()
        if i > 0:       # the previous step's losses, read while this one runs
            lb.append(b.loss_of(b.t - 2).numpy())
    lb.append(b.last_loss().numpy())
    with pytest.raises(ValueError):
        b.loss_of(b.t - 3)
    torch.cuda.synchronize()
    assert int(a.dev_step.item()) == int(b.dev_step.item()) == 5
    for x_, y_ in zip(la, lb):
        np.testing.assert_allclose(y_, x_, rtol=1e-3)
    for n in ("x", "z"):
        ga, gb = groups(getattr(a, n)), groups(getattr(b, n))
        for k in ga:
            assert rel_l2(gb[k], ga[k]) < REL_L2, (n, k)


def test_split_xstep_equals_one_part(mods):
    """dg_xstep_part: part 1 (groups of 128 copies without a kept record)
    then part 2 (the rest) takes the step of part 0 bit for bit; part 1
    alone leaves the groups with a kept record untouched."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=23)
    tr = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, rho=(1e-2,) * 5, loss="dssim", overlap=False)
    tr.calibrate_capacity()
    tr.step(graph=False)                       # non-zero moments and anchors
    vb = tr.vb
    vb.dev_cams.copy_(tr.cam_pool[tr.t % len(tr.view_sets)])
    D.dg_project(tr.x, vb)
    D.dg_bin_sort(vb)
    D.dg_rasterize_fwd(vb, tr.bg)
    tr._loss(tr.targets[tr.t % len(tr.view_sets)])
    D.dg_rasterize_bwd_records(vb, bg=tr.bg)
    torch.cuda.synchronize()
    st = {n: getattr(tr, n).clone() for n in ("x", "m", "v")}
    args = (tr.anchor, tr.shared, tr.rho, tr.lr)
    one = {n: st[n].clone() for n in st}
    D.dg_xstep_part(0, vb, one["x"], one["m"], one["v"], *args, step=2)
    two = {n: st[n].clone() for n in st}
    D.dg_xstep_part(1, vb, two["x"], two["m"], two["v"], *args, step=2)
    torch.cuda.synchronize()
    rect = vb.rect.view(-1, 2)[:vb.n_rec].cpu().numpy().view(np.uint32)
    kept = np.zeros(wl.split.n_copies, bool)
    vis = (rect[:, 0] & 0xFFFF) != (rect[:, 1] & 0xFFFF)
    for c in vb.host_cams:
        b, e = int(c.gauss_begin), int(c.gauss_end)
        kept[b:e] |= vis[int(c.rec_off):int(c.rec_off) + e - b]
    ng = -(-len(kept) // 128)
    act = np.repeat(np.pad(kept, (0, ng * 128 - len(kept))).reshape(ng, 128).any(1), 128)[:len(kept)]
    assert 0 < act.mean() < 1
    x0, x1 = groups(st["x"]), groups(two["x"])
    for k in x0:
        np.testing.assert_array_equal(x1[k][act], x0[k][act])
        assert not np.array_equal(x1[k][~act], x0[k][~act])
    D.dg_xstep_part(2, vb, two["x"], two["m"], two["v"], *args, step=2)
    torch.cuda.synchronize()
    for n in ("x", "m", "v"):
        assert torch.equal(one[n].data, two[n].data), n


@pytest.mark.parametrize("ctas", [0, 3])
def test_streamed_idle_xstep_equals_part1(mods, ctas):
    """dg_xstep_stream (the groups without a kept record, streamed by
    persistent CTAs through shared memory) takes part 1's step bit for bit,
    with the unshared copies' store into z, and part 2 after it completes
    the one-part step."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=37)
    tr = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, rho=(1e-2,) * 5, loss="dssim", intv=1)
    tr.calibrate_capacity()
    assert tr._zfuse(True)
    tr.step(graph=False)                       # non-zero moments and anchors
    vb = tr.vb
    vb.dev_cams.copy_(tr.cam_pool[tr.t % len(tr.view_sets)])
    D.dg_project(tr.x, vb)
    D.dg_bin_sort(vb)
    D.dg_rasterize_fwd(vb, tr.bg)
    tr._loss(tr.targets[tr.t % len(tr.view_sets)])
    D.dg_rasterize_bwd_records(vb, bg=tr.bg)
    torch.cuda.synchronize()
    args = (tr.anchor, tr.shared, tr.rho, tr.lr)
    ref = {n: getattr(tr, n).clone() for n in ("x", "m", "v", "z")}
    out = {n: getattr(tr, n).clone() for n in ("x", "m", "v", "z")}
    D.dg_xstep_part(1, vb, ref["x"], ref["m"], ref["v"], *args, step=2, z_unshared=ref["z"], gid=tr.gid)
    ws = D.xstep_stream_workspace(tr.x)
    ws.fill_(-1)                               # the call zeroes its own counters
    D.dg_xstep_stream(vb, out["x"], out["m"], out["v"], *args, ws, step=2, ctas=ctas, z_unshared=out["z"],
                      gid=tr.gid)
    torch.cuda.synchronize()
    for n in ref:
        assert torch.equal(ref[n].data, out[n].data), n
    n_groups = -(-tr.x.n // 128)
    n_idle = int(ws[0].item())
    assert 0 < n_idle < n_groups
    listed = ws[4:4 + n_idle].cpu().numpy()
    assert len(np.unique(listed)) == n_idle and listed.min() >= 0 and listed.max() < n_groups
    # a second call with the same workspace takes the next step the same way
    D.dg_xstep_part(1, vb, ref["x"], ref["m"], ref["v"], *args, step=3)
    D.dg_xstep_stream(vb, out["x"], out["m"], out["v"], *args, ws, step=3, ctas=ctas)
    D.dg_xstep_part(2, vb, ref["x"], ref["m"], ref["v"], *args, step=3)
    D.dg_xstep_part(2, vb, out["x"], out["m"], out["v"], *args, step=3)
    torch.cuda.synchronize()
    for n in ("x", "m", "v"):
        assert torch.equal(ref[n].data, out[n].data), n


@pytest.mark.parametrize("ctas", [0, 5])
def test_listed_xstep_equals_one_part(mods, ctas):
    """dg_xstep_groups lists every group of 128 copies once, those without a
    kept record from the front of the workspace's list and the others from
    its back; dg_xstep_listed part 1 then part 2 over those lists takes the
    one-part step bit for bit, with the unshared copies' store into z."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=41)
    tr = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, rho=(1e-2,) * 5, loss="dssim", intv=1)
    tr.calibrate_capacity()
    assert tr._zfuse(True)
    tr.step(graph=False)                       # non-zero moments and anchors
    vb = tr.vb
    vb.dev_cams.copy_(tr.cam_pool[tr.t % len(tr.view_sets)])
    D.dg_project(tr.x, vb)
    D.dg_bin_sort(vb)
    D.dg_rasterize_fwd(vb, tr.bg)
    tr._loss(tr.targets[tr.t % len(tr.view_sets)])
    D.dg_rasterize_bwd_records(vb, bg=tr.bg)
    torch.cuda.synchronize()
    args = (tr.anchor, tr.shared, tr.rho, tr.lr)
    ref = {n: getattr(tr, n).clone() for n in ("x", "m", "v", "z")}
    out = {n: getattr(tr, n).clone() for n in ("x", "m", "v", "z")}
    D.dg_xstep_part(0, vb, ref["x"], ref["m"], ref["v"], *args, step=2, z_unshared=ref["z"], gid=tr.gid)
    ws = D.xstep_stream_workspace(tr.x)
    ws.fill_(-1)                               # the call zeroes its own counters
    D.dg_xstep_groups(vb, tr.x, ws)
    torch.cuda.synchronize()
    n_groups = -(-tr.x.n // 128)
    n_idle, n_act = int(ws[0].item()), int(ws[1].item())
    assert n_idle + n_act == n_groups and 0 < n_idle < n_groups
    entries = ws[4:4 + n_groups].cpu().numpy()
    idle, act = entries[:n_idle], entries[n_groups - n_act:]
    assert sorted(np.concatenate([idle, act]).tolist()) == list(range(n_groups))
    rect = vb.rect.view(-1, 2)[:vb.n_rec].cpu().numpy().view(np.uint32)
    kept = np.zeros(tr.x.n, bool)
    vis = (rect[:, 0] & 0xFFFF) != (rect[:, 1] & 0xFFFF)
    for c in vb.host_cams:
        b, e = int(c.gauss_begin), int(c.gauss_end)
        kept[b:e] |= vis[int(c.rec_off):int(c.rec_off) + e - b]
    g_act = np.pad(kept, (0, n_groups * 128 - len(kept))).reshape(n_groups, 128).any(1)
    assert sorted(act.tolist()) == np.flatnonzero(g_act).tolist()
    D.dg_xstep_listed(1, vb, out["x"], out["m"], out["v"], *args, ws, step=2, ctas=ctas, z_unshared=out["z"],
                      gid=tr.gid)
    D.dg_xstep_listed(2, vb, out["x"], out["m"], out["v"], *args, ws, step=2, z_unshared=out["z"], gid=tr.gid)
    torch.cuda.synchronize()
    for n in ref:
        assert torch.equal(ref[n].data, out[n].data), n
    # the same lists serve the next step too, the parts in either order
    D.dg_xstep_part(0, vb, ref["x"], ref["m"], ref["v"], *args, step=3)
    D.dg_xstep_listed(2, vb, out["x"], out["m"], out["v"], *args, ws, step=3)
    D.dg_xstep_listed(1, vb, out["x"], out["m"], out["v"], *args, ws, step=3, ctas=ctas)
    torch.cuda.synchronize()
    for n in ("x", "m", "v"):
        assert torch.equal(ref[n].data, out[n].data), n


@pytest.mark.parametrize("mode,listed", [("stream", True), ("stream", False), ("grid", True), ("grid", False)])
def test_trainer_listed_part2_matches_one_part(mods, mode, listed):
    """Graph replays of the trainer with the idle part on the side stream,
    streamed or as a grid, and part 2 over the side stream's list or one CTA
    per group, equal the one-part step (up to the float atomics of the
    compositing adjoint)."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=43)
    kw = dict(rho=(1e-2,) * 5, loss="dssim", intv=2)
    a = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, overlap=True, **kw)
    a.idle_mode, a.listed_part2 = mode, listed
    a.calibrate_capacity()
    b = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, overlap=False, **kw)
    b.calibrate_capacity()
    for _ in range(5):
        a.step()
        b.step()
    torch.cuda.synchronize()
    for n in ("x", "z", "m"):
        ga, gb = groups(getattr(a, n)), groups(getattr(b, n))
        for k in ga:
            assert rel_l2(ga[k], gb[k]) < REL_L2, (n, k)


@pytest.mark.parametrize("consensus", [False, True])
def test_autotune_times_both_idle_forms_and_applies_the_faster(mods, consensus):
    """A reduced search (one tile shape, two variants): both side-stream
    forms are timed by replays, with or without the consensus, the faster
    one and the chosen variants are applied, and the tuned trainer keeps
    stepping without overflow."""
    D, srv, T = mods
    from paper_2405_13943_b300 import autotune
    wl, z0, targets = small_setup(D, srv, seed=47)
    tr = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, rho=(1e-2,) * 5, loss="dssim", intv=1)
    tr.calibrate_capacity()
    out = autotune.tune(tr, tiles=((16, 16),), warps=(1, 2), stages=(1,), steps=1, use_cache=False,
                        consensus=consensus)
    assert set(out["idle_modes"]) == {"stream", "grid"}
    assert all(0 < t < float("inf") for t in out["idle_modes"].values())
    assert out["idle_mode"] == min(out["idle_modes"], key=out["idle_modes"].get) == tr.idle_mode
    assert tuple(out["tile"]) == (16, 16) and tr.tile == (16, 16)
    assert not tr.graphs                       # the timing's graphs are dropped
    for _ in range(3):
        tr.step(consensus=consensus)
    torch.cuda.synchronize()
    assert not tr.overflowed()


@pytest.mark.parametrize("mode", ["stream", "grid"])
def test_overlapped_xstep_trainer_matches(mods, mode):
    """Graph replays with the idle part of the x-step on a side stream equal
    the one-part step (up to the float atomics of the compositing adjoint)."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=29)
    kw = dict(rho=(1e-2,) * 5, loss="dssim", intv=2)
    a = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, overlap=True, **kw)
    a.idle_mode = mode
    a.calibrate_capacity()
    b = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, overlap=False, **kw)
    b.calibrate_capacity()
    assert a._split_xstep() and not b._split_xstep()
    for _ in range(5):
        a.step()
        b.step()
    torch.cuda.synchronize()
    for n in ("x", "z", "m"):
        ga, gb = groups(getattr(a, n)), groups(getattr(b, n))
        for k in ga:
            assert rel_l2(ga[k], gb[k]) < REL_L2, (n, k)
    assert not a.overflowed()


def test_xstep_stores_unshared_copies_into_z(mods):
    """With z_unshared, the x-step's parts store every unshared copy's
    stepped value at its global id (what the consensus's z = x would write)
    and leave the shared globals of z alone; the trainer's consensus over the
    shared globals then gives the z of the full consensus."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=31)
    kw = dict(rho=(1e-2,) * 5, loss="dssim", intv=1)
    tr = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, **kw)
    tr.calibrate_capacity()
    assert tr._shared_first and tr._zfuse(True)
    tr.step(graph=False)
    vb = tr.vb
    vb.dev_cams.copy_(tr.cam_pool[tr.t % len(tr.view_sets)])
    D.dg_project(tr.x, vb)
    D.dg_bin_sort(vb)
    D.dg_rasterize_fwd(vb, tr.bg)
    tr._loss(tr.targets[tr.t % len(tr.view_sets)])
    D.dg_rasterize_bwd_records(vb, bg=tr.bg)
    torch.cuda.synchronize()
    args = (tr.anchor, tr.shared, tr.rho, tr.lr)
    z_before = tr.z.clone()
    x1, m1, v1 = tr.x.clone(), tr.m.clone(), tr.v.clone()
    D.dg_xstep_part(1, vb, x1, m1, v1, *args, step=2, z_unshared=tr.z, gid=tr.gid)
    D.dg_xstep_part(2, vb, x1, m1, v1, *args, step=2, z_unshared=tr.z, gid=tr.gid)
    torch.cuda.synchronize()
    xs, zs, zb = groups(x1), groups(tr.z), groups(z_before)
    sh = wl.split.copy_shared().astype(bool)
    gid = wl.split.copy_gid
    ns = int(wl.split.n_shared_globals)
    for k in xs:
        np.testing.assert_array_equal(zs[k][gid[~sh]], xs[k][~sh])
        np.testing.assert_array_equal(zs[k][:ns], zb[k][:ns])
    # trainer: consensus over the shared globals after the fused store equals the full consensus
    a = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, **kw)
    b = T.DogsTrainer(wl.split, z0.clone(), wl.views, targets, **kw)
    b._shared_first = False
    for t_ in (a, b):
        t_.calibrate_capacity()
    for _ in range(3):
        a.step()
        b.step()
    torch.cuda.synchronize()
    for n in ("z", "x", "u"):
        ga, gb = groups(getattr(a, n)), groups(getattr(b, n))
        for k in ga:
            assert rel_l2(ga[k], gb[k]) < REL_L2, (n, k)


def test_u8_host_targets_equal_device_targets(mods):
    """8-bit targets in pinned host memory (a quarter of the bytes over the
    link, widened to v / 255 on the device) give the losses and state of the
    same targets resident as float32."""
    D, srv, T = mods
    wl, z0, targets = small_setup(D, srv, seed=37)
    t8 = []
    for t in targets:
        b = torch.empty(t.numel(), dtype=torch.uint8, device="cuda")
        D.dg_image_f32_to_u8(t, b)
        t8.append(b)
    tf = []
    for b in t8:
        f = torch.empty(b.numel(), dtype=torch.float32, device="cuda")
        D.dg_image_u8_to_f32(b, f)
        tf.append(f)
    torch.cuda.synchronize()
    # the conversions: round(clamp(v) 255) and exactly v / 255
    ref8 = np.clip(np.rint(np.clip(targets[0].cpu().numpy(), 0, 1) * np.float32(255)), 0, 255).astype(np.uint8)
    np.testing.assert_array_equal(t8[0].cpu().numpy(), ref8)
    np.testing.assert_array_equal(tf[0].cpu().numpy(), ref8.astype(np.float32) / np.float32(255))
    kw = dict(rho=(1e-2,) * 5, loss="dssim", intv=2)
    a = T.DogsTrainer(wl.split, z0.clone(), wl.views, tf, **kw)
    a.calibrate_capacity()
    b = T.DogsTrainer(wl.split, z0.clone(), wl.views, tf, **kw)
    b.calibrate_capacity()
    b.use_host_targets([x.cpu() for x in t8])
    assert b.h2d_bytes_per_step() == t8[0].numel()
    for _ in range(4):
        a.step()
        b.step()
        # equal up to the order of the floating-point atomics of the loss sums and the adjoint
        np.testing.assert_allclose(b.last_loss().numpy(), a.vb.loss.cpu().numpy(), rtol=1e-6)
